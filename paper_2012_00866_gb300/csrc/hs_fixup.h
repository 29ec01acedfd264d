// Host-side interface of the refinement's dense window array (fixup.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hs_internal.h"

namespace hs {

// win[i] = the window key of string i (bytes offsets[i] .. offsets[i+1]) at
// refinement depth `depth`: the 7 bytes from window_offset(prefix_len,
// depth) and the length tag, as window_key gives them.  One pass in string
// order over all n strings.  win holds n words.
cudaError_t launch_window_dense(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, int prefix_len,
                                uint32_t depth, uint64_t *win, int num_sms, cudaStream_t s);

// launch_refine_keys, with each member's window key (and its run's first
// member's) read from win (launch_window_dense at win_depth) for runs at
// depth win_depth instead of gathered from the member's offsets and bytes.
// win == nullptr: every member is gathered.
cudaError_t launch_refine_keys_win(const uint8_t *bytes, const uint64_t *offsets, const void *perm, int perm_u64,
                                   const RunEntry *runs, uint64_t count, const unsigned long long *run_base,
                                   uint64_t total, Instances inst, int prefix_len, const uint64_t *win,
                                   uint32_t win_depth, uint64_t *keys, uint32_t *segs, uint32_t *vals,
                                   DevFlags *flags, cudaStream_t s);

}  // namespace hs
