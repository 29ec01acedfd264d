// Host-side interface of bignum.cu (the BigInteger coder).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hs_device.cuh"

namespace hs {

// Values longer than this many bytes are rejected (the header holds L).
constexpr uint64_t kBigMaxLen = 32767;

// For each of n big integers (minimal two's complement, big-endian, bytes
// offsets[i] .. offsets[i+1]) writes the byte string header(L) || value to
// out_bytes at out_offsets[i] = (offsets[i] - offsets[0]) + 2i, where L is
// the value's length and header(L) = the big-endian u16 0x8000 + L for a
// value >= 0, 0x7FFF - L for a value < 0.  out_offsets[n] closes the last.
// Unsigned-byte order of these strings is the values' numeric order, and
// equal values give equal strings.  An empty, non-minimal or too long value,
// or one that would end past out_cap bytes, is not written and sets
// flags->error |= kErrOffsets.
cudaError_t launch_bigint_encode(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, uint8_t *out_bytes,
                                 uint64_t out_cap, uint64_t *out_offsets, DevFlags *flags, int num_sms,
                                 cudaStream_t s);

}  // namespace hs
