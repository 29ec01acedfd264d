// Device-side helpers shared by the library's kernels (internal header).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hs {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kRadixBits = 9;          // radix digit width
constexpr int kBins = 1 << kRadixBits; // 512 digit values
constexpr uint32_t kFlagBit = 0x80000000u;  // "not exactly encoded" payload bit
constexpr uint32_t kIdxMask = 0x7FFFFFFFu;

// Device error word bits (DevFlags::error).
enum : uint32_t {
    kErrTimeout = 1u,    // a bounded look-back / queue wait gave up
    kErrOffsets = 2u,    // offsets decreasing
    kErrInternal = 4u,   // index out of range, capacity exceeded
};

// Small device-resident control block, zeroed at the start of every call.
struct DevFlags {
    unsigned int error;
    unsigned int nonexact;   // 1 if any string is not exactly represented
    unsigned int domain;     // 1 if ASCII7 saw a byte >= 0x80
    unsigned int nonconst;   // refinement: some large run is not constant
    unsigned long long qcount[8];   // run-queue lengths (see QueueId)
    unsigned long long kmin, kmax;  // range of the keys the encoder wrote (kmin preset to ~0)
    unsigned int active[16];        // plan: radix pass p is needed
    unsigned int alpha_lo_inv;      // byte-range coder: 255 - smallest byte of the strings (max-reduced)
    unsigned int alpha_hi;          // byte-range coder: largest byte of the strings
    unsigned int alpha_w, alpha_k;  // byte-range coder: bits per char and chars coded (written by the encoder)
    unsigned int alpha_spec_lo_inv, alpha_spec_hi;  // byte-range coder: the range a speculative encode used
    unsigned int idx_packed;        // byte-range coder: codes written as (code << idx_bits) | index
    unsigned int descent;           // sorted-input test: some string is smaller than its predecessor
    unsigned long long pairs;       // sorted-input test: adjacent pairs left to a full comparison
    unsigned int pad[2];
    unsigned long long dirty_lo, dirty_hi;  // fix-up: permutation positions rewritten (lo preset to ~0)
};

// Run queue entry: a run of equal keys at positions [start, start + len)
// whose members agree on their first byte_offset(depth) bytes.
struct RunEntry {
    unsigned long long start;
    unsigned int len;
    unsigned int depth;
};

// Decoupled look-back words: a 6-bit epoch in bits 58..63 (which launch
// wrote the word; 0 = never written), a 2-bit status in bits 56..57
// (aggregate of this tile only / inclusive prefix), a 56-bit value.  Words
// from earlier launches carry another epoch and read as "not ready", so the
// array is cleared once per call rather than once per pass.
constexpr uint64_t kLbAggregate = 1ull << 56;
constexpr uint64_t kLbInclusive = 2ull << 56;
constexpr uint64_t kLbValueMask = (1ull << 56) - 1;
constexpr uint32_t kLbEpochs = 63;          // usable epochs 1..63
constexpr uint32_t kSpinLimit = 1u << 22;   // polls before a wait gives up

__host__ __device__ __forceinline__ uint64_t lb_word(uint32_t epoch, uint64_t status, uint64_t value) {
    return ((uint64_t)epoch << 58) | status | (value & kLbValueMask);
}

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Asynchronous global -> shared copies (no registers held while in flight).
// cp_async8/16 copy 8/16 bytes from naturally aligned addresses; with
// src_bytes = 0 the destination is zero-filled and nothing is read.
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src, unsigned src_bytes = 8) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem_src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp whose radix digit equals this lane's, restricted to
// `active`, from the hardware match instruction.  Call with the full warp
// converged (lanes outside `active` pass any digit).  Its cost grows with the
// number of distinct digits in the warp; match_by_ballots below costs the
// same always.
__device__ __forceinline__ unsigned match_digit(unsigned d, unsigned active) {
    return __match_any_sync(kFull, d) & active;
}

// The same peer mask from one ballot per digit bit, for digits below 2^9.
// Always nine ballots: where a pass's digits are narrower, their upper bits
// are 0 in every lane, those ballots are 0 and change nothing, and a
// runtime bound on the loop measured 10% slower in onesweep.  Its cost is
// fixed, where the match instruction's grows with the number of distinct
// values the warp holds (see prefer_ballots).  Call with the full warp
// converged.
__device__ __forceinline__ unsigned match_by_ballots(unsigned d) {
    unsigned diff = 0;
#pragma unroll
    for (int j = 0; j < kRadixBits; ++j) {
        const unsigned t = 0u - ((d >> j) & 1u);  // all ones where bit j is set
        diff |= __ballot_sync(kFull, t != 0u) ^ t;
    }
    return ~diff;
}

// Whether a warp ranks its items with ballots rather than the match
// instruction, from the match result `peers` of one of its items: the
// leaders of the equal-digit groups count the warp's distinct digits, and
// at kBallotDistinct or more the nine ballots cost less (measured on
// GB300).  Call with the full warp converged.
constexpr unsigned kBallotDistinct = 21;
__device__ __forceinline__ bool prefer_ballots(unsigned peers) {
    return (unsigned)__popc(__ballot_sync(kFull, (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1))) >= kBallotDistinct;
}

// Shared-memory histogram increment of digit d: when the whole warp holds
// the same digit (constant or low-entropy digits), one add of the lane count
// replaces 32 contending atomics.  Call with the full warp converged; lanes
// with valid == false contribute nothing.
__device__ __forceinline__ void hist_add(uint32_t *hist, unsigned d, bool valid) {
    const unsigned active = __ballot_sync(kFull, valid);
    if (active == 0) return;
    const int src = __ffs(active) - 1;
    const unsigned d0 = __shfl_sync(kFull, d, src);
    const bool same = __all_sync(kFull, !valid || d == d0);
    if (same) {
        if ((threadIdx.x & 31) == (unsigned)src) atomicAdd(&hist[d0], (uint32_t)__popc(active));
    } else if (valid) {
        atomicAdd(&hist[d], 1u);
    }
}

// Byte offset at which refinement depth `depth` starts comparing: the first
// `prefix_len` bytes are covered by the husky code, each later depth by a
// 7-byte window.
__device__ __forceinline__ uint64_t window_offset(int prefix_len, uint32_t depth) {
    return (uint64_t)prefix_len + 7ull * depth;
}

// Refinement key of a string of length len at byte offset o: the 7 bytes
// [o, o+7) big-endian (zero padded) in bits 5..60 and a tag in bits 0..4,
//   tag = min(len + prefix_len - o, prefix_len + 8)   (at most 17 < 32).
// Among strings that agree on their first o bytes (or, at o = prefix_len,
// share a husky code), unsigned key order is lexicographic order on the
// window; equal keys with tag < prefix_len + 8 mean identical strings; tag ==
// prefix_len + 8 means both continue past the window.  The key fits in 61
// bits, so it sorts in seven 9-bit digits.
constexpr int kTagBits = 5;
__device__ __forceinline__ uint32_t window_tag(uint64_t key) { return (uint32_t)(key & ((1u << kTagBits) - 1)); }

__device__ __forceinline__ uint64_t window_key(const uint8_t *s, uint64_t len,
                                               uint64_t o, int prefix_len) {
    // Only the bytes that exist are loaded (a runtime-bounded loop); the rest
    // of the window stays zero.
    const uint64_t avail = len > o ? len - o : 0;
    const uint32_t m = avail < 7 ? (uint32_t)avail : 7u;
    uint64_t key = 0;
    for (uint32_t i = 0; i < m; ++i) key |= (uint64_t)s[o + i] << (8 * (6 - i));
    int64_t t = (int64_t)len + prefix_len - (int64_t)o;
    int64_t cap = prefix_len + 8;
    if (t > cap) t = cap;
    if (t < 0) t = 0;
    return (key << kTagBits) | (uint64_t)t;
}

// Three-way unsigned-byte comparison of a and b starting at byte `from`
// (both strings agree before it).
// True iff strings (a, la) and (b, lb) are equal, given that they already
// agree on their first `from` bytes (members of one run of equal keys).
__device__ __forceinline__ bool equal_from(const uint8_t *a, uint64_t la, const uint8_t *b, uint64_t lb,
                                           uint64_t from) {
    if (la != lb) return false;
    for (uint64_t i = from; i < la; ++i)
        if (a[i] != b[i]) return false;
    return true;
}

// Bytes [from, min(len, from + 8)) of a string as a little-endian word, each
// loaded independently (no chain of early exits).
__device__ __forceinline__ uint64_t suffix_word(const uint8_t *s, uint64_t len, uint64_t from) {
    uint64_t x = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (from + k < len) x |= (uint64_t)s[from + k] << (8 * k);
    return x;
}

// Two strings of length len agree on [from, len), given their suffix words
// (bytes from .. from + 7); the rest is compared bytewise.
__device__ __forceinline__ bool same_from(const uint8_t *a, const uint8_t *b, uint64_t len, uint64_t from,
                                          uint64_t wa, uint64_t wb) {
    if (wa != wb) return false;
    for (uint64_t i = from + 8; i < len; ++i)
        if (a[i] != b[i]) return false;
    return true;
}

// Positions [start, start + len) of the permutation were rewritten.
__device__ __forceinline__ void mark_dirty(DevFlags *flags, uint64_t start, uint64_t len) {
    if (flags == nullptr || len == 0) return;
    atomicMin(&flags->dirty_lo, (unsigned long long)start);
    atomicMax(&flags->dirty_hi, (unsigned long long)(start + len - 1));
}

__device__ __forceinline__ int compare_from(const uint8_t *a, uint64_t la,
                                            const uint8_t *b, uint64_t lb,
                                            uint64_t from) {
    uint64_t m = la < lb ? la : lb;
    for (uint64_t i = from; i < m; ++i) {
        unsigned ca = a[i], cb = b[i];
        if (ca != cb) return ca < cb ? -1 : 1;
    }
    return la < lb ? -1 : (la > lb ? 1 : 0);
}

}  // namespace hs
