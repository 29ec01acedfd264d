// Step 1: husky encoding (Algorithm 4 stringToLong; Algorithms 2/3 over the
// array with the per-element perfection test; Section 4.3 asciiToLong and
// constants: 7 bits x 64/7 = 9 chars, mask 0x7F).
//
// One pass over offsets and bytes produces, per string i, the code (or the
// sort key (code << 1) | not_exact, see below), the "not exactly represented"
// bit, and -- fused so the keys are not read back -- the digit histograms the
// radix sort needs up front.
//
// Sort key.  Under ASCII7 the code uses 63 bits.  Appending the not-exact bit
// below it keeps the order of distinct codes and, among equal codes, puts the
// exactly represented string first -- its true place, since an exact member
// of a run of equal codes is a prefix of every other member (they agree on
// the first 9 chars, and the exact one ends there or earlier).  Runs of equal
// sort keys then either consist of identical strings (bit 0 clear: already in
// index order after a stable sort) or need the fix-up (bit 0 set).
//
// Layout: a CTA takes a tile of 1024 consecutive strings.  Their offsets are
// loaded coalesced into shared memory; their bytes, which are contiguous,
// are staged into shared memory with 16-byte vector loads when the tile's
// byte range fits (the common case for words); otherwise each thread reads
// its own string's first maxLength bytes from global memory.  The grid is a
// multiple of the SM count and loops over tiles.
#include "hs_internal.h"

namespace hs {
namespace {

constexpr int kEncThreads = 256;
constexpr int kEncTile = 1024;
constexpr int kEncItems = kEncTile / kEncThreads;
constexpr int kEncStage = 28672;   // staged bytes per tile
constexpr int kEncHistPasses = kKeyPasses;
constexpr size_t kEncOffBytes = (((size_t)kEncTile + 1) * 8 + 15) & ~(size_t)15;  // keeps s_bytes 16-B aligned
constexpr size_t kEncSmem = kEncOffBytes + kEncStage + (size_t)kEncHistPasses * kBins * 4;
static_assert(kEncStage % 16 == 0, "staging buffer must keep 16-byte alignment");

template <int CODER> struct CoderTraits;
template <> struct CoderTraits<1> {   // ASCII7
    static constexpr int K = 9, W = 7;
    static constexpr unsigned MASK = 0x7F;
};
template <> struct CoderTraits<2> {   // BYTE8
    static constexpr int K = 8, W = 8;
    static constexpr unsigned MASK = 0xFF;
};

template <int CODER, bool KEYFLAG>
__global__ void __launch_bounds__(kEncThreads)
encode_kernel(const uint8_t *__restrict__ bytes,
              const uint64_t *__restrict__ offsets, uint64_t n,
              uint64_t *__restrict__ codes, uint32_t *__restrict__ nonexact_bits,
              unsigned long long *__restrict__ hist, DevFlags *flags) {
    using C = CoderTraits<CODER>;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_off = reinterpret_cast<uint64_t *>(smem);
    uint8_t *s_bytes = smem + kEncOffBytes;
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_bytes + kEncStage);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t total = offsets[n];
    const uintptr_t base = reinterpret_cast<uintptr_t>(bytes);

    if (hist)
        for (int i = tid; i < kEncHistPasses * kBins; i += kEncThreads) s_hist[i] = 0;

    bool any_nonexact = false, any_domain = false;
    uint64_t kmin = ~0ull, kmax = 0;
    const uint64_t num_tiles = (n + kEncTile - 1) / kEncTile;
    for (uint64_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
        const uint64_t t0 = tile * kEncTile;
        const int cnt = (int)umin64(kEncTile, n - t0);
        __syncthreads();
        for (int i = tid; i <= cnt; i += kEncThreads) s_off[i] = offsets[t0 + i];
        __syncthreads();
        // Offsets must be non-decreasing and end inside the byte buffer;
        // a tile that fails reads no bytes.
        bool bad = false;
        for (int i = tid; i < cnt; i += kEncThreads) bad |= s_off[i + 1] < s_off[i];
        if (tid == 0) bad |= s_off[cnt] > total;
        if (__syncthreads_or(bad)) {
            if (tid == 0) atomicOr(&flags->error, kErrOffsets);
            continue;
        }
        const uint64_t lo = s_off[0], hi = s_off[cnt];
        const uintptr_t a0 = (base + lo) & ~uintptr_t(15);
        const uintptr_t a1 = (base + hi + 15) & ~uintptr_t(15);
        const bool staged = (a1 - a0) <= (uintptr_t)kEncStage;
        if (staged) {
            const int chunks = (int)((a1 - a0) >> 4);
            for (int c = tid; c < chunks; c += kEncThreads) {
                const uintptr_t a = a0 + 16 * (uintptr_t)c;
                if (a >= base && a + 16 <= base + total) {
                    *reinterpret_cast<uint4 *>(s_bytes + 16 * c) =
                        __ldg(reinterpret_cast<const uint4 *>(a));
                } else {  // chunk straddles the buffer ends: bytewise
                    for (int b = 0; b < 16; ++b) {
                        const uintptr_t q = a + b;
                        s_bytes[16 * c + b] =
                            (q >= base && q < base + total) ? *reinterpret_cast<const uint8_t *>(q) : 0;
                    }
                }
            }
        }
        __syncthreads();

#pragma unroll
        for (int k = 0; k < kEncItems; ++k) {
            const int j = k * kEncThreads + tid;   // a warp covers 32 consecutive strings
            const bool valid = j < cnt;
            uint64_t code = 0;
            bool exact = true;
            if (valid) {
                const uint64_t off = s_off[j];
                const uint64_t len = s_off[j + 1] - off;
                const int m = (int)umin64(len, C::K);
                const uint8_t *src = staged ? s_bytes + (base + off - a0) : bytes + off;
                unsigned last = 0;
                for (int i = 0; i < m; ++i) {
                    const unsigned c = src[i];
                    if (CODER == 1) any_domain |= c >= 0x80u;
                    code = (code << C::W) | (uint64_t)(c & C::MASK);
                    last = c;
                }
                const int shift = C::W * (C::K - m);
                code = shift >= 64 ? 0 : (code << shift);
                exact = len <= (uint64_t)C::K && (len == 0 || last != 0);
                if (KEYFLAG) code = (code << 1) | (exact ? 0u : 1u);
                codes[t0 + j] = code;
                kmin = code < kmin ? code : kmin;
                kmax = code > kmax ? code : kmax;
            }
            if (hist) {  // whole warp converged here
#pragma unroll
                for (int p = 0; p < kEncHistPasses; ++p)
                    hist_add(s_hist + p * kBins, (unsigned)((code >> digit_shift(p)) & digit_mask(p)), valid);
            }
            const unsigned ne = __ballot_sync(kFull, valid && !exact);
            any_nonexact |= valid && !exact;
            const uint64_t w0 = t0 + (uint64_t)k * kEncThreads + (uint64_t)warp * 32;
            if (nonexact_bits && lane == 0 && w0 < n) nonexact_bits[w0 >> 5] = ne;
        }
    }
    __syncthreads();
    if (hist)
        for (int i = tid; i < kEncHistPasses * kBins; i += kEncThreads)
            if (s_hist[i]) atomicAdd(&hist[i], (unsigned long long)s_hist[i]);
    any_nonexact = __syncthreads_or(any_nonexact);
    any_domain = __syncthreads_or(any_domain);
    if (tid == 0) {
        if (any_nonexact) atomicOr(&flags->nonexact, 1u);
        if (any_domain) atomicOr(&flags->domain, 1u);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t a = __shfl_xor_sync(kFull, kmin, o), b = __shfl_xor_sync(kFull, kmax, o);
        kmin = a < kmin ? a : kmin;
        kmax = b > kmax ? b : kmax;
    }
    if (lane == 0 && kmin <= kmax) {
        atomicMin(&flags->kmin, (unsigned long long)kmin);
        atomicMax(&flags->kmax, (unsigned long long)kmax);
    }
}

template <int CODER, bool KEYFLAG>
cudaError_t launch_enc(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, uint64_t *codes,
                       uint32_t *nonexact_bits, unsigned long long *hist, DevFlags *flags, unsigned grid,
                       cudaStream_t s) {
    auto kern = encode_kernel<CODER, KEYFLAG>;
    static bool configured = false;  // attribute is per function, idempotent
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEncSmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    kern<<<grid, kEncThreads, kEncSmem, s>>>(bytes, offsets, n, codes, nonexact_bits, hist, flags);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_encode(int coder, bool key_flag, const uint8_t *bytes,
                          const uint64_t *offsets, uint64_t n, uint64_t *codes,
                          uint32_t *nonexact_bits, unsigned long long *hist,
                          DevFlags *flags, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t tiles = (n + kEncTile - 1) / kEncTile;
    const unsigned grid = (unsigned)umin64(tiles, (uint64_t)num_sms * 4);
    if (coder == 2) {
        if (key_flag) return cudaErrorInvalidValue;  // BYTE8 codes use all 64 bits
        return launch_enc<2, false>(bytes, offsets, n, codes, nonexact_bits, hist, flags, grid, s);
    }
    if (key_flag) return launch_enc<1, true>(bytes, offsets, n, codes, nonexact_bits, hist, flags, grid, s);
    return launch_enc<1, false>(bytes, offsets, n, codes, nonexact_bits, hist, flags, grid, s);
}

}  // namespace hs
