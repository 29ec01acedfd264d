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
// copied into shared memory and their bytes, which are contiguous, staged
// there in aligned 16-byte pieces when the tile's byte range fits (the
// common case for words), all with asynchronous copies that are in flight
// together; otherwise each thread reads its own string's first maxLength
// bytes from global memory.  A staged string's code is built from two
// aligned words of the stage.  The grid is a multiple of the SM count and
// loops over tiles.
#include "hs_internal.h"

namespace hs {
namespace {

constexpr int kEncThreads = 256;
constexpr int kEncTile = 1024;
constexpr int kEncItems = kEncTile / kEncThreads;
constexpr int kEncStage = 28672;   // staged bytes per tile
constexpr int kEncHistPasses = kKeyPasses;
constexpr size_t kEncOffBytes = (((size_t)kEncTile + 1) * 8 + 15) & ~(size_t)15;  // keeps s_bytes 16-B aligned
constexpr int kEncPad = 16;        // word reads of the last staged string may run 15 bytes past the stage
constexpr size_t kEncSmem = kEncOffBytes + kEncStage + kEncPad + (size_t)kEncHistPasses * kBins * 4;
static_assert(kEncStage % 16 == 0, "staging buffer must keep 16-byte alignment");

template <int CODER> struct CoderTraits;
template <> struct CoderTraits<1> {   // ASCII7
    static constexpr int K = 9, W = 7;
    static constexpr unsigned MASK = 0x7F;
};
template <> struct CoderTraits<3> {   // alphabet coder when it does not apply: ASCII7
    static constexpr int K = 9, W = 7;
    static constexpr unsigned MASK = 0x7F;
};
template <> struct CoderTraits<2> {   // BYTE8
    static constexpr int K = 8, W = 8;
    static constexpr unsigned MASK = 0xFF;
};

// Bytes b[0..7] of a little-endian word in the code's order (b[0] most
// significant), each cut to its low 7 bits and packed into 56 bits: the
// stringToLong loop of Algorithm 4 for eight ASCII7 chars at once.
__device__ __forceinline__ uint64_t pack7x8(uint64_t x) {
    uint64_t t = __byte_perm((uint32_t)(x >> 32), 0, 0x0123) |
                 ((uint64_t)__byte_perm((uint32_t)x, 0, 0x0123) << 32);   // byte swap
    t &= 0x7F7F7F7F7F7F7F7Full;
    t = (t & 0x007F007F007F007Full) | ((t & 0x7F007F007F007F00ull) >> 1);  // 14-bit pairs
    t = (t & 0x00003FFF00003FFFull) | ((t & 0x3FFF00003FFF0000ull) >> 2);  // 28-bit quads
    t = (t & 0x000000000FFFFFFFull) | ((t & 0x0FFFFFFF00000000ull) >> 4);  // 56 bits
    return t;
}

// Code, exactness and (ASCII7) domain bit of a string whose first bytes are
// the little-endian words w0 (bytes 0..7) and b8 (byte 8), length len.
template <int CODER>
__device__ __forceinline__ uint64_t code_from_words(uint64_t w0, unsigned b8, uint64_t len, bool &exact,
                                                    bool &domain) {
    using C = CoderTraits<CODER>;
    const int m = (int)umin64(len, C::K);
    if (m == 0) {
        exact = true;
        domain = false;
        return 0;
    }
    const uint64_t low = m >= 8 ? ~0ull : ((1ull << (8 * m)) - 1);   // the first min(m, 8) bytes
    const unsigned last = m == 9 ? b8 : (unsigned)(w0 >> (8 * (m - 1))) & 0xFFu;
    exact = len <= (uint64_t)C::K && last != 0;
    uint64_t code;
    if (CODER == 1) {
        domain = ((w0 & low) & 0x8080808080808080ull) != 0 || (m == 9 && (b8 & 0x80u));
        code = (pack7x8(w0) << 7) | (b8 & 0x7Fu);          // nine chars, 63 bits
        const int sh = 7 * (9 - m);
        code = (code >> sh) << sh;                         // chars past m are padding zeros
    } else {
        domain = false;
        code = (uint64_t)__byte_perm((uint32_t)(w0 >> 32), 0, 0x0123) |
               ((uint64_t)__byte_perm((uint32_t)w0, 0, 0x0123) << 32);
        const int sh = 8 * (8 - m);
        code = sh >= 64 ? 0 : ((code >> sh) << sh);
    }
    return code;
}

// Histogram add of digit d for a full warp (every lane valid): one match
// finds whether all lanes hold the same digit, in which case one add of 32
// replaces 32 contending atomics.
__device__ __forceinline__ void hist_add_full(uint32_t *hist, unsigned d) {
    int same;
    __match_all_sync(kFull, d, &same);
    if (same) {
        if ((threadIdx.x & 31) == 0) atomicAdd(&hist[d], 32u);
    } else {
        atomicAdd(&hist[d], 1u);
    }
}

// ---- byte range (coder 3) ----------------------------------------------------
// The byte-range coder (this library's generalisation of the 5-bit and 6-bit
// letter codings of Section 3.2) needs the smallest and largest byte of the
// string data first: one streaming pass, four bytes per SIMD min/max, four
// 16-byte pieces per thread in flight.  A thread whose own bytes already
// span more than max_span values stops: the range is too wide for the coder
// either way, and the reduced range still shows it.

constexpr int kAlphaThreads = 256;

__global__ void __launch_bounds__(kAlphaThreads)
alphabet_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets, uint64_t n,
                int max_span, DevFlags *flags) {
    const uint64_t b0 = offsets[0], b1 = offsets[n];
    uint32_t vmin = 0xFFFFFFFFu, vmax = 0;  // four byte lanes each
    if (b1 > b0) {
        const uintptr_t lo = reinterpret_cast<uintptr_t>(bytes) + b0, hi = reinterpret_cast<uintptr_t>(bytes) + b1;
        const uintptr_t a0 = lo & ~uintptr_t(15);
        const uint64_t chunks = (uint64_t)((hi - a0 + 15) >> 4);
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        constexpr int kPer = 4;
        for (uint64_t c0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c0 < chunks; c0 += stride * kPer) {
            uint4 v[kPer];
            bool whole[kPer];
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const uint64_t ch = c0 + u * stride;
                const uintptr_t a = a0 + 16 * (uintptr_t)ch;
                whole[u] = ch < chunks && a >= lo && a + 16 <= hi;
                v[u] = whole[u] ? __ldg(reinterpret_cast<const uint4 *>(a)) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const uint64_t ch = c0 + u * stride;
                if (whole[u]) {
                    vmin = __vminu4(__vminu4(vmin, v[u].x), __vminu4(v[u].y, __vminu4(v[u].z, v[u].w)));
                    vmax = __vmaxu4(__vmaxu4(vmax, v[u].x), __vmaxu4(v[u].y, __vmaxu4(v[u].z, v[u].w)));
                } else if (ch < chunks) {  // the ragged ends: only the bytes inside [lo, hi)
                    const uintptr_t a = a0 + 16 * (uintptr_t)ch;
                    for (int b = 0; b < 16; ++b) {
                        const uintptr_t q = a + b;
                        if (q >= lo && q < hi) {
                            const uint32_t c4 = *reinterpret_cast<const uint8_t *>(q) * 0x01010101u;
                            vmin = __vminu4(vmin, c4);
                            vmax = __vmaxu4(vmax, c4);
                        }
                    }
                }
            }
            const uint32_t m2 = __vminu4(vmin, vmin >> 16), x2 = __vmaxu4(vmax, vmax >> 16);
            const int span = (int)max(x2 & 0xFFu, (x2 >> 8) & 0xFFu) - (int)min(m2 & 0xFFu, (m2 >> 8) & 0xFFu) + 1;
            if (span > max_span) break;
        }
    }
    const uint32_t mn = __vminu4(vmin, vmin >> 16), mx = __vmaxu4(vmax, vmax >> 16);
    const uint32_t mn1 = min(mn & 0xFFu, (mn >> 8) & 0xFFu), mx1 = max(mx & 0xFFu, (mx >> 8) & 0xFFu);
    const uint32_t wmn = __reduce_min_sync(kFull, mn1), wmx = __reduce_max_sync(kFull, mx1);
    if ((threadIdx.x & 31) == 0) {
        if (wmn < 256u && 255u - wmn > 0u) atomicMax(&flags->alpha_lo_inv, 255u - wmn);
        if (wmx > 0u) atomicMax(&flags->alpha_hi, wmx);
    }
}

// Bytes of a little-endian word in code order (byte 0 most significant),
// each a value below 2^w, packed into 8w bits: the stringToLong loop of
// Algorithm 4 for eight chars at once (w = 7 is pack7x8 without the mask).
__device__ __forceinline__ uint64_t pack_w(uint64_t x, int w) {
    uint64_t t = __byte_perm((uint32_t)(x >> 32), 0, 0x0123) |
                 ((uint64_t)__byte_perm((uint32_t)x, 0, 0x0123) << 32);   // byte swap
    t = (t & 0x00FF00FF00FF00FFull) | ((t & 0xFF00FF00FF00FF00ull) >> (8 - w));
    t = (t & 0x0000FFFF0000FFFFull) | ((t & 0xFFFF0000FFFF0000ull) >> (16 - 2 * w));
    t = (t & 0x00000000FFFFFFFFull) | ((t & 0xFFFFFFFF00000000ull) >> (32 - 4 * w));
    return t;
}


template <int CODER, bool KEYFLAG>
__global__ void __launch_bounds__(kEncThreads)
encode_kernel(const uint8_t *__restrict__ bytes,
              const uint64_t *__restrict__ offsets, uint64_t n,
              uint64_t *__restrict__ codes, uint32_t *__restrict__ nonexact_bits,
              unsigned long long *__restrict__ hist, DevFlags *flags, int alpha_max_w, int alpha_max_bits,
              EncPack pk) {
    using C = CoderTraits<CODER>;
    constexpr int CW = CODER == 3 ? 1 : CODER;  // word path: the coder itself, ASCII7 for coder 3
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *s_off = reinterpret_cast<uint64_t *>(smem);
    uint8_t *s_bytes = smem + kEncOffBytes;
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_bytes + kEncStage + kEncPad);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t total = offsets[n];
    const uintptr_t base = reinterpret_cast<uintptr_t>(bytes);

    if (hist)
        for (int i = tid; i < kEncHistPasses * kBins; i += kEncThreads) s_hist[i] = 0;

    // Coder 3: byte c codes as c - lo + 1 over the data's byte range
    // [lo, hi] (0 is the padding), w = ceil(log2(hi - lo + 2)) bits each,
    // K = 8 chars: a sort key of 8w + 1 bits.  Past alpha_max_w bits, or
    // when the key does not fit alpha_max_bits (room the caller keeps above
    // it), it is not applied and the kernel encodes as ASCII7.
    int aw = 7, ak = 9;
    bool alpha = false;
    uint32_t alo4 = 0;
    // c - lo + 1 for all eight bytes of a word at once: x + d8 with d8 the
    // byte (1 - lo) repeated, as one 64-bit add.  No byte of the string
    // carries or borrows (lo <= c <= hi and hi - lo + 1 < 2^w <= 64), and
    // the bytes past its end, which may, sit above it and are cleared.
    uint64_t d8 = 0;
    if (CODER == 3) {
        int lo = 255 - (int)(pk.spec_range ? flags->alpha_spec_lo_inv : flags->alpha_lo_inv);
        int hi = (int)(pk.spec_range ? flags->alpha_spec_hi : flags->alpha_hi);
        if (hi < lo) lo = hi = 0;  // no bytes at all
        int w = 1;
        while ((1 << w) < hi - lo + 2) ++w;
        const int k = 8;
        alpha = w <= alpha_max_w && k * w + 1 <= alpha_max_bits;
        aw = w;
        ak = k;
        alo4 = (uint32_t)((lo - 1) & 0xFF) * 0x01010101u;
        d8 = (uint64_t)(int64_t)(1 - lo) * 0x0101010101010101ull;
        if (blockIdx.x == 0 && tid == 0) {
            flags->alpha_w = (unsigned)w;
            flags->alpha_k = (unsigned)k;
        }
    }

    // Digits above the key's width are zero for every string: counted in
    // bin 0 once per tile instead of per string (the byte-range coder's
    // K*w + 1 bits; the other keys use all eight digits).
    // Batched, byte-range coder: the instance id goes above the code.
    // Single sort, byte-range coder: the string's index goes below it when
    // both fit one word (the not-exact bit then stays out of the key).
    const bool pack = CODER == 3 && alpha && pk.seg_offsets != nullptr;
    const bool pack_idx = CODER == 3 && alpha && !pack && pk.idx_bits > 0 && ak * aw + pk.idx_bits <= 64;
    if (CODER == 3 && blockIdx.x == 0 && tid == 0) flags->idx_packed = pack_idx ? 1u : 0u;
    const int code_bits = (CODER == 3 && alpha) ? ak * aw + ((KEYFLAG && !pack_idx) ? 1 : 0) : 64;
    const int key_bits = pack ? code_bits + pk.seg_bits : code_bits;
    int hist_digits = kEncHistPasses;
    while (hist_digits > 0 && digit_shift(hist_digits - 1) >= key_bits) --hist_digits;

    bool any_nonexact = false, any_domain = false, any_bad_local = false;
    uint64_t kmin = ~0ull, kmax = 0;
    const uint64_t num_tiles = (n + kEncTile - 1) / kEncTile;
    for (uint64_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
        const uint64_t t0 = tile * kEncTile;
        const int cnt = (int)umin64(kEncTile, n - t0);
        __syncthreads();
        for (int i = tid; i <= cnt; i += kEncThreads) cp_async8(&s_off[i], offsets + t0 + i);
        cp_async_wait_all();
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
        if (hist && tid == 0)
            for (int p = hist_digits; p < kEncHistPasses; ++p) atomicAdd(&s_hist[p * kBins], (uint32_t)cnt);
        const uint64_t lo = s_off[0], hi = s_off[cnt];
        const uintptr_t a0 = (base + lo) & ~uintptr_t(15);
        const uintptr_t a1 = (base + hi + 15) & ~uintptr_t(15);
        const bool staged = (a1 - a0) <= (uintptr_t)kEncStage;
        if (staged) {
            const int chunks = (int)((a1 - a0) >> 4);
            for (int c = tid; c < chunks; c += kEncThreads) {
                const uintptr_t a = a0 + 16 * (uintptr_t)c;
                if (a >= base && a + 16 <= base + total) {
                    cp_async16(s_bytes + 16 * c, reinterpret_cast<const void *>(a));
                } else {  // chunk straddles the buffer ends: bytewise
                    for (int b = 0; b < 16; ++b) {
                        const uintptr_t q = a + b;
                        s_bytes[16 * c + b] =
                            (q >= base && q < base + total) ? *reinterpret_cast<const uint8_t *>(q) : 0;
                    }
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();

#pragma unroll
        for (int k = 0; k < kEncItems; ++k) {
            const int j = k * kEncThreads + tid;   // a warp covers 32 consecutive strings
            const bool valid = j < cnt;
            uint64_t code = 0, hkey = 0;  // hkey: the key the digit histograms count
            bool exact = true;
            if (valid) {
                const uint64_t off = s_off[j];
                const uint64_t len = s_off[j + 1] - off;
                if (CODER == 3 && alpha) {
                    const int m = (int)umin64(len, (uint64_t)ak);
                    if (staged) {
                        // bytes q .. q+7 from the two aligned words at q & ~7,
                        // mapped to c - lo + 1, bytes past m cleared, packed
                        const uint32_t q = (uint32_t)(base + off - a0);
                        const uint64_t *wp = reinterpret_cast<const uint64_t *>(s_bytes + (q & ~7u));
                        const uint64_t x0 = wp[0], x1 = wp[1];
                        const int r = 8 * (int)(q & 7u);
                        const uint64_t w0 = r ? (x0 >> r) | (x1 << (64 - r)) : x0;
                        const uint64_t keep = m >= 8 ? ~0ull : ((1ull << (8 * m)) - 1);
                        code = pack_w((w0 + d8) & keep, aw);  // the 8 chars, 8w bits
                    } else {
                        const uint8_t *src = staged ? s_bytes + (uint32_t)(base + off - a0) : bytes + off;
                        const unsigned lo1 = (alo4 & 0xFFu);
                        for (int i = 0; i < m; ++i) code = (code << aw) | (uint64_t)((src[i] - lo1) & 0xFFu);
                        code <<= aw * (ak - m);  // ak * aw <= 63
                    }
                    exact = len <= (uint64_t)ak;
                } else if (staged) {
                    // the two aligned words holding bytes q .. q+15 of the stage
                    const uint32_t q = (uint32_t)(base + off - a0);
                    const uint64_t *wp = reinterpret_cast<const uint64_t *>(s_bytes + (q & ~7u));
                    const uint64_t lo = wp[0], hi = wp[1];
                    const int r = 8 * (int)(q & 7u);
                    const uint64_t w0 = r ? (lo >> r) | (hi << (64 - r)) : lo;
                    const unsigned b8 = (unsigned)(hi >> r) & 0xFFu;
                    bool dom;
                    code = code_from_words<CW>(w0, b8, len, exact, dom);
                    any_domain |= dom;
                } else {
                    const int m = (int)umin64(len, C::K);
                    const uint8_t *src = bytes + off;
                    unsigned last = 0;
                    for (int i = 0; i < m; ++i) {
                        const unsigned c = src[i];
                        if (CW == 1) any_domain |= c >= 0x80u;
                        code = (code << C::W) | (uint64_t)(c & C::MASK);
                        last = c;
                    }
                    const int shift = C::W * (C::K - m);
                    code = shift >= 64 ? 0 : (code << shift);
                    exact = len <= (uint64_t)C::K && (len == 0 || last != 0);
                }
                hkey = code;
                if (pack_idx) {
                    code = (code << pk.idx_bits) | (pk.idx_base + t0 + j);
                } else if (KEYFLAG) {
                    code = (code << 1) | (exact ? 0u : 1u);
                    hkey = code;
                }
                if (pack) {
                    // the instance of string i lies between the tile's first and last
                    const uint64_t i = t0 + j;
                    uint64_t lo = pk.tile_seg[tile], hi = (uint64_t)pk.tile_seg[tile + 1] + 1;
                    if (hi > pk.num_segs) hi = pk.num_segs;
                    while (hi - lo > 1) {
                        const uint64_t mid = (lo + hi) >> 1;
                        if (pk.seg_offsets[mid] <= i) lo = mid; else hi = mid;
                    }
                    const uint64_t local = i - pk.seg_offsets[lo];
                    if (local > kIdxMask) any_bad_local = true;
                    code |= lo << (code_bits & 63);
                    hkey = code;
                    pk.vals[i] = (uint32_t)local & kIdxMask;
                }
                codes[t0 + j] = code;
                kmin = code < kmin ? code : kmin;
                kmax = code > kmax ? code : kmax;
            }
            if (hist) {  // whole warp converged here
                if (k * kEncThreads + warp * 32 + 32 <= cnt) {
#pragma unroll
                    for (int p = 0; p < kEncHistPasses; ++p)
                        if (p < hist_digits)
                            hist_add_full(s_hist + p * kBins, (unsigned)((hkey >> digit_shift(p)) & digit_mask(p)));
                } else {
#pragma unroll
                    for (int p = 0; p < kEncHistPasses; ++p)
                        if (p < hist_digits)
                            hist_add(s_hist + p * kBins, (unsigned)((hkey >> digit_shift(p)) & digit_mask(p)), valid);
                }
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
    if (__syncthreads_or(any_bad_local) && tid == 0) atomicOr(&flags->error, kErrInternal);
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
                       int alpha_max_w, int alpha_max_bits, EncPack pk, cudaStream_t s) {
    auto kern = encode_kernel<CODER, KEYFLAG>;
    static bool configured = false;  // attribute is per function, idempotent
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEncSmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    kern<<<grid, kEncThreads, kEncSmem, s>>>(bytes, offsets, n, codes, nonexact_bits, hist, flags, alpha_max_w,
                                              alpha_max_bits, pk);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_encode(int coder, bool key_flag, const uint8_t *bytes,
                          const uint64_t *offsets, uint64_t n, uint64_t *codes,
                          uint32_t *nonexact_bits, unsigned long long *hist,
                          DevFlags *flags, int num_sms, cudaStream_t s, int alpha_max_w, int alpha_max_bits,
                          EncPack pack) {
    if (n == 0) return cudaSuccess;
    const uint64_t tiles = (n + kEncTile - 1) / kEncTile;
    const unsigned grid = (unsigned)umin64(tiles, (uint64_t)num_sms * 4);
    if (coder == 2) {
        if (key_flag) return cudaErrorInvalidValue;  // BYTE8 codes use all 64 bits
        return launch_enc<2, false>(bytes, offsets, n, codes, nonexact_bits, hist, flags, grid, alpha_max_w, alpha_max_bits, pack, s);
    }
    if (coder == 3) {
        if (key_flag) return launch_enc<3, true>(bytes, offsets, n, codes, nonexact_bits, hist, flags, grid, alpha_max_w, alpha_max_bits, pack, s);
        return launch_enc<3, false>(bytes, offsets, n, codes, nonexact_bits, hist, flags, grid, alpha_max_w, alpha_max_bits, pack, s);
    }
    if (key_flag) return launch_enc<1, true>(bytes, offsets, n, codes, nonexact_bits, hist, flags, grid, alpha_max_w, alpha_max_bits, pack, s);
    return launch_enc<1, false>(bytes, offsets, n, codes, nonexact_bits, hist, flags, grid, alpha_max_w, alpha_max_bits, pack, s);
}

__global__ void tile_segs_kernel(const uint64_t *__restrict__ seg_offsets, uint64_t num_segs, uint64_t n,
                                 uint64_t tiles, uint32_t *__restrict__ tile_seg) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > tiles) return;
    const uint64_t i = umin64(t * (uint64_t)kEncTile, n - 1);
    uint64_t lo = 0, hi = num_segs;  // seg_offsets[lo] <= i < seg_offsets[hi]
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (seg_offsets[mid] <= i) lo = mid; else hi = mid;
    }
    tile_seg[t] = (uint32_t)lo;
}

cudaError_t launch_tile_segs(const uint64_t *seg_offsets, uint64_t num_segs, uint64_t n, uint32_t *tile_seg,
                             cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t tiles = (n + kEncTile - 1) / kEncTile;
    tile_segs_kernel<<<(unsigned)((tiles + 256) / 256), 256, 0, s>>>(seg_offsets, num_segs, n, tiles, tile_seg);
    return cudaGetLastError();
}

// Sorted-input test over the keys the encoder wrote: each string's order
// key (the key, or the code above a packed index) against its
// predecessor's.  The key preserves the order, so a descent proves the input
// unsorted; equal keys of strings that are not both exact leave the pair to a
// full comparison.  Every tile first looks whether some tile has already
// found a descent and stops if so, so an unsorted input costs about one wave.
constexpr int kSortedThreads = 256;
constexpr int kSortedItems = 4;

__global__ void __launch_bounds__(kSortedThreads)
sorted_test_kernel(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ nonexact_bits, uint64_t n,
                   int flag_in_key_requested, int idx_bits, uint64_t *__restrict__ pairs, uint64_t pairs_cap,
                   DevFlags *flags) {
    constexpr int kTile = kSortedThreads * kSortedItems;
    const int tid = threadIdx.x;
    const bool packed = flags->idx_packed != 0;  // written by the encoder this call
    const int sh = packed ? idx_bits : 0;
    const bool flag_in_key = flag_in_key_requested && !packed;
    const uint64_t tiles = (n + kTile - 1) / kTile;
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        if (tile != blockIdx.x &&  // a block's first tile does not wait for the flag
            __syncthreads_or(tid == 0 && *reinterpret_cast<volatile unsigned int *>(&flags->descent) != 0u))
            return;
        bool desc = false;
        uint32_t cand = 0;
#pragma unroll
        for (int k = 0; k < kSortedItems; ++k) {
            const uint64_t i = tile * kTile + (uint64_t)k * kSortedThreads + tid;  // pair (i - 1, i)
            if (i == 0 || i >= n) continue;
            const uint64_t va = keys[i - 1], vb = keys[i];
            const uint64_t a = va >> sh, b = vb >> sh;
            if (a > b) {
                desc = true;
            } else if (a == b) {
                bool both_exact;
                if (flag_in_key) {
                    both_exact = ((va | vb) & 1u) == 0;
                } else {
                    const bool ea = ((nonexact_bits[(i - 1) >> 5] >> ((i - 1) & 31)) & 1u) == 0;
                    const bool eb = ((nonexact_bits[i >> 5] >> (i & 31)) & 1u) == 0;
                    both_exact = ea && eb;
                }
                if (!both_exact) cand |= 1u << k;
            }
        }
        if (__syncthreads_or(desc)) {
            if (tid == 0) atomicOr(&flags->descent, 1u);
            return;
        }
#pragma unroll
        for (int k = 0; k < kSortedItems; ++k) {
            if (!((cand >> k) & 1u)) continue;
            const unsigned long long q = atomicAdd(&flags->pairs, 1ull);
            if (q < pairs_cap) pairs[q] = tile * kTile + (uint64_t)k * kSortedThreads + tid - 1;
        }
    }
}

cudaError_t launch_sorted_test(const uint64_t *keys, const uint32_t *nonexact_bits, uint64_t n, bool flag_in_key,
                               int idx_bits, uint64_t *pairs, uint64_t pairs_cap, DevFlags *flags, int num_sms,
                               cudaStream_t s) {
    if (n < 2) return cudaSuccess;
    if (!flag_in_key && nonexact_bits == nullptr) return cudaErrorInvalidValue;
    const uint64_t tiles = (n + kSortedThreads * kSortedItems - 1) / (kSortedThreads * kSortedItems);
    const unsigned grid = (unsigned)umin64(tiles, (uint64_t)num_sms * 2);  // a small first wave
    sorted_test_kernel<<<grid, kSortedThreads, 0, s>>>(keys, nonexact_bits, n, flag_in_key ? 1 : 0, idx_bits, pairs,
                                                        pairs_cap, flags);
    return cudaGetLastError();
}

// Numeric coders (the order-preserving unsigned keys of husky.h's hs_numeric).
__device__ __forceinline__ uint64_t numeric_code(const void *values, uint64_t i, int type) {
    switch (type) {
        case 1:    // int64
        case 5: {  // date-time, int64 ns
            return static_cast<const uint64_t *>(values)[i] ^ 0x8000000000000000ull;
        }
        case 2:  // int32
            return (uint64_t)(static_cast<const uint32_t *>(values)[i] ^ 0x80000000u);
        case 3: {  // binary64
            uint64_t x = static_cast<const uint64_t *>(values)[i];
            if ((x & 0x7FF0000000000000ull) == 0x7FF0000000000000ull && (x & 0x000FFFFFFFFFFFFFull) != 0)
                x = 0x7FF8000000000000ull;
            return (x >> 63) ? ~x : (x | 0x8000000000000000ull);
        }
        case 4: {  // binary32
            uint32_t x = static_cast<const uint32_t *>(values)[i];
            if ((x & 0x7F800000u) == 0x7F800000u && (x & 0x007FFFFFu) != 0) x = 0x7FC00000u;
            return (uint64_t)((x >> 31) ? ~x : (x | 0x80000000u));
        }
        default:
            return static_cast<const uint64_t *>(values)[i];
    }
}

constexpr int kNumThreads = 512;

// codes[i] = numeric code of values[i], or with pack_bits > 0 the word
// (code << pack_bits) | i; with hist, the 8 digit histograms of the codes
// (accumulated).
__global__ void __launch_bounds__(kNumThreads)
numeric_encode_kernel(const void *__restrict__ values, uint64_t n, int type, uint64_t *__restrict__ codes,
                      unsigned long long *__restrict__ hist, int pack_bits) {
    __shared__ uint32_t s_hist[kKeyPasses * kBins];
    if (hist)
        for (int i = threadIdx.x; i < kKeyPasses * kBins; i += kNumThreads) s_hist[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * kNumThreads;
    const uint64_t n_round = (n + 31) & ~31ull;  // whole warps iterate together
    // 32-bit codes: the digits above bit 35 are zero for every value, counted
    // in bin 0 at the end instead of per value
    const int nd = (type == 2 || type == 4) ? 4 : kKeyPasses;
    uint32_t valid_count = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * kNumThreads + threadIdx.x; i < n_round; i += stride) {
        const bool valid = i < n;
        const uint64_t k = valid ? numeric_code(values, i, type) : 0;
        if (valid) codes[i] = pack_bits > 0 ? (k << pack_bits) | i : k;
        valid_count += valid ? 1u : 0u;
        if (hist) {
#pragma unroll
            for (int p = 0; p < kKeyPasses; ++p)
                if (p < nd) hist_add(s_hist + p * kBins, (unsigned)((k >> digit_shift(p)) & digit_mask(p)), valid);
        }
    }
    if (!hist) return;
    const uint32_t warp_count = __reduce_add_sync(kFull, valid_count);
    if ((threadIdx.x & 31) == 0 && warp_count)
        for (int p = nd; p < kKeyPasses; ++p) atomicAdd(&s_hist[p * kBins], warp_count);
    __syncthreads();
    for (int i = threadIdx.x; i < kKeyPasses * kBins; i += kNumThreads)
        if (s_hist[i]) atomicAdd(&hist[i], (unsigned long long)s_hist[i]);
}

cudaError_t launch_numeric_encode(const void *values, uint64_t n, int type, uint64_t *codes,
                                  unsigned long long *hist, int num_sms, cudaStream_t s, int pack_bits) {
    if (n == 0) return cudaSuccess;
    if (pack_bits < 0 || pack_bits > 32) return cudaErrorInvalidValue;  // 32-bit codes only
    const uint64_t blocks = (n + kNumThreads * 8 - 1) / (kNumThreads * 8);
    const unsigned grid = (unsigned)umin64(blocks, (uint64_t)num_sms * 4);
    numeric_encode_kernel<<<grid, kNumThreads, 0, s>>>(values, n, type, codes, hist, pack_bits);
    return cudaGetLastError();
}

cudaError_t launch_alphabet(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, int max_span,
                            DevFlags *flags, int num_sms, cudaStream_t s) {
    alphabet_kernel<<<(unsigned)num_sms * 4, kAlphaThreads, 0, s>>>(bytes, offsets, n, max_span, flags);
    return cudaGetLastError();
}

}  // namespace hs
