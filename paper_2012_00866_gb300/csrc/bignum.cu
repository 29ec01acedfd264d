// BigInteger coder.  Section 6.1 and Table 4 sort BigInteger arrays with Huskysort; the
// paper gives no coder for them.  A big integer here is its minimal two's
// complement bytes, big-endian (Java's toByteArray).  A two-byte header that
// orders by sign and length turns it into a byte string whose unsigned-byte
// order is numeric order: negatives (header 0x7FFF - L, below 0x8000) before
// non-negatives (0x8000 + L); among non-negatives a longer minimal value is
// larger, among negatives a longer one is smaller; at equal length and sign
// the two's complement bytes compare in numeric order.  The strings then go
// through the string path unchanged (byte coder, radix sort, fix-up).
#include "hs_bignum.h"

namespace hs {
namespace {

constexpr int kBigThreads = 256;

__global__ void __launch_bounds__(kBigThreads)
bigint_encode_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets, uint64_t n,
                     uint8_t *__restrict__ out_bytes, uint64_t out_cap, uint64_t *__restrict__ out_offsets,
                     DevFlags *flags) {
    const uint64_t stride = (uint64_t)gridDim.x * kBigThreads;
    const uint64_t base = offsets[0];
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * kBigThreads + threadIdx.x; i < n; i += stride) {
        const uint64_t o = offsets[i], e = offsets[i + 1];
        const uint64_t dst = (o - base) + 2 * i;
        out_offsets[i] = dst;
        if (i + 1 == n) out_offsets[n] = (e - base) + 2 * n;
        if (e <= o || e - o > kBigMaxLen || o < base || dst + 2 + (e - o) > out_cap) {
            bad = true;  // empty, decreasing, too long or past the buffer the caller sized
            continue;
        }
        const uint64_t len = e - o;
        const uint8_t b0 = bytes[o];
        const bool neg = b0 >= 0x80u;
        if (len >= 2) {  // minimal: no redundant sign byte
            const uint8_t b1 = bytes[o + 1];
            bad |= (b0 == 0x00u && b1 < 0x80u) || (b0 == 0xFFu && b1 >= 0x80u);
        }
        const uint32_t h = neg ? 0x7FFFu - (uint32_t)len : 0x8000u + (uint32_t)len;
        out_bytes[dst] = (uint8_t)(h >> 8);
        out_bytes[dst + 1] = (uint8_t)h;
        for (uint64_t k = 0; k < len; ++k) out_bytes[dst + 2 + k] = bytes[o + k];
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&flags->error, kErrOffsets);
}

// ---- BigDecimal coder ----------------------------------------------------------
//
// Section 6.1 and Table 4 sort BigDecimal arrays with Huskysort; the paper
// gives no coder.  A value here is its decimal text (an optional sign, digits
// with at most one decimal point, an optional exponent [eE][+-]digits: the
// form Java's BigDecimal(String) accepts).  With the value written as
// 0.d1 d2 ... dk x 10^X (d1 != 0, no trailing zero digit) the byte string is
// a class byte, the exponent, and the digits two to a byte:
//   class     0x00 / 0x01 / 0x02 negative with X >= 2^23 / |X| < 2^23 /
//             X < -2^23; 0x03 zero (alone); 0x04 / 0x05 / 0x06 positive with
//             X < -2^23 / |X| < 2^23 / X >= 2^23
//   exponent  X + 2^23 in 3 big-endian bytes (|X| < 2^23), else X + 2^39 in
//             5; complemented for negatives
//   digits    each pair d(2i-1) d(2i) as the byte 10 d(2i-1) + d(2i) (an odd
//             last digit paired with 0), as 99 minus that for negatives,
//             which end with 0xFF
// Its unsigned-byte order is numeric order, and equal values (1.0 and 1.00)
// give equal strings, as compareTo wants.  Among positives of one class a
// larger X is larger, and at equal X the digits compare as decimal
// fractions: pairs compare as two digits do, and a shorter string that is a
// prefix is smaller (no trailing zero digits, so the longer one continues
// with a nonzero digit); negatives reverse both, the 0xFF terminator putting
// a prefix (a smaller magnitude) after its extensions.  The first 8 bytes,
// which the byte coder turns into the sort key, hold up to 8 digits.
// Three kernels: each value's encoded length and a tile total; an exclusive
// scan of the tile totals; each tile's offsets and bytes.

constexpr int kDecThreads = 256;
constexpr int kDecPer = 4;                       // values a thread, consecutive
constexpr int kDecTile = kDecThreads * kDecPer;  // values a tile
constexpr int64_t kDecMaxExp = 999999999;        // |exponent| below 10^9
constexpr int64_t kDecBias = 1ll << 39;            // 5-byte exponents
constexpr int64_t kDecSmall = 1ll << 23;           // |X| below this: 3-byte exponents
constexpr uint32_t kDecStage = 24576;            // a tile's text bytes staged in shared memory
constexpr uint32_t kDecOutStage = 20480;         // a tile's output bytes, gathered before one coalesced copy

struct DecForm {
    bool ok;
    int cls;                 // 0 negative, 1 zero, 2 positive
    int64_t X;               // the value is 0.d1 d2 ... dk x 10^X
    uint32_t mstart, mend;   // the mantissa's characters (digits and at most one '.')
    uint32_t z, k;           // leading zero digits, then the k digits kept
};

__device__ DecForm dec_parse(const uint8_t *__restrict__ s, uint32_t len) {
    DecForm f{};
    uint32_t i = 0;
    bool neg = false;
    if (i < len && (s[i] == '+' || s[i] == '-')) {
        neg = s[i] == '-';
        ++i;
    }
    f.mstart = i;
    // one pass over the mantissa: digits t (p before the point), the number
    // of leading zero digits z and the position of the last nonzero one
    uint32_t t = 0, p = 0, z = 0, last = 0;
    bool dot = false, seen = false;
    for (; i < len; ++i) {
        const uint8_t c = s[i];
        const bool digit = (unsigned)(c - '0') < 10u;
        const bool point = c == '.' && !dot;
        if (!digit && !point) break;
        dot |= point;
        const bool nz = digit && c != '0';
        t += digit;
        p += digit && !dot;
        z = (nz && !seen) ? t - 1 : z;
        seen |= nz;
        last = nz ? t : last;
    }
    f.mend = i;
    if (t == 0) return f;
    int64_t ex = 0;
    if (i < len && (s[i] == 'e' || s[i] == 'E')) {
        ++i;
        bool eneg = false;
        if (i < len && (s[i] == '+' || s[i] == '-')) {
            eneg = s[i] == '-';
            ++i;
        }
        uint32_t nd = 0;
        for (; i < len && s[i] >= '0' && s[i] <= '9'; ++i, ++nd) {
            ex = ex * 10 + (s[i] - '0');
            if (ex > kDecMaxExp) return f;
        }
        if (nd == 0) return f;
        if (eneg) ex = -ex;
    }
    if (i != len) return f;
    f.ok = true;
    if (!seen) {
        f.cls = 1;
        return f;
    }
    f.cls = neg ? 0 : 2;
    f.z = z;
    f.k = last - z;
    f.X = (int64_t)p - (int64_t)z + ex;
    return f;
}

__device__ __forceinline__ bool dec_small(const DecForm &f) { return f.X > -kDecSmall && f.X < kDecSmall; }

__device__ __forceinline__ uint32_t dec_len(const DecForm &f) {
    if (f.cls == 1) return 1u;
    return 1u + (dec_small(f) ? 3u : 5u) + (f.k + 1) / 2 + (f.cls == 0 ? 1u : 0u);
}

__device__ void dec_write(const uint8_t *__restrict__ s, const DecForm &f, uint8_t *__restrict__ out) {
    if (f.cls == 1) {
        out[0] = 0x03;
        return;
    }
    const bool neg = f.cls == 0, small = dec_small(f);
    const uint32_t band = small ? 1u : (f.X < 0 ? 0u : 2u);  // tiny, small or huge |value| scale
    out[0] = (uint8_t)(neg ? 2u - band : 4u + band);
    const int nb = small ? 3 : 5;
    uint64_t e = (uint64_t)(f.X + (small ? kDecSmall : kDecBias));
    if (neg) e = ~e & ((1ull << (8 * nb)) - 1);
    for (int b = 0; b < nb; ++b) out[1 + b] = (uint8_t)(e >> (8 * (nb - 1 - b)));
    uint32_t idx = 0, w = 1 + nb, pending = 0;
    bool half = false;  // a first digit of a pair is pending
    for (uint32_t j = f.mstart; j < f.mend && idx < f.z + f.k; ++j) {
        const uint8_t c = s[j];
        if (c == '.') continue;
        if (idx >= f.z) {
            const uint32_t d = c - '0';
            if (half) {
                const uint32_t v = 10 * pending + d;
                out[w++] = (uint8_t)(neg ? 99u - v : v);
            } else {
                pending = d;
            }
            half = !half;
        }
        ++idx;
    }
    if (half) out[w++] = (uint8_t)(neg ? 99u - 10 * pending : 10 * pending);
    if (neg) out[w] = 0xFFu;
}

// Value i's text, or false when its offsets decrease, pass the buffer, or
// the text is longer than kDecMaxLen.
__device__ __forceinline__ bool dec_text(const uint64_t *__restrict__ offsets, uint64_t i, uint64_t total,
                                         uint64_t *o, uint32_t *len) {
    const uint64_t a = offsets[i], b = offsets[i + 1];
    if (b < a || b > total || b - a > kDecMaxLen) return false;
    *o = a;
    *len = (uint32_t)(b - a);
    return true;
}

// Copies the tile's text bytes (strings t0 .. t0 + cnt - 1, contiguous when
// their offsets are in order) into s_text with coalesced loads; returns the
// first byte's offset, or ~0 when they do not fit (or the offsets are out of
// order), in which case every string is read from global memory.  Ends with a
// barrier.
__device__ uint64_t dec_stage(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                              uint64_t t0, uint64_t cnt, uint64_t total, uint8_t *s_text, uint32_t *span) {
    const uint64_t lo = offsets[t0], hi = offsets[t0 + cnt];
    const bool fits = lo <= hi && hi <= total && hi - lo <= kDecStage;
    if (fits)
        for (uint64_t k = threadIdx.x; k < hi - lo; k += kDecThreads) s_text[k] = bytes[lo + k];
    __syncthreads();
    *span = fits ? (uint32_t)(hi - lo) : 0u;
    return fits ? lo : ~0ull;
}

// Where value i's text is read from: the stage when it lies inside the
// staged bytes [lo, lo + span).
__device__ __forceinline__ const uint8_t *dec_src(const uint8_t *__restrict__ bytes, const uint8_t *s_text,
                                                  uint64_t lo, uint32_t span, uint64_t o, uint32_t len) {
    return (lo != ~0ull && o >= lo && o - lo + len <= span) ? s_text + (o - lo) : bytes + o;
}

// Exclusive scan over the block of one u64 per thread; *block_total: the sum.
__device__ uint64_t dec_block_scan(uint64_t v, uint64_t *block_total) {
    __shared__ unsigned long long s_w[kDecThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    unsigned long long pre = 0, all = 0;
    for (int w = 0; w < kDecThreads / 32; ++w) {
        pre += w < warp ? s_w[w] : 0ull;
        all += s_w[w];
    }
    __syncthreads();
    *block_total = all;
    return pre + x - v;
}

__global__ void __launch_bounds__(kDecThreads)
dec_len_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets, uint64_t n, uint64_t total,
               unsigned long long *__restrict__ tile_sum, DevFlags *flags) {
    __shared__ uint8_t s_text[kDecStage];
    const uint64_t t0 = (uint64_t)blockIdx.x * kDecTile;
    uint32_t span;
    const uint64_t lo = dec_stage(bytes, offsets, t0, umin64(kDecTile, n - t0), total, s_text, &span);
    const uint64_t i0 = t0 + (uint64_t)threadIdx.x * kDecPer;
    uint64_t sum = 0;
    bool bad = false;
    for (int q = 0; q < kDecPer; ++q) {
        const uint64_t i = i0 + q;
        if (i >= n) break;
        uint64_t o;
        uint32_t len;
        if (!dec_text(offsets, i, total, &o, &len)) {
            bad = true;
            continue;
        }
        const DecForm f = dec_parse(dec_src(bytes, s_text, lo, span, o, len), len);
        bad |= !f.ok;
        sum += f.ok ? dec_len(f) : 0u;
    }
    uint64_t all;
    dec_block_scan(sum, &all);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = all;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&flags->error, kErrOffsets);
}

// Exclusive scan of the tile totals in place (one CTA, chunks of its size);
// the grand total goes to tile_sum[tiles].
__global__ void __launch_bounds__(kDecThreads) dec_scan_kernel(unsigned long long *__restrict__ tile_sum,
                                                               uint64_t tiles) {
    uint64_t carry = 0;
    for (uint64_t c0 = 0; c0 < tiles; c0 += kDecThreads) {
        const uint64_t t = c0 + threadIdx.x;
        const uint64_t v = t < tiles ? tile_sum[t] : 0ull;
        uint64_t all;
        const uint64_t ex = dec_block_scan(v, &all);
        if (t < tiles) tile_sum[t] = carry + ex;
        carry += all;
    }
    if (threadIdx.x == 0) tile_sum[tiles] = carry;
}

__global__ void __launch_bounds__(kDecThreads)
dec_write_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets, uint64_t n, uint64_t total,
                 const unsigned long long *__restrict__ tile_base, uint8_t *__restrict__ out_bytes, uint64_t out_cap,
                 uint64_t *__restrict__ out_offsets, DevFlags *flags) {
    __shared__ uint8_t s_text[kDecStage];
    __shared__ __align__(16) uint8_t s_out[kDecOutStage];
    const uint64_t t0 = (uint64_t)blockIdx.x * kDecTile;
    uint32_t span;
    const uint64_t lo = dec_stage(bytes, offsets, t0, umin64(kDecTile, n - t0), total, s_text, &span);
    const uint64_t i0 = t0 + (uint64_t)threadIdx.x * kDecPer;
    // The tile's strings are contiguous in the output: when they fit the
    // stage they are written there and leave in one coalesced copy, instead
    // of each thread's bytes going out to its own scattered sectors.
    const uint64_t out0 = tile_base[blockIdx.x], out1 = tile_base[blockIdx.x + 1];
    const bool staged_out = out1 >= out0 && out1 - out0 <= kDecOutStage && out1 <= out_cap;
    uint32_t lens[kDecPer];
    uint64_t sum = 0;
    for (int q = 0; q < kDecPer; ++q) {
        const uint64_t i = i0 + q;
        lens[q] = 0;
        uint64_t o;
        uint32_t len;
        if (i < n && dec_text(offsets, i, total, &o, &len)) {
            const DecForm f = dec_parse(dec_src(bytes, s_text, lo, span, o, len), len);
            lens[q] = f.ok ? dec_len(f) : 0u;
        }
        sum += lens[q];
    }
    uint64_t all;
    uint64_t dst = tile_base[blockIdx.x] + dec_block_scan(sum, &all);
    bool bad = false;
    for (int q = 0; q < kDecPer; ++q) {
        const uint64_t i = i0 + q;
        if (i >= n) break;
        out_offsets[i] = dst;
        if (lens[q]) {
            if (dst + lens[q] > out_cap) {
                bad = true;
            } else {
                uint64_t o;
                uint32_t len;
                dec_text(offsets, i, total, &o, &len);
                const uint8_t *src = dec_src(bytes, s_text, lo, span, o, len);
                dec_write(src, dec_parse(src, len), staged_out ? s_out + (dst - out0) : out_bytes + dst);
            }
        }
        dst += lens[q];
        if (i + 1 == n) out_offsets[n] = dst;
    }
    __syncthreads();
    if (staged_out)
        for (uint64_t k = threadIdx.x; k < out1 - out0; k += kDecThreads) out_bytes[out0 + k] = s_out[k];
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&flags->error, kErrInternal);
}

}  // namespace

cudaError_t launch_bigdecimal_lengths(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, uint64_t total,
                                      unsigned long long *tile_sum, DevFlags *flags, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t tiles = (n + kDecTile - 1) / kDecTile;
    dec_len_kernel<<<(unsigned)tiles, kDecThreads, 0, s>>>(bytes, offsets, n, total, tile_sum, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dec_scan_kernel<<<1, kDecThreads, 0, s>>>(tile_sum, tiles);
    return cudaGetLastError();
}

cudaError_t launch_bigdecimal_write(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, uint64_t total,
                                    const unsigned long long *tile_base, uint8_t *out_bytes, uint64_t out_cap,
                                    uint64_t *out_offsets, DevFlags *flags, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t tiles = (n + kDecTile - 1) / kDecTile;
    dec_write_kernel<<<(unsigned)tiles, kDecThreads, 0, s>>>(bytes, offsets, n, total, tile_base, out_bytes, out_cap,
                                                             out_offsets, flags);
    return cudaGetLastError();
}

uint64_t bigdecimal_tiles(uint64_t n) { return (n + kDecTile - 1) / kDecTile; }

cudaError_t launch_bigint_encode(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, uint8_t *out_bytes,
                                 uint64_t out_cap, uint64_t *out_offsets, DevFlags *flags, int num_sms,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + kBigThreads - 1) / kBigThreads;
    const unsigned grid = (unsigned)(blocks < (uint64_t)num_sms * 8 ? blocks : (uint64_t)num_sms * 8);
    bigint_encode_kernel<<<grid, kBigThreads, 0, s>>>(bytes, offsets, n, out_bytes, out_cap, out_offsets, flags);
    return cudaGetLastError();
}

}  // namespace hs
