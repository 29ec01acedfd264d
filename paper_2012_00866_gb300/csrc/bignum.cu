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

}  // namespace

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
