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

// BigDecimal texts longer than this many bytes are rejected.
constexpr uint64_t kDecMaxLen = 32767;

// BigDecimal coder, step 1: checks each of n decimal texts (bytes
// offsets[i] .. offsets[i+1] of a buffer of `total` bytes) and computes the
// length of its order-preserving byte string; tile_sum (bigdecimal_tiles(n)
// + 1 entries) receives the exclusive scan of the per-tile totals, the grand
// total last.  A text outside the grammar, offsets that decrease or pass the
// buffer, or a text longer than kDecMaxLen set flags->error |= kErrOffsets.
cudaError_t launch_bigdecimal_lengths(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, uint64_t total,
                                      unsigned long long *tile_sum, DevFlags *flags, cudaStream_t s);
// Step 2 (once step 1 reported no error): writes each value's byte string to
// out_bytes at out_offsets[i] (out_offsets[n] closes the last), placed by the
// scanned tile totals.  For the value 0.d1 .. dk x 10^X (d1, dk nonzero) the
// string is a class byte (0x03 for zero, alone; 0x04..0x06 for positives
// with X < -2^23, |X| < 2^23, X >= 2^23; 0x02..0x00 for negatives likewise),
// the exponent (X + 2^23 in 3 big-endian bytes when |X| < 2^23, else X + 2^39
// in 5; complemented for negatives), and the digits two to a byte (10 a + b,
// an odd last digit paired with 0; 99 minus that for negatives, which end
// with 0xFF).  Their unsigned-byte order is numeric order, and equal values
// give equal strings.
cudaError_t launch_bigdecimal_write(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, uint64_t total,
                                    const unsigned long long *tile_base, uint8_t *out_bytes, uint64_t out_cap,
                                    uint64_t *out_offsets, DevFlags *flags, cudaStream_t s);
uint64_t bigdecimal_tiles(uint64_t n);

}  // namespace hs
