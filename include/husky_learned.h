/*
 * husky_learned.h -- component entry points of the learned bucketer used by
 * hs_argsort(HS_MODE_LEARNED), exposed so each piece can be checked on its
 * own.  The paper has no learned model: these support the learned form of
 * Step 2 (Section 3.1), whose only requirement -- a bucket order that never
 * contradicts the code order (Section 3.2) -- the model meets by being
 * monotone.  Conventions as in husky.h: d_* device pointers owned by the
 * caller, work enqueued on `stream`, every call synchronises it and returns
 * the final status.
 *
 * Model: root y = w3 . h(W2 h(W1 x + b1) + b2) + b3 with h(z) = min(max(z,0),1),
 * 1 -> 32 -> 32 -> 1; parameters packed as 1153 floats in the order
 * W1[32] b1[32] W2[32][32] (row i = second-layer unit i) b2[32] w3[32] b3.
 */
#ifndef HUSKY_LEARNED_H
#define HUSKY_LEARNED_H

#include "husky.h"

#ifdef __cplusplus
extern "C" {
#endif

#define HS_RMI_PARAMS 1153
#define HS_RMI_MAX_POINTS 2048

/* Mean squared error (1/T) sum (root(x_i) - t_i)^2 and its gradient with
 * respect to the 1153 parameters, in FP32 with deterministic (fixed-order)
 * sums -- the kernel the learned path trains with.
 *   d_params in, 1153 floats; d_x, d_t in, T floats; d_grad out, 1153 floats;
 *   d_loss out, 1 float.  1 <= T <= HS_RMI_MAX_POINTS. */
HS_API hs_status hs_rmi_grad(const float *d_params, const float *d_x,
                             const float *d_t, uint32_t T, float *d_grad,
                             float *d_loss, void *stream);

/* Least-squares line per leaf over contiguous point ranges (FP64 sums):
 * leaf l owns points d_leaf_start[l] .. d_leaf_start[l+1]-1 (leaves + 1
 * entries, non-decreasing, last = m).  Outputs per leaf: slope (clamped >= 0;
 * 0 when fewer than two points or no spread), intercept (mean of t when the
 * slope is 0, band start when empty), band lo = leaf_start[l]/m, band hi =
 * leaf_start[l+1]/m. */
HS_API hs_status hs_rmi_leaf_fit(const float *d_x, const float *d_t,
                                 const uint32_t *d_leaf_start, uint32_t m,
                                 uint32_t leaves, float *d_slope,
                                 float *d_icept, float *d_lo, float *d_hi,
                                 void *stream);

/* The 1% sample the learned path trains on: for k < n/100, index
 * k*100 + splitmix64(k ^ seed) mod 100, splitmix64 being the SplitMix64
 * output function (Steele, Lea and Flood 2014).  d_out: n/100 uint64. */
HS_API hs_status hs_rmi_sample_indices(uint64_t n, uint64_t seed,
                                       uint64_t *d_out, void *stream);

/* Runs the learned path's Step 1 and model fit on n strings (ASCII7 coder
 * required) and writes, per string i, its sort key (d_keys, n uint64: code
 * << 1 | not exact) and its bucket (d_buckets, n uint32) under the trained
 * model, or under the untrained linear map bucket = floor(x B) when linear
 * != 0.  h_info (nullable, 4 entries): bucket bits, sample size, training
 * loss before and after the gradient steps (as IEEE doubles).  Workspace:
 * hs_workspace_size(n, 0, HS_MODE_LEARNED, ...); n >= 65536. */
HS_API hs_status hs_learned_profile(const uint8_t *d_bytes,
                                    const uint64_t *d_offsets, uint64_t n,
                                    int linear, uint64_t *d_keys,
                                    uint32_t *d_buckets, double *h_info,
                                    void *d_ws, size_t ws_bytes, void *stream);

/* Test support: the number of bucket-id bits the learned path uses.  By
 * default (bits = 0), for keys of the byte-range coder (the bucket id then
 * rides above the key in one word), enough bits for an average bucket of at
 * most about 2048 keys, up to 18 (two 9-bit partition passes); for ASCII7
 * keys, about n/256 buckets rounded to whole partition passes: 18 bits up to
 * about 2.7e8 keys, 23 or 24 above.  A value of 1..24 forces that many bits
 * for every later learned sort in the process, so that each branch (one to
 * three partition passes, buckets longer than the in-CTA window, a separate
 * bucket array when the id does not fit above the key) can be checked at
 * sizes the oracle sorts quickly; the result never depends on it.
 * Workspace sizes follow the setting.  HS_ERR_INVALID_ARG for other
 * values. */
HS_API hs_status hs_learned_force_bucket_bits(int bits);

#ifdef __cplusplus
}
#endif

#endif /* HUSKY_LEARNED_H */
