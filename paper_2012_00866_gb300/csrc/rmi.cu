// Learned bucketing for Step 2 (a recursive-model index over the sort keys).
//
// Huskysort's first pass only needs a key order that agrees with the codes
// (Section 3.1 Step 2; Section 3.2: x > y must never map below y).  Here a
// small learned CDF model maps each 64-bit sort key to one of B = 2^k
// buckets by a function that is monotone non-decreasing in the key, so a
// stable partition by bucket followed by a sort inside each bucket is the
// full sort by key -- two or three partition passes instead of seven radix
// passes.  The model never decides the order, only the speed.
//
//   feature   X = min((key - kmin) >> shift, 2^24 - 1), x = X 2^-24 (exact);
//   root      y = w3 . h(W2 h(W1 x + b1) + b2) + b3, h(z) = min(max(z,0),1),
//             1 -> 32 -> 32 -> 1, W1, W2, w3 >= 0: monotone in x (every FP32
//             operation used is monotone in its varying operand);
//   init      first-layer ramps between consecutive 1/32-quantiles of a 1%
//             sample, identity second layer: the root starts as the
//             piecewise-linear empirical CDF; then projected gradient steps
//             on the mean squared error (forward and backward in this file);
//   leaves    4096 leaves; leaf(X) = number of table thresholds <= X, the
//             table being the exact step function of the root (bisection);
//             leaf l fitted by least squares (FP64 sums), slope >= 0, output
//             clamped to the band [c_l, c_{l+1}] of sample fractions;
//   bucket    min(B - 1, floor(clamp(a_l x + b_l, c_l, c_{l+1}) B)).
#include <type_traits>

#include "hs_internal.h"

namespace hs {
namespace {

constexpr int kP_W1 = 0, kP_B1 = 32, kP_W2 = 64, kP_B2 = 64 + 1024, kP_W3 = kP_B2 + 32, kP_B3 = kP_W3 + 32;
static_assert(kP_B3 + 1 == kRmiParams, "parameter layout");
constexpr int kTrainThreads = 1024;
constexpr int kChunk = 128;           // training points per forward/backward chunk
constexpr int kRow = 33;              // padded activation row
constexpr float kMaxSlope = 1048576.0f;

__device__ __forceinline__ float ramp(float z) { return fminf(fmaxf(z, 0.0f), 1.0f); }
__device__ __forceinline__ float ramp_grad(float z) { return (z > 0.0f && z < 1.0f) ? 1.0f : 0.0f; }

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Root network, sequential order of operations (used for the leaf table).
__device__ float rmi_root(const float *__restrict__ P, float x) {
    float h1[kRmiHidden];
#pragma unroll
    for (int j = 0; j < kRmiHidden; ++j) h1[j] = ramp(fmaf(P[kP_W1 + j], x, P[kP_B1 + j]));
    float y = P[kP_B3];
#pragma unroll 4
    for (int i = 0; i < kRmiHidden; ++i) {
        float z = P[kP_B2 + i];
#pragma unroll
        for (int j = 0; j < kRmiHidden; ++j) z = fmaf(P[kP_W2 + i * kRmiHidden + j], h1[j], z);
        y = fmaf(P[kP_W3 + i], ramp(z), y);
    }
    return y;
}

__device__ __forceinline__ uint32_t root_leaf(const float *P, uint32_t X) {
    const float y = rmi_root(P, (float)X * 5.9604644775390625e-8f);  // X * 2^-24, exact
    const float v = fminf(fmaxf(y * (float)kRmiLeaves, 0.0f), (float)(kRmiLeaves - 1));
    return (uint32_t)v;
}

__device__ __forceinline__ uint32_t table_leaf(const uint32_t *__restrict__ thresh, uint32_t X) {
    // number of thresholds <= X among kRmiLeaves - 1 sorted entries
    uint32_t lo = 0, hi = kRmiLeaves - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (thresh[mid] <= X) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t feature_of(uint64_t key, uint64_t kmin, int shift) {
    const uint64_t d = key >= kmin ? (key - kmin) >> shift : 0;
    return d < (1u << kRmiFeatureBits) ? (uint32_t)d : (1u << kRmiFeatureBits) - 1;
}

// ---- loss and gradient over T points, one 1024-thread block --------------------
//
// Points are processed in chunks of 128, eight threads per point (each owns
// four of the 32 second-layer units); activations go to shared memory and
// then each thread accumulates the gradient of its own parameters over the
// chunk in point order, so the sums are deterministic.

struct GradSmem {
    float H1[kChunk][kRow], Z1[kChunk][kRow], DZ2[kChunk][kRow], H2[kChunk][kRow];
    float DY[kChunk], XC[kChunk], R2[kChunk];
};

// W2p: the second-layer weights again with a padded row stride of 33, so the
// eight threads of a point (eight different rows) read different banks.
__device__ void loss_grad_block(const float *__restrict__ P, const float (*__restrict__ W2p)[kRow],
                                const float *__restrict__ X, const float *__restrict__ Tt, int T, GradSmem &s,
                                float *__restrict__ G, float *loss_out) {
    const int tid = threadIdx.x, pt = tid >> 3, g = tid & 7;
    float acc_w2 = 0.f, acc_small = 0.f, acc_loss = 0.f;
    const float invT = 1.0f / (float)T;
    for (int c0 = 0; c0 < T; c0 += kChunk) {
        const int i = c0 + pt;
        const bool valid = i < T;
        const float x = valid ? X[i] : 0.f, t = valid ? Tt[i] : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = g * 4 + u;
            const float z1 = fmaf(P[kP_W1 + j], x, P[kP_B1 + j]);
            s.Z1[pt][j] = z1;
            s.H1[pt][j] = ramp(z1);
        }
        __syncwarp();
        float z2[4], yp = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = g * 4 + u;
            float z = P[kP_B2 + r];
#pragma unroll 8
            for (int j = 0; j < kRmiHidden; ++j) z = fmaf(W2p[r][j], s.H1[pt][j], z);
            z2[u] = z;
            yp = fmaf(P[kP_W3 + r], ramp(z), yp);
        }
        yp += __shfl_xor_sync(kFull, yp, 1);
        yp += __shfl_xor_sync(kFull, yp, 2);
        yp += __shfl_xor_sync(kFull, yp, 4);
        const float y = yp + P[kP_B3];
        const float res = valid ? y - t : 0.f;
        const float dy = 2.0f * res * invT;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = g * 4 + u;
            s.DZ2[pt][r] = dy * P[kP_W3 + r] * ramp_grad(z2[u]);
            s.H2[pt][r] = ramp(z2[u]);
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // dz1_j = (sum_r W2[r][j] dz2_r) h'(z1_j), stored over Z1
            const int j = g * 4 + u;
            float dh = 0.f;
#pragma unroll 8
            for (int r = 0; r < kRmiHidden; ++r) dh = fmaf(W2p[r][j], s.DZ2[pt][r], dh);
            s.Z1[pt][j] = dh * ramp_grad(s.Z1[pt][j]);
        }
        if (g == 0) {
            s.DY[pt] = dy;
            s.XC[pt] = x;
            s.R2[pt] = res * res;
        }
        __syncthreads();
        {   // W2[r][j]: thread tid = r * 32 + j
            const int r = tid >> 5, j = tid & 31;
            for (int q = 0; q < kChunk; ++q) acc_w2 = fmaf(s.DZ2[q][r], s.H1[q][j], acc_w2);
        }
        if (tid < 32) {
            for (int q = 0; q < kChunk; ++q) acc_small = fmaf(s.Z1[q][tid], s.XC[q], acc_small);       // W1
        } else if (tid < 64) {
            for (int q = 0; q < kChunk; ++q) acc_small += s.Z1[q][tid - 32];                            // b1
        } else if (tid < 96) {
            for (int q = 0; q < kChunk; ++q) acc_small += s.DZ2[q][tid - 64];                           // b2
        } else if (tid < 128) {
            for (int q = 0; q < kChunk; ++q) acc_small = fmaf(s.DY[q], s.H2[q][tid - 96], acc_small);  // w3
        } else if (tid == 128) {
            for (int q = 0; q < kChunk; ++q) acc_small += s.DY[q];                                      // b3
        } else if (tid == 129) {
            for (int q = 0; q < kChunk; ++q) acc_loss += s.R2[q];
        }
        __syncthreads();
    }
    G[kP_W2 + tid] = acc_w2;
    if (tid < 32) G[kP_W1 + tid] = acc_small;
    else if (tid < 64) G[kP_B1 + tid - 32] = acc_small;
    else if (tid < 96) G[kP_B2 + tid - 64] = acc_small;
    else if (tid < 128) G[kP_W3 + tid - 96] = acc_small;
    else if (tid == 128) G[kP_B3] = acc_small;
    else if (tid == 129) *loss_out = acc_loss * invT;
    __syncthreads();
}

struct TrainSmem {
    float P[kRmiParams + 3];
    float W2p[kRmiHidden][kRow];
    float G[kRmiParams + 3];
    float X[kRmiTrain], T[kRmiTrain];
    float red[32];
    float loss;
    GradSmem g;
};

// hs_rmi_grad test hook: one loss/gradient evaluation.
__global__ void __launch_bounds__(kTrainThreads)
rmi_grad_kernel(const float *__restrict__ params, const float *__restrict__ x, const float *__restrict__ t, int T,
                float *__restrict__ grad, float *__restrict__ loss) {
    extern __shared__ __align__(16) unsigned char train_smem[];
    TrainSmem &s = *reinterpret_cast<TrainSmem *>(train_smem);
    for (int k = threadIdx.x; k < kRmiParams; k += kTrainThreads) s.P[k] = params[k];
    __syncthreads();
    s.W2p[threadIdx.x >> 5][threadIdx.x & 31] = s.P[kP_W2 + threadIdx.x];
    __syncthreads();
    loss_grad_block(s.P, s.W2p, x, t, T, s.g, s.G, &s.loss);
    for (int k = threadIdx.x; k < kRmiParams; k += kTrainThreads) grad[k] = s.G[k];
    if (threadIdx.x == 0) *loss = s.loss;
}

// Features and targets of the sorted sample; T training points spread evenly.
__global__ void rmi_features_kernel(const uint64_t *__restrict__ S, uint32_t m, uint64_t kmin, int shift,
                                    uint32_t *__restrict__ Xi, float *__restrict__ xf, float *__restrict__ tf) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const uint32_t X = feature_of(S[j], kmin, shift);
        Xi[j] = X;
        xf[j] = (float)X * 5.9604644775390625e-8f;
        tf[j] = (float)(((double)j + 0.5) / (double)m);
    }
}

__global__ void __launch_bounds__(kTrainThreads)
rmi_train_kernel(const float *__restrict__ xf, uint32_t m, RmiModel *model, int steps, float lr) {
    extern __shared__ __align__(16) unsigned char train_smem[];
    TrainSmem &s = *reinterpret_cast<TrainSmem *>(train_smem);
    const int tid = threadIdx.x;
    const int T = (int)umin64(m, kRmiTrainPoints);
    for (int i = tid; i < T; i += kTrainThreads) {
        const uint32_t j = (uint32_t)(((uint64_t)i * m) / (uint64_t)T);
        s.X[i] = xf[j];
        s.T[i] = (float)(((double)j + 0.5) / (double)m);
    }
    // quantile init
    if (tid < kRmiHidden) {
        const float q0 = xf[umin64(m - 1, ((uint64_t)tid * m) / kRmiHidden)];
        const float q1 = tid + 1 < kRmiHidden ? xf[umin64(m - 1, ((uint64_t)(tid + 1) * m) / kRmiHidden)] : xf[m - 1];
        const float width = q1 - q0;
        const float w = (width * kMaxSlope <= 1.0f) ? kMaxSlope : 1.0f / width;
        s.P[kP_W1 + tid] = w;
        s.P[kP_B1 + tid] = -q0 * w;
        s.P[kP_B2 + tid] = 0.f;
        s.P[kP_W3 + tid] = 1.0f / kRmiHidden;
    }
    s.P[kP_W2 + tid] = ((tid >> 5) == (tid & 31)) ? 1.0f : 0.0f;
    if (tid == 0) s.P[kP_B3] = 0.f;
    __syncthreads();
    for (int step = 0; step <= steps; ++step) {
        s.W2p[tid >> 5][tid & 31] = s.P[kP_W2 + tid];
        __syncthreads();
        loss_grad_block(s.P, s.W2p, s.X, s.T, T, s.g, s.G, &s.loss);
        if (step == 0 && tid == 0) model->loss0 = s.loss;
        if (step == steps) break;
        // global gradient norm (fixed-order reduction), clip to 1
        float sq = 0.f;
        for (int k = tid; k < kRmiParams; k += kTrainThreads) sq = fmaf(s.G[k], s.G[k], sq);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
        if ((tid & 31) == 0) s.red[tid >> 5] = sq;
        __syncthreads();
        float tot = 0.f;
        for (int w = 0; w < kTrainThreads / 32; ++w) tot += s.red[w];
        const float scale = tot > 1.0f ? lr * rsqrtf(tot) : lr;
        for (int k = tid; k < kRmiParams; k += kTrainThreads) {
            float v = s.P[k] - scale * s.G[k];
            const bool weight = (k < kP_B1) || (k >= kP_W2 && k < kP_B2) || (k >= kP_W3 && k < kP_B3);
            if (weight) v = fmaxf(v, 0.f);  // projection keeps the root monotone
            s.P[k] = v;
        }
        __syncthreads();
    }
    for (int k = tid; k < kRmiParams; k += kTrainThreads) model->p[k] = s.P[k];
    if (tid == 0) model->loss1 = s.loss;
}

// thresh[l-1] = least X with root_leaf(X) >= l (bisection), l = 1..L-1.
__global__ void rmi_thresholds_kernel(RmiModel *model) {
    __shared__ float P[kRmiParams];
    for (int k = threadIdx.x; k < kRmiParams; k += blockDim.x) P[k] = model->p[k];
    __syncthreads();
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (l >= (uint32_t)kRmiLeaves) return;
    uint32_t lo = 0, hi = 1u << kRmiFeatureBits;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (root_leaf(P, mid) >= l) hi = mid; else lo = mid + 1;
    }
    model->thresh[l - 1] = lo;
}

// Make the table non-decreasing (prefix maximum), so table_leaf is monotone
// whatever the rounding of the root evaluation did.
constexpr int kFixThreads = 1024;
constexpr int kFixPer = kRmiLeaves / kFixThreads;  // 4

__global__ void __launch_bounds__(kFixThreads) rmi_table_fix_kernel(RmiModel *model) {
    __shared__ uint32_t s_warp[kFixThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t v[kFixPer];
    uint32_t run = 0;
#pragma unroll
    for (int u = 0; u < kFixPer; ++u) {
        const int i = tid * kFixPer + u;
        v[u] = i < kRmiLeaves - 1 ? model->thresh[i] : (1u << kRmiFeatureBits);
        run = max(run, v[u]);
    }
    uint32_t x = run;  // inclusive max-scan of thread maxima
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x = max(x, y);
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; ++w) pre = max(pre, s_warp[w]);
    const uint32_t xp = __shfl_up_sync(kFull, x, 1);
    run = max(pre, lane ? xp : 0u);  // maximum over earlier threads
#pragma unroll
    for (int u = 0; u < kFixPer; ++u) {
        const int i = tid * kFixPer + u;
        run = max(run, v[u]);
        if (i < kRmiLeaves) model->thresh[i] = i < kRmiLeaves - 1 ? run : (1u << kRmiFeatureBits);
    }
}

// leaf_start[l] = first sample index routed to a leaf >= l (the sample is
// sorted and routing is monotone); leaf_start[L] = m.
__global__ void rmi_leaf_start_kernel(const uint32_t *__restrict__ Xi, uint32_t m, RmiModel *model) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= m; j += stride) {
        const uint32_t lj = j < m ? table_leaf(model->thresh, Xi[j]) : (uint32_t)kRmiLeaves;
        const uint32_t lp = j > 0 ? table_leaf(model->thresh, Xi[j - 1]) : 0u;
        const uint32_t from = j > 0 ? lp + 1 : 0u;
        for (uint32_t l = from; l <= lj; ++l) model->leaf_start[l] = j;
    }
}

// Least squares per leaf over its contiguous sample range, FP64 sums in a
// fixed order (lane-strided, then a fixed shuffle tree); one warp per leaf.
__global__ void rmi_leaf_fit_kernel(const float *__restrict__ xf, const float *__restrict__ tf,
                                    const uint32_t *__restrict__ leaf_start, uint32_t m, int leaves,
                                    float *__restrict__ slope, float *__restrict__ icept, float *__restrict__ lo_out,
                                    float *__restrict__ hi_out) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp_id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t l = warp_id; l < (uint32_t)leaves; l += nwarps) {
        const uint32_t a = leaf_start[l], b = leaf_start[l + 1];
        double Sx = 0, Sy = 0, Sxx = 0, Sxy = 0;
        for (uint32_t j = a + lane; j < b; j += 32) {
            const double x = xf[j], y = tf[j];
            Sx += x;
            Sy += y;
            Sxx += x * x;
            Sxy += x * y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Sx += __shfl_xor_sync(kFull, Sx, o);
            Sy += __shfl_xor_sync(kFull, Sy, o);
            Sxx += __shfl_xor_sync(kFull, Sxx, o);
            Sxy += __shfl_xor_sync(kFull, Sxy, o);
        }
        if (lane == 0) {
            const double S = (double)(b - a);
            const double lo = m ? (double)a / m : 0.0, hi = m ? (double)b / m : 0.0;
            double k = 0.0, c = lo;
            if (b > a) {
                const double den = S * Sxx - Sx * Sx;
                if (b - a >= 2 && den > 0.0) k = (S * Sxy - Sx * Sy) / den;
                if (k < 0.0) k = 0.0;
                c = (Sy - k * Sx) / S;
            }
            slope[l] = (float)k;
            icept[l] = (float)c;
            lo_out[l] = (float)lo;
            hi_out[l] = (float)hi;
        }
    }
}

// kbase[l] = kmin + (T_l << shift), T_0 = 0, T_l = thresh[l-1]; kscale[l] =
// 2^-e, e = bit length of the leaf's key range (T_{l+1} - T_l) << shift.
__global__ void rmi_leaf_base_kernel(RmiModel *model) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= (uint32_t)kRmiLeaves) return;
    const uint64_t t0 = l == 0 ? 0u : model->thresh[l - 1];
    const uint64_t t1 = l + 1 < (uint32_t)kRmiLeaves ? model->thresh[l] : (1ull << kRmiFeatureBits);
    const int shift = model->shift;
    model->kbase[l] = model->kmin + (t0 << shift);
    const uint64_t range = t1 > t0 ? (t1 - t0) << shift : 0ull;
    const int e = range ? 64 - __clzll((long long)range) : 0;
    model->kscale[l] = range ? ldexpf(1.0f, -e) : 1.0f;
}

// Leaf-relative inputs of the sorted sample (the least-squares x).
__global__ void rmi_leaf_input_kernel(const uint64_t *__restrict__ S, const uint32_t *__restrict__ Xi, uint32_t m,
                                      const RmiModel *__restrict__ model, float *__restrict__ xf) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const uint32_t l = table_leaf(model->thresh, Xi[j]);
        const uint64_t kb = model->kbase[l];
        xf[j] = (float)(S[j] >= kb ? S[j] - kb : 0ull) * model->kscale[l];
    }
}

// ---- bucketing ---------------------------------------------------------------

constexpr int kBucketThreads = 512;

__device__ __forceinline__ uint32_t bucket_of(const RmiModel &M, const uint32_t *s_thresh, uint64_t key,
                                              uint64_t kmin, int shift, int bits, bool linear) {
    const uint32_t X = feature_of(key, kmin, shift);
    const float x = (float)X * 5.9604644775390625e-8f;
    float pos;
    if (linear) {
        pos = x;
    } else {
        const uint32_t l = table_leaf(s_thresh, X);
        const uint64_t kb = __ldg(&M.kbase[l]);
        const float xl = (float)(key >= kb ? key - kb : 0ull) * __ldg(&M.kscale[l]);
        pos = fminf(fmaxf(fmaf(__ldg(&M.slope[l]), xl, __ldg(&M.icept[l])), __ldg(&M.lo[l])), __ldg(&M.hi[l]));
    }
    const float B = (float)(1u << bits);
    const float v = fminf(fmaxf(pos * B, 0.0f), B - 1.0f);
    return (uint32_t)v;
}

__global__ void __launch_bounds__(kBucketThreads)
rmi_bucket_kernel(const uint64_t *__restrict__ keys, uint64_t n, const RmiModel *__restrict__ model, int bits,
                  int linear, uint32_t *__restrict__ buckets, uint32_t *__restrict__ vals,
                  unsigned long long *__restrict__ hist) {
    __shared__ uint32_t s_thresh[kRmiLeaves];
    __shared__ uint32_t s_hist[kSegPasses * kBins];
    for (int i = threadIdx.x; i < kRmiLeaves; i += kBucketThreads) s_thresh[i] = model->thresh[i];
    for (int i = threadIdx.x; i < kSegPasses * kBins; i += kBucketThreads) s_hist[i] = 0;
    __syncthreads();
    const uint64_t kmin = model->kmin;
    const int shift = model->shift;
    const uint64_t stride = (uint64_t)gridDim.x * kBucketThreads;
    const uint64_t n_round = (n + 31) & ~31ull;  // whole warps iterate together
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    for (uint64_t i = (uint64_t)blockIdx.x * kBucketThreads + threadIdx.x; i < n_round; i += stride) {
        const bool valid = i < n;
        uint32_t b = 0;
        if (valid) {
            b = bucket_of(*model, s_thresh, keys[i], kmin, shift, bits, linear != 0);
            buckets[i] = b;
            if (vals) vals[i] = (uint32_t)i;
        }
        if (hist) {
            for (int p = 0; p < passes; ++p)
                hist_add(s_hist + p * kBins, (b >> (kRadixBits * p)) & (kBins - 1), valid);
        }
    }
    __syncthreads();
    if (hist)
        for (int i = threadIdx.x; i < kSegPasses * kBins; i += kBucketThreads)
            if (s_hist[i]) atomicAdd(&hist[kKeyPasses * kBins + i], (unsigned long long)s_hist[i]);
}

// ---- composite keys: the bucket id above the key -------------------------------
//
// When the sort key has kb bits and the bucket id fits above it, the
// partition moves one word per element, (bucket << kb) | key, instead of a
// key and a separate bucket id.  Leaves are found through an index over the
// top 12 feature bits: slice s of the 24-bit feature holds only the leaves
// between the leaf of its first value and the leaf of the next slice's first
// value (the threshold table is non-decreasing), so the bisection runs over
// those few leaves instead of all 4096; each leaf's parameters are one
// 32-byte record.  The compose kernel holds all 4096 records (128 KB) in
// shared memory, one CTA of 1024 threads per SM: from L1/L2 the records'
// loads were its longest waits.
constexpr int kAccel = 1 << kRmiAccelBits;
constexpr int kAccelShift = kRmiFeatureBits - kRmiAccelBits;
constexpr int kCmpThreads = 1024;
constexpr int kCmpItems = 4;
using LeafPk = RmiModel::LeafPk;
static_assert(sizeof(LeafPk) == 32, "one leaf record is two 16-byte loads");

// The index and the leaf records, once per model (after the leaf fits).
__global__ void rmi_pack_kernel(RmiModel *model) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= (uint32_t)kAccel) model->accel[i] = (uint16_t)table_leaf(model->thresh, i << kAccelShift);
    if (i < (uint32_t)kRmiLeaves) {
        LeafPk r;
        r.kbase = model->kbase[i];
        r.kscale = model->kscale[i];
        r.slope = model->slope[i];
        r.icept = model->icept[i];
        r.lo = model->lo[i];
        r.hi = model->hi[i];
        r.pad = 0.f;
        model->leafpk[i] = r;
    }
}

// table_leaf(X) restricted to the leaves of X's slice: the largest l in
// [s_accel[s], s_accel[s + 1]] with l == 0 or thresh[l - 1] <= X.
__device__ __forceinline__ uint32_t accel_leaf(const uint32_t *s_thresh, const uint16_t *s_accel, uint32_t X) {
    const uint32_t sl = X >> kAccelShift;
    uint32_t lo = s_accel[sl], hi = s_accel[sl + 1];
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (s_thresh[mid - 1] <= X) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// bucket_of (trained model) with the indexed leaf search: the same
// arithmetic.  pk: the leaf records in shared memory.
__device__ __forceinline__ uint32_t bucket_fast(const LeafPk *pk, const uint32_t *s_thresh,
                                                const uint16_t *s_accel, uint64_t key, uint64_t kmin, int shift,
                                                float B) {
    const uint32_t X = feature_of(key, kmin, shift);
    const uint32_t l = accel_leaf(s_thresh, s_accel, X);
    const ulonglong2 r0 = *reinterpret_cast<const ulonglong2 *>(pk + l);
    const float4 r1 = *(reinterpret_cast<const float4 *>(pk + l) + 1);
    const uint64_t kbase = r0.x;
    const float kscale = __uint_as_float((unsigned)r0.y), slope = __uint_as_float((unsigned)(r0.y >> 32));
    const float icept = r1.x, lo = r1.y, hi = r1.z;
    const float xl = (float)(key >= kbase ? key - kbase : 0ull) * kscale;
    const float pos = fminf(fmaxf(fmaf(slope, xl, icept), lo), hi);
    return (uint32_t)fminf(fmaxf(pos * B, 0.0f), B - 1.0f);
}

// keys[i] |= bucket(keys[i]) << kb in place, with the 9-bit digit histograms
// of the bucket ids in hist rows 0..passes-1.  Four keys a thread are loaded
// before any is bucketed, so their loads overlap.
__global__ void __launch_bounds__(kCmpThreads)
rmi_compose_kernel(uint64_t *__restrict__ keys, uint64_t n, const RmiModel *__restrict__ model, int bits, int kb,
                   unsigned long long *__restrict__ hist) {
    extern __shared__ __align__(16) unsigned char cmp_smem[];
    LeafPk *s_leaf = reinterpret_cast<LeafPk *>(cmp_smem);
    uint32_t *s_thresh = reinterpret_cast<uint32_t *>(s_leaf + kRmiLeaves);
    uint16_t *s_accel = reinterpret_cast<uint16_t *>(s_thresh + kRmiLeaves);
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_accel + kAccel + 8);
    for (int i = threadIdx.x; i < kRmiLeaves * 2; i += kCmpThreads)
        reinterpret_cast<uint4 *>(s_leaf)[i] = reinterpret_cast<const uint4 *>(model->leafpk)[i];
    for (int i = threadIdx.x; i < kRmiLeaves; i += kCmpThreads) s_thresh[i] = model->thresh[i];
    for (int i = threadIdx.x; i < (kAccel + 8) / 8; i += kCmpThreads)
        reinterpret_cast<uint4 *>(s_accel)[i] = reinterpret_cast<const uint4 *>(model->accel)[i];
    for (int i = threadIdx.x; i < 3 * kBins; i += kCmpThreads) s_hist[i] = 0;
    __syncthreads();
    const uint64_t kmin = model->kmin;
    const int shift = model->shift;
    const float B = (float)(1u << bits);
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    const LeafPk *pk = s_leaf;
    constexpr uint64_t kGroup = (uint64_t)kCmpThreads * kCmpItems;
    for (uint64_t g = (uint64_t)blockIdx.x * kGroup; g < n; g += (uint64_t)gridDim.x * kGroup) {
        uint64_t key[kCmpItems];
#pragma unroll
        for (int k = 0; k < kCmpItems; ++k) {
            const uint64_t i = g + (uint64_t)k * kCmpThreads + threadIdx.x;
            key[k] = i < n ? keys[i] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < kCmpItems; ++k) {
            const uint64_t i = g + (uint64_t)k * kCmpThreads + threadIdx.x;
            if (i < n) {
                const uint32_t b = bucket_fast(pk, s_thresh, s_accel, key[k], kmin, shift, B);
                keys[i] = key[k] | ((uint64_t)b << kb);
                for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p * kBins + ((b >> (kRadixBits * p)) & (kBins - 1))], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kBins; i += kCmpThreads)
        if (s_hist[i]) atomicAdd(&hist[i], (unsigned long long)s_hist[i]);
}

// ---- in-bucket sorts over windows of whole buckets ------------------------------
//
// After the partition the composite keys are grouped by bucket in bucket
// order, and the bucket is a non-decreasing function of the key, so sorting
// any run of whole buckets by key alone puts it in its final order.  A CTA
// claims ranges of kTsRange positions and takes every bucket that starts in
// its range: it loads the next window of keys, cuts it after the last bucket
// that ends inside, and sorts that window in shared memory.  Each element
// becomes one word, (key - min(window)) << place bits | its place in the
// window, so the payload is fetched once, at the end; a stable LSD radix
// sort on the key part, 9 bits a pass, takes as many passes as the window's
// key span needs, the words held in registers between passes.  The CTA then
// writes the permutation and queues the window's runs of equal keys that
// hold an inexactly coded string for the fix-up (equal keys share a bucket,
// so no run crosses a window).  A bucket longer than the window is queued;
// a second kernel with windows twice as long (one CTA per SM) sorts those it
// can hold, and the overflow sort takes the rest.
constexpr uint64_t kTsRange = 1ull << 18;

template <int THREADS, int ITEMS, bool RANK_REGS, int MIN_BLOCKS>
struct TsShape {
    static constexpr bool kRankRegs = RANK_REGS;  // ranks in registers (else in shared memory)
    static constexpr int kMinBlocks = MIN_BLOCKS;  // CTAs per SM the launch bounds ask for
    static constexpr int kThreads = THREADS;
    static constexpr int kWarps = THREADS / 32;
    static constexpr int kItems = ITEMS;
    static constexpr int kWin = THREADS * ITEMS;
    static constexpr int kIdxBits = kWin <= (1 << 13) ? 13 : 14;
    static_assert(kWin <= (1 << kIdxBits), "the place field indexes the window");
    static_assert(THREADS % 32 == 0 && ITEMS % 4 == 0, "whole warps, whole groups of four items");
    static_assert(kWin < (1 << 16), "per-warp counts and offsets within a digit fit 16 bits");
    // Per-warp digit counts are 16-bit, two to a word for the shared
    // atomics; after the digit phase the same halves hold each warp's first
    // place for the digit in the window.  Ranks go to shared memory rather
    // than registers, which keeps the register count at 64.
    struct Smem {
        uint64_t word[kWin];
        uint32_t whist2[kWarps * kBins / 2];
        uint16_t rank[kWin];
        uint32_t heads[kWin / 32];
        RunEntry runs[512];  // the window's small tie runs, queued together
        uint32_t wsum[kWarps];
        unsigned long long kmin, kmax, found, rbase;
        unsigned int cut, job, nruns;
    };
};
// Two CTAs per SM: measured faster than 12288-key windows at one CTA per
// SM (skewed_1e9: 28.5 vs 34.6 ms for the in-bucket sorts).
using TsMain = TsShape<512, 12, true, 2>;   // windows cut from ranges
using TsBig = TsShape<1024, 12, false, 1>;  // one oversize bucket at a time, one CTA per SM
static_assert(64 - TsBig::kIdxBits >= kTsMaxKeyBits && 64 - TsMain::kIdxBits >= kTsMaxKeyBits,
              "every shape's words hold a key span of kTsMaxKeyBits");

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kFull, v, o);
        v = y < v ? y : v;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kFull, v, o);
        v = y > v ? y : v;
    }
    return v;
}

// A run of equal keys [start, start + len) that needs the fix-up, to its
// size-class queue.
__device__ void queue_run(const RunQueues &q, DevFlags *flags, uint64_t start, uint64_t len) {
    if (start >= q.perm_n || len > q.perm_n - start) {
        atomicOr(&flags->error, kErrInternal);
        return;
    }
    const RunEntry e{start, (unsigned)umin64(len, 0xFFFFFFFFull), 0u};
    if (len <= kSmallMax) {
        const unsigned long long i = atomicAdd(&flags->qcount[kQSmall], 1ull);
        if (i < q.cap_small) q.small[i] = e; else atomicOr(&flags->error, kErrInternal);
    } else if (len <= kMediumMax) {
        const unsigned long long i = atomicAdd(&flags->qcount[kQMedium], 1ull);
        if (i < q.cap_medium) q.medium[i] = e; else atomicOr(&flags->error, kErrInternal);
    } else {
        const unsigned long long i = atomicAdd(&flags->qcount[kQLargeA], 1ull);
        if (i < q.cap_large && len < 0xFFFFFFFFull) q.large[i] = e; else atomicOr(&flags->error, kErrInternal);
    }
}

// A bucket longer than a window, to a queue of RunEntry (count in *count).
__device__ void queue_bucket(RunEntry *qb, unsigned long long *count, uint64_t cap, DevFlags *flags, uint64_t start,
                             uint64_t len) {
    const unsigned long long i = atomicAdd(count, 1ull);
    if (i < cap && len < 0xFFFFFFFFull) qb[i] = RunEntry{start, (unsigned)len, 0u};
    else atomicOr(&flags->error, kErrInternal);
}

// First position >= from whose bucket (key >> kb) is not b, or n.  Every key
// at or after `from` has a bucket >= b.  Block-wide (all threads call it and
// get the same value): one coalesced look at the next window of keys, then,
// if the bucket runs on past them, a galloping search and a bisection.
template <class S>
__device__ uint64_t bucket_end(const uint64_t *__restrict__ keys, uint64_t n, int kb, uint64_t from, uint64_t b,
                               typename S::Smem &s) {
    if (threadIdx.x == 0) s.found = ~0ull;
    __syncthreads();
    unsigned long long best = ~0ull;
#pragma unroll
    for (int k = 0; k < S::kItems; ++k) {
        const uint64_t j = from + (uint64_t)k * S::kThreads + threadIdx.x;
        if (j < n && (keys[j] >> kb) != b && j < best) best = j;
    }
    best = warp_min_u64(best);
    if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&s.found, best);
    __syncthreads();
    unsigned long long f = s.found;
    if (f == ~0ull) {
        if (from + S::kWin >= n) {
            f = n;
        } else {
            if (threadIdx.x == 0) {  // keys [from, from + kWin) are all in bucket b
                uint64_t lo = from + S::kWin - 1, step = S::kWin, hi;
                for (;;) {
                    hi = lo + step;
                    if (hi >= n) {
                        hi = n;
                        break;
                    }
                    if ((keys[hi] >> kb) != b) break;
                    lo = hi;
                    step <<= 1;
                }
                while (hi - lo > 1) {  // bucket(lo) == b, hi == n or bucket(hi) != b
                    const uint64_t mid = lo + ((hi - lo) >> 1);
                    if ((keys[mid] >> kb) == b) lo = mid; else hi = mid;
                }
                s.found = hi;
            }
            __syncthreads();
            f = s.found;
        }
    }
    __syncthreads();
    return f;
}

// Exclusive scan of one u32 per thread over the block.
template <class S>
__device__ __forceinline__ uint32_t ts_exclusive_scan(uint32_t v, uint32_t *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t pre = 0;
#pragma unroll
    for (int w = 0; w < S::kWarps; ++w) pre += w < warp ? wsum[w] : 0u;
    return pre + x - v;
}

// The CTA's small tie runs gathered in shared memory go to the small-run
// queue with one global atomic for all of them.  Call with every thread,
// after a barrier that follows the last write to s.runs.
template <class S>
__device__ void flush_runs(typename S::Smem &s, const RunQueues &q, DevFlags *flags) {
    const unsigned int cnt = min(s.nruns, 512u);
    if (cnt) {
        if (threadIdx.x == 0) s.rbase = atomicAdd(&flags->qcount[kQSmall], (unsigned long long)cnt);
        __syncthreads();
        const unsigned long long rb = s.rbase;
        for (unsigned int t = threadIdx.x; t < cnt; t += S::kThreads) {
            if (rb + t < q.cap_small) q.small[rb + t] = s.runs[t];
            else atomicOr(&flags->error, kErrInternal);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) s.nruns = 0;
}

// Windows keep adding small runs to the CTA's buffer until it is half full;
// a run that finds it full goes to the queue on its own.
constexpr unsigned kRunFlushAt = 256;

// Sorts elements [0, cut) of a window held in w (item k of lane l of warp wp
// is element 32 * ITEMS * wp + 32k + l; w[k] its composite key, anything at
// or past cut), writes their payload in key order to perm[pos ..] and, with
// ties set, queues the window's runs of equal keys whose bit 0 (not exact)
// is set.  On entry s.kmin = ~0 and s.kmax = 0 are visible to every thread;
// returns after a barrier.
template <class S, typename IdxT>
__device__ void sort_window(typename S::Smem &s, uint64_t (&w)[S::kItems], uint64_t pos, uint32_t cut,
                            uint64_t kmask, const uint32_t *__restrict__ vals_in, IdxT *__restrict__ perm,
                            bool ties, const RunQueues &q, DevFlags *flags) {
    constexpr int IB = S::kIdxBits;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t wb = (uint32_t)warp * 32 * S::kItems;
    uint32_t *mh2 = s.whist2 + warp * (kBins / 2);
    const uint16_t *mh16 = reinterpret_cast<const uint16_t *>(mh2);

    unsigned long long lo = ~0ull, hi = 0;
#pragma unroll
    for (int k = 0; k < S::kItems; ++k) {
        const uint32_t e = wb + k * 32 + lane;
        if (e < cut) {
            const uint64_t v = w[k] & kmask;
            lo = v < lo ? v : lo;
            hi = v > hi ? v : hi;
        }
    }
    lo = warp_min_u64(lo);
    hi = warp_max_u64(hi);
    if (lane == 0 && lo != ~0ull) {
        atomicMin(&s.kmin, lo);
        atomicMax(&s.kmax, hi);
    }
    __syncthreads();
    const uint64_t wmin = s.kmin;
    const uint64_t span = s.kmax - wmin;
    const int npass = span ? (64 - __clzll((long long)span) + kRadixBits - 1) / kRadixBits : 0;
    // elements past the cut sort after every element of the window
#pragma unroll
    for (int k = 0; k < S::kItems; ++k) {
        const uint32_t e = wb + k * 32 + lane;
        w[k] = e < cut ? (((w[k] & kmask) - wmin) << IB) | e : ~0ull;
    }
    if (npass == 0) {  // one key value: the window is in order
#pragma unroll
        for (int k = 0; k < S::kItems; ++k) s.word[wb + k * 32 + lane] = w[k];
        __syncthreads();
    }
    for (int qp = 0; qp < npass; ++qp) {
        const int sh = IB + qp * kRadixBits;
        for (int i = tid; i < S::kWarps * kBins / 2; i += S::kThreads) s.whist2[i] = 0;
        __syncthreads();
        // rank among the warp's earlier elements with the same digit, four
        // peer masks in flight (the match instruction, or ballots when the
        // warp's first item holds many distinct digits, prefer_ballots: each
        // form unrolled on its own); each leader's add is ordered before the
        // next item's by the __syncwarp (stability)
        uint32_t rankp[S::kItems / 2];
#pragma unroll
        for (int k = 0; k < S::kItems / 2; ++k) rankp[k] = 0;
        unsigned peers0 = 0;
        auto rank_items = [&](auto by_ballots) {
            constexpr bool BALLOTS = decltype(by_ballots)::value;
#pragma unroll
            for (int g = 0; g < S::kItems; g += 4) {
                unsigned peers[4], before[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned d = (unsigned)(w[g + u] >> sh) & (kBins - 1);
                    peers[u] = g + u == 0 ? peers0 : BALLOTS ? match_by_ballots(d) : __match_any_sync(kFull, d);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned d = (unsigned)(w[g + u] >> sh) & (kBins - 1);
                    before[u] = 0;
                    if (lane == __ffs(peers[u]) - 1) {
                        const unsigned half = 16 * (d & 1);
                        before[u] = (atomicAdd(&mh2[d >> 1], (unsigned)__popc(peers[u]) << half) >> half) & 0xFFFFu;
                    }
                    __syncwarp();
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned bb = __shfl_sync(kFull, before[u], __ffs(peers[u]) - 1);
                    const unsigned rk = bb + __popc(peers[u] & lanemask_lt());
                    if (S::kRankRegs) rankp[(g + u) / 2] |= rk << (16 * ((g + u) & 1));
                    else s.rank[wb + (g + u) * 32 + lane] = (uint16_t)rk;
                }
            }
        };
        peers0 = __match_any_sync(kFull, (unsigned)(w[0] >> sh) & (kBins - 1));  // also item 0's mask
        if (prefer_ballots(peers0))
            rank_items(std::true_type{});
        else
            rank_items(std::false_type{});
        __syncthreads();
        // digit tid: offsets over the warps (in place of the counts), then
        // the window's digit start
        uint32_t run = 0;
        if (tid < kBins) {
            uint16_t *col = reinterpret_cast<uint16_t *>(s.whist2) + tid;
#pragma unroll
            for (int w2 = 0; w2 < S::kWarps; ++w2) {
                const uint32_t c = col[w2 * kBins];
                col[w2 * kBins] = (uint16_t)run;
                run += c;
            }
        }
        const uint32_t ds = ts_exclusive_scan<S>(run, s.wsum);
        if (tid < kBins) {  // each warp's place for the digit, window-wide
            uint16_t *col = reinterpret_cast<uint16_t *>(s.whist2) + tid;
#pragma unroll
            for (int w2 = 0; w2 < S::kWarps; ++w2) col[w2 * kBins] = (uint16_t)(col[w2 * kBins] + ds);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < S::kItems; ++k) {
            const unsigned d = (unsigned)(w[k] >> sh) & (kBins - 1);
            const uint32_t rk = S::kRankRegs ? (rankp[k / 2] >> (16 * (k & 1))) & 0xFFFFu : s.rank[wb + k * 32 + lane];
            s.word[mh16[d] + rk] = w[k];
        }
        __syncthreads();
        if (qp + 1 < npass) {
#pragma unroll
            for (int k = 0; k < S::kItems; ++k) w[k] = s.word[wb + k * 32 + lane];
        }
    }
    // permutation (payload fetched through the place field) and run heads
    for (uint32_t c = warp; c < S::kWin / 32; c += S::kWarps) {
        const uint32_t j = c * 32 + lane;
        const bool v = j < cut;
        const uint64_t wj = v ? s.word[j] : 0ull;
        const uint64_t wp = (v && j > 0) ? s.word[j - 1] : 0ull;
        const bool head = v && (j == 0 || (wj >> IB) != (wp >> IB));
        const unsigned hb = __ballot_sync(kFull, head);
        if (lane == 0) s.heads[c] = hb;
        if (v) perm[pos + j] = (IdxT)vals_in[pos + (wj & ((1u << IB) - 1))];
    }
    if (ties) {
        __syncthreads();
        // a run needs the fix-up when it has two or more members and their
        // key's not-exact bit (bit 0) is set
        for (uint32_t c = warp; c * 32 < cut; c += S::kWarps) {
            const uint32_t j = c * 32 + lane;
            if (j < cut && ((s.heads[c] >> lane) & 1u)) {
                const uint64_t key = (s.word[j] >> IB) + wmin;
                if (key & 1ull) {
                    uint32_t end = cut;
                    const uint32_t later = lane == 31 ? 0u : (s.heads[c] & (~0u << (lane + 1)));
                    if (later) {
                        end = c * 32 + __ffs(later) - 1;
                    } else {
                        for (uint32_t c2 = c + 1; c2 * 32 < cut; ++c2)
                            if (s.heads[c2]) {
                                end = c2 * 32 + __ffs(s.heads[c2]) - 1;
                                break;
                            }
                    }
                    if (end > cut) end = cut;
                    const uint32_t len = end - j;
                    if (len >= 2) {
                        // small runs wait in shared memory: one queue update for many windows
                        const unsigned int slot = len <= kSmallMax ? atomicAdd(&s.nruns, 1u) : ~0u;
                        if (slot < 512u) s.runs[slot] = RunEntry{pos + j, len, 0u};
                        else queue_run(q, flags, pos + j, len);
                    }
                }
            }
        }
        __syncthreads();
        if (s.nruns >= kRunFlushAt) flush_runs<S>(s, q, flags);  // the same value in every thread
    }
    __syncthreads();
}

template <typename IdxT>
__global__ void __launch_bounds__(TsMain::kThreads, TsMain::kMinBlocks) bucket_tile_sort_kernel(const TileSortArgs a) {
    using S = TsMain;
    extern __shared__ __align__(16) unsigned char ts_raw[];
    S::Smem &s = *reinterpret_cast<S::Smem *>(ts_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t n = a.n;
    const int kb = a.kb;
    const uint64_t kmask = (1ull << kb) - 1;
    IdxT *perm = static_cast<IdxT *>(a.perm);
    const uint32_t wb = (uint32_t)warp * 32 * S::kItems;
    if (tid == 0) s.nruns = 0;
    for (;;) {
        if (tid == 0) {  // after an error elsewhere (a full queue) no more ranges are taken
            const unsigned int err = *(volatile const unsigned int *)&a.flags->error;
            s.job = err ? 0xFFFFFFFFu : atomicAdd(a.range_counter, 1u);
        }
        __syncthreads();
        const uint64_t r0 = (uint64_t)s.job * kTsRange;
        __syncthreads();
        if (r0 >= n) break;
        const uint64_t r1 = umin64(n, r0 + kTsRange);
        // the bucket holding position r0 - 1 belongs to an earlier range
        uint64_t pos = r0 == 0 ? 0 : bucket_end<S>(a.keys_in, n, kb, r0, a.keys_in[r0 - 1] >> kb, s);
        while (pos < r1) {
            const uint64_t avail = umin64((uint64_t)S::kWin, n - pos);
            if (tid == 0) {
                s.cut = 0;
                s.kmin = ~0ull;
                s.kmax = 0;
            }
            uint64_t w[S::kItems];
#pragma unroll
            for (int k = 0; k < S::kItems; ++k) {
                const uint32_t e = wb + k * 32 + lane;
                w[k] = e < avail ? a.keys_in[pos + e] : ~0ull;
            }
            __syncthreads();
            // e ends its bucket when the next element's bucket differs or
            // there is no next element; the window is cut after the last such e
            uint32_t mycut = 0;
#pragma unroll
            for (int k = 0; k < S::kItems; ++k) {
                const uint32_t e = wb + k * 32 + lane;
                uint64_t nxt = __shfl_down_sync(kFull, w[k], 1);
                const uint64_t wrap = __shfl_sync(kFull, w[k + 1 < S::kItems ? k + 1 : k], 0);
                if (lane == 31) nxt = wrap;
                if (e < avail) {
                    bool boundary = true;
                    if (pos + e + 1 < n) {
                        if (e + 1 >= avail || (lane == 31 && k == S::kItems - 1)) nxt = a.keys_in[pos + e + 1];
                        boundary = (w[k] >> kb) != (nxt >> kb);
                    }
                    if (boundary) mycut = e + 1;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mycut = max(mycut, __shfl_xor_sync(kFull, mycut, o));
            if (lane == 0 && mycut) atomicMax(&s.cut, mycut);
            __syncthreads();
            const uint32_t cut = s.cut;
            if (cut == 0) {  // one bucket fills the window and goes on
                const uint64_t b = a.keys_in[pos] >> kb;
                const uint64_t end = bucket_end<S>(a.keys_in, n, kb, pos + S::kWin, b, s);
                if (tid == 0)
                    queue_bucket(a.overflow, &a.flags->qcount[kQOverflow], a.cap_overflow, a.flags, pos, end - pos);
                pos = end;
                continue;
            }
            sort_window<S, IdxT>(s, w, pos, cut, kmask, a.vals_in, perm, a.ties != 0, a.q, a.flags);
            pos += cut;
        }
    }
    if (a.ties) flush_runs<S>(s, a.q, a.flags);
}

// The buckets the range kernel found longer than its window, one at a time
// in windows twice as long; longer ones go on to `rest`.
template <typename IdxT>
__global__ void __launch_bounds__(TsBig::kThreads, TsBig::kMinBlocks) bucket_run_sort_kernel(const RunSortArgs a) {
    using S = TsBig;
    extern __shared__ __align__(16) unsigned char ts_raw[];
    S::Smem &s = *reinterpret_cast<S::Smem *>(ts_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t kmask = (1ull << a.kb) - 1;
    IdxT *perm = static_cast<IdxT *>(a.perm);
    const uint32_t wb = (uint32_t)warp * 32 * S::kItems;
    if (tid == 0) s.nruns = 0;
    for (uint64_t r = blockIdx.x; r < a.count; r += gridDim.x) {
        const uint64_t pos = a.runs[r].start;
        const uint32_t len = a.runs[r].len;
        if (len > (uint32_t)S::kWin) {
            if (tid == 0) queue_bucket(a.rest, &a.flags->qcount[kQOverflow2], a.cap_rest, a.flags, pos, len);
            continue;
        }
        if (tid == 0) {
            s.kmin = ~0ull;
            s.kmax = 0;
        }
        uint64_t w[S::kItems];
#pragma unroll
        for (int k = 0; k < S::kItems; ++k) {
            const uint32_t e = wb + k * 32 + lane;
            w[k] = e < len ? a.keys_in[pos + e] : ~0ull;
        }
        __syncthreads();
        sort_window<S, IdxT>(s, w, pos, len, kmask, a.vals_in, perm, a.ties != 0, a.q, a.flags);
    }
    __syncthreads();
    if (a.ties) flush_runs<S>(s, a.q, a.flags);
}

// Runs of equal keys inside the overflow buckets (sorted keys, key bit 0 =
// not exact): a bucket whose first and last keys agree is one run; any other
// is walked by one CTA in chunks, carrying the head of the run open at each
// chunk's start.
constexpr int kOtThreads = 512;

__global__ void __launch_bounds__(kOtThreads)
oversize_ties_kernel(const RunEntry *__restrict__ runs, uint64_t count, const uint64_t *__restrict__ keys,
                     const RunQueues q, DevFlags *flags) {
    __shared__ unsigned long long s_wmax[kOtThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint64_t r = blockIdx.x; r < count; r += gridDim.x) {
        const uint64_t start = runs[r].start, len = runs[r].len;
        if (len == 0) continue;
        const uint64_t k0 = keys[start];
        if (keys[start + len - 1] == k0) {  // sorted: one key value, one run
            if (tid == 0 && len >= 2 && (k0 & 1ull)) queue_run(q, flags, start, len);
            continue;
        }
        unsigned long long open = start;  // head of the run open at the chunk start
        for (uint64_t c0 = 0; c0 < len; c0 += kOtThreads) {
            const uint64_t j = c0 + tid;
            const bool v = j < len;
            const uint64_t k = v ? keys[start + j] : 0ull;
            const bool head = v && (j == 0 || keys[start + j - 1] != k);
            const bool tail = v && (j + 1 == len || keys[start + j + 1] != k);
            // inclusive max-scan of head positions over the chunk
            unsigned long long h = head ? start + j : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kFull, h, o);
                if (lane >= o && y > h) h = y;
            }
            if (lane == 31) s_wmax[warp] = h;
            __syncthreads();
            unsigned long long pre = open;
            for (int w2 = 0; w2 < warp; ++w2) pre = s_wmax[w2] > pre ? s_wmax[w2] : pre;
            const unsigned long long run_head = h > pre ? h : pre;
            if (tail && (k & 1ull)) {
                const uint64_t rl = start + j - run_head + 1;
                if (rl >= 2) queue_run(q, flags, run_head, rl);
            }
            unsigned long long all = open;
            for (int w2 = 0; w2 < kOtThreads / 32; ++w2) all = s_wmax[w2] > all ? s_wmax[w2] : all;
            __syncthreads();
            open = all;
        }
    }
}

// first[b] / last[b]: positions of bucket b's first and last element after the
// stable partition (buckets are contiguous and in increasing order).
__global__ void bucket_bounds_kernel(const uint32_t *__restrict__ bk, uint64_t n, unsigned long long *__restrict__ first,
                                     unsigned long long *__restrict__ last) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint32_t b = bk[j];
        if (j == 0 || bk[j - 1] != b) first[b] = j;
        if (j + 1 == n || bk[j + 1] != b) last[b] = j;
    }
}

// Sort inside each bucket by key (stable: ties keep partition order, which is
// input order).  Buckets up to kBsRankMax keys: each key's rank counted
// against the others; up to kBucketCap: bitonic in shared memory on (key,
// position).  Larger buckets are queued: a grid-wide pass copies their
// payload and flags the ones holding different keys for the segmented
// overflow sort.  Writes keys back in place and the payload to the
// permutation.
constexpr int kBsThreads = 256;
constexpr int kBsRankMax = 256;  // rank counting (n^2 / 2 compares) up to here, bitonic above

template <typename IdxT>
__global__ void __launch_bounds__(kBsThreads)
bucket_sort_kernel(const unsigned long long *__restrict__ first, const unsigned long long *__restrict__ last,
                   uint64_t num_buckets, uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                   IdxT *__restrict__ perm, RunEntry *__restrict__ overflow, uint64_t cap_overflow,
                   DevFlags *flags) {
    extern __shared__ __align__(16) unsigned char bs_smem[];
    uint64_t *s_key = reinterpret_cast<uint64_t *>(bs_smem);
    uint32_t *s_pos = reinterpret_cast<uint32_t *>(s_key + kBucketCap);
    const int tid = threadIdx.x;
    for (uint64_t b = blockIdx.x; b < num_buckets; b += gridDim.x) {
        const unsigned long long f = first[b];
        if (f == ~0ull) continue;  // empty
        const uint64_t len = last[b] - f + 1;
        if (len > (uint64_t)kBucketCap) {  // handled grid-wide afterwards
            if (tid == 0) {
                const unsigned long long q = atomicAdd(&flags->qcount[kQOverflow], 1ull);
                if (q < cap_overflow && len < 0xFFFFFFFFull) overflow[q] = RunEntry{f, (uint32_t)len, 0u};
                else atomicOr(&flags->error, kErrInternal);
            }
            continue;
        }
        const int n_b = (int)len;
        __syncthreads();
        if (n_b <= kBsRankMax) {
            // rank of element i = number of elements before it in (key, position) order
            for (int j = tid; j < n_b; j += kBsThreads) s_key[j] = keys[f + j];
            __syncthreads();
            for (int i = tid; i < n_b; i += kBsThreads) {
                const uint64_t ki = s_key[i];
                int r = 0;
                for (int j = 0; j < i; ++j) r += s_key[j] <= ki;      // earlier: equal keys count
                for (int j = i + 1; j < n_b; ++j) r += s_key[j] < ki;  // later: only smaller keys
                keys[f + r] = ki;
                perm[f + r] = (IdxT)vals[f + i];
            }
            continue;
        }
        int P = 1;
        while (P < n_b) P <<= 1;
        bool unsorted = false;
        for (int j = tid; j < P; j += kBsThreads) {
            if (j < n_b) {
                s_key[j] = keys[f + j];
                s_pos[j] = (uint32_t)j;
            } else {
                s_key[j] = ~0ull;
                s_pos[j] = 0xFFFFFFFFu;
            }
        }
        __syncthreads();
        for (int j = tid; j + 1 < n_b; j += kBsThreads) unsorted |= s_key[j] > s_key[j + 1];
        if (__syncthreads_or(unsorted)) {
            for (int k = 2; k <= P; k <<= 1) {
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    for (int i = tid; i < P; i += kBsThreads) {
                        const int ixj = i ^ jj;
                        if (ixj > i) {
                            const bool up = (i & k) == 0;
                            const bool gt = s_key[i] != s_key[ixj] ? s_key[i] > s_key[ixj] : s_pos[i] > s_pos[ixj];
                            if (gt == up) {
                                const uint64_t tk = s_key[i]; s_key[i] = s_key[ixj]; s_key[ixj] = tk;
                                const uint32_t tp = s_pos[i]; s_pos[i] = s_pos[ixj]; s_pos[ixj] = tp;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int j = tid; j < n_b; j += kBsThreads) {
                keys[f + j] = s_key[j];
                perm[f + j] = (IdxT)vals[f + s_pos[j]];
            }
        } else {
            for (int j = tid; j < n_b; j += kBsThreads) perm[f + j] = (IdxT)vals[f + j];
        }
    }
}

// Oversize buckets, flattened over their elements: payload -> perm (and,
// when keys_out is given, key & kmask -> keys_out), and a flag for every
// bucket holding two different keys.
template <typename IdxT>
__global__ void big_bucket_kernel(const RunEntry *__restrict__ big, uint64_t count,
                                  const unsigned long long *__restrict__ base, uint64_t total,
                                  const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                                  IdxT *__restrict__ perm, uint32_t *__restrict__ mixed,
                                  uint64_t *__restrict__ keys_out, uint64_t kmask) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < total; a += stride) {
        uint64_t lo = 0, hi = count;
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (base[mid] <= a) lo = mid; else hi = mid;
        }
        const uint64_t start = big[lo].start;
        const uint64_t pos = start + (a - base[lo]);
        perm[pos] = (IdxT)vals[pos];
        if (keys_out) keys_out[pos] = keys[pos] & kmask;
        if (keys[pos] != keys[start] && mixed[lo] == 0u) mixed[lo] = 1u;
    }
}

__global__ void collect_mixed_kernel(const RunEntry *__restrict__ big, uint64_t count, const uint32_t *__restrict__ mixed,
                                     RunEntry *__restrict__ q_mixed, uint64_t cap, DevFlags *flags) {
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count || !mixed[r]) return;
    const unsigned long long q = atomicAdd(&flags->qcount[kQMixed], 1ull);
    if (q < cap) q_mixed[q] = big[r]; else atomicOr(&flags->error, kErrInternal);
}

// Overflow buckets: gather (key & kmask, bucket run id, payload) into
// compacted arrays, and scatter the sorted result back.
__global__ void overflow_gather_kernel(const RunEntry *__restrict__ runs, uint64_t count,
                                       const unsigned long long *__restrict__ run_base, uint64_t total,
                                       const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                                       uint64_t kmask, uint64_t *__restrict__ ck, uint32_t *__restrict__ cs,
                                       uint32_t *__restrict__ cv) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < total; a += stride) {
        uint64_t lo = 0, hi = count;
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (run_base[mid] <= a) lo = mid; else hi = mid;
        }
        const uint64_t pos = runs[lo].start + (a - run_base[lo]);
        ck[a] = keys[pos] & kmask;
        cs[a] = (uint32_t)lo;
        cv[a] = vals[pos];
    }
}

template <typename IdxT>
__global__ void overflow_scatter_kernel(const RunEntry *__restrict__ runs, const unsigned long long *__restrict__ run_base,
                                        uint64_t total, const uint64_t *__restrict__ ck, const uint32_t *__restrict__ cs,
                                        const uint32_t *__restrict__ cv, uint64_t *__restrict__ keys,
                                        IdxT *__restrict__ perm) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < total; a += stride) {
        const uint32_t r = cs[a];
        const uint64_t pos = runs[r].start + (a - run_base[r]);
        keys[pos] = ck[a];
        perm[pos] = (IdxT)cv[a];
    }
}

__global__ void rmi_sample_kernel(const uint64_t *__restrict__ keys, uint64_t n, uint64_t seed,
                                  uint64_t *__restrict__ out, uint32_t m) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += stride) {
        const uint64_t i = (uint64_t)k * kRmiStride + splitmix64((uint64_t)k ^ seed) % kRmiStride;
        out[k] = i < n ? keys[i] : keys[n - 1];
    }
}

__global__ void sample_index_kernel(uint64_t n, uint64_t seed, uint64_t *__restrict__ out, uint32_t m) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += stride)
        out[k] = (uint64_t)k * kRmiStride + splitmix64((uint64_t)k ^ seed) % kRmiStride;
}

size_t train_smem_bytes() { return sizeof(TrainSmem); }

cudaError_t set_train_attr() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(rmi_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem_bytes());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rmi_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem_bytes());
    if (e != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_rmi_sample(const uint64_t *keys, uint64_t n, uint64_t seed, uint64_t *out, uint32_t m,
                              cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    rmi_sample_kernel<<<(m + 255) / 256, 256, 0, s>>>(keys, n, seed, out, m);
    return cudaGetLastError();
}

cudaError_t launch_sample_indices(uint64_t n, uint64_t seed, uint64_t *out, uint32_t m, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    sample_index_kernel<<<(m + 255) / 256, 256, 0, s>>>(n, seed, out, m);
    return cudaGetLastError();
}

cudaError_t launch_rmi_train(const uint64_t *sorted_sample, uint32_t m, RmiModel *model, uint64_t kmin, int shift,
                             uint32_t *Xi, float *xf, float *tf, int steps, float lr, cudaStream_t s) {
    cudaError_t e = set_train_attr();
    if (e != cudaSuccess) return e;
    rmi_features_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_sample, m, kmin, shift, Xi, xf, tf);
    rmi_train_kernel<<<1, kTrainThreads, train_smem_bytes(), s>>>(xf, m, model, steps, lr);
    return cudaGetLastError();
}

cudaError_t launch_rmi_table(RmiModel *model, cudaStream_t s) {
    rmi_thresholds_kernel<<<(kRmiLeaves + 127) / 128, 128, 0, s>>>(model);
    rmi_table_fix_kernel<<<1, kFixThreads, 0, s>>>(model);
    return cudaGetLastError();
}

cudaError_t launch_rmi_leaves(const uint64_t *sorted_sample, const uint32_t *Xi, float *xf, const float *tf,
                              uint32_t m, RmiModel *model, cudaStream_t s) {
    rmi_leaf_start_kernel<<<(m + 256) / 256, 256, 0, s>>>(Xi, m, model);
    rmi_leaf_base_kernel<<<kRmiLeaves / 256, 256, 0, s>>>(model);
    rmi_leaf_input_kernel<<<(m + 255) / 256, 256, 0, s>>>(sorted_sample, Xi, m, model, xf);
    rmi_leaf_fit_kernel<<<kRmiLeaves / 8, 256, 0, s>>>(xf, tf, model->leaf_start, m, kRmiLeaves, model->slope,
                                                        model->icept, model->lo, model->hi);
    rmi_pack_kernel<<<(kAccel + 1 + 255) / 256, 256, 0, s>>>(model);
    return cudaGetLastError();
}

cudaError_t launch_big_buckets(const RunEntry *big, uint64_t count, const unsigned long long *base, uint64_t total,
                               const uint64_t *keys, const uint32_t *vals, void *perm, int perm_u64, uint32_t *mixed,
                               uint64_t *keys_out, uint64_t kmask, cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64((total + 255) / 256, 152ull * 16);
    if (perm_u64)
        big_bucket_kernel<uint64_t><<<grid, 256, 0, s>>>(big, count, base, total, keys, vals,
                                                         static_cast<uint64_t *>(perm), mixed, keys_out, kmask);
    else
        big_bucket_kernel<uint32_t><<<grid, 256, 0, s>>>(big, count, base, total, keys, vals,
                                                         static_cast<uint32_t *>(perm), mixed, keys_out, kmask);
    return cudaGetLastError();
}

cudaError_t launch_collect_mixed(const RunEntry *big, uint64_t count, const uint32_t *mixed, RunEntry *q_mixed,
                                 uint64_t cap, DevFlags *flags, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    collect_mixed_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(big, count, mixed, q_mixed, cap, flags);
    return cudaGetLastError();
}

cudaError_t launch_rmi_grad(const float *params, const float *x, const float *t, int T, float *grad, float *loss,
                            cudaStream_t s) {
    cudaError_t e = set_train_attr();
    if (e != cudaSuccess) return e;
    rmi_grad_kernel<<<1, kTrainThreads, train_smem_bytes(), s>>>(params, x, t, T, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_leaf_fit(const float *x, const float *t, const uint32_t *leaf_start, uint32_t m, int leaves,
                            float *slope, float *icept, float *lo, float *hi, cudaStream_t s) {
    const unsigned grid = (unsigned)((leaves + 7) / 8);
    rmi_leaf_fit_kernel<<<grid, 256, 0, s>>>(x, t, leaf_start, m, leaves, slope, icept, lo, hi);
    return cudaGetLastError();
}

cudaError_t launch_rmi_bucket(const uint64_t *keys, uint64_t n, const RmiModel *model, int bits, int linear,
                              uint32_t *buckets, uint32_t *vals, unsigned long long *hist, int num_sms,
                              cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + kBucketThreads * 8 - 1) / (kBucketThreads * 8);
    const unsigned grid = (unsigned)umin64(blocks, (uint64_t)num_sms * 4);
    rmi_bucket_kernel<<<grid, kBucketThreads, 0, s>>>(keys, n, model, bits, linear, buckets, vals, hist);
    return cudaGetLastError();
}

cudaError_t launch_bucket_bounds(const uint32_t *bk, uint64_t n, unsigned long long *first, unsigned long long *last,
                                 int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64((n + 255) / 256, (uint64_t)num_sms * 16);
    bucket_bounds_kernel<<<grid, 256, 0, s>>>(bk, n, first, last);
    return cudaGetLastError();
}

cudaError_t launch_bucket_sort(const unsigned long long *first, const unsigned long long *last, uint64_t num_buckets,
                               uint64_t *keys, const uint32_t *vals, void *perm, int perm_u64, RunEntry *overflow,
                               uint64_t cap_overflow, DevFlags *flags, int num_sms, cudaStream_t s) {
    const unsigned grid = (unsigned)umin64(num_buckets, (uint64_t)num_sms * 8);
    const size_t smem = (size_t)kBucketCap * 12;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(bucket_sort_kernel<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(bucket_sort_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (perm_u64)
        bucket_sort_kernel<uint64_t><<<grid, kBsThreads, smem, s>>>(first, last, num_buckets, keys, vals,
                                                                    static_cast<uint64_t *>(perm), overflow,
                                                                    cap_overflow, flags);
    else
        bucket_sort_kernel<uint32_t><<<grid, kBsThreads, smem, s>>>(first, last, num_buckets, keys, vals,
                                                                    static_cast<uint32_t *>(perm), overflow,
                                                                    cap_overflow, flags);
    return cudaGetLastError();
}

cudaError_t launch_overflow_gather(const RunEntry *runs, uint64_t count, const unsigned long long *run_base,
                                   uint64_t total, const uint64_t *keys, const uint32_t *vals, uint64_t kmask,
                                   uint64_t *ck, uint32_t *cs, uint32_t *cv, cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64((total + 255) / 256, 152ull * 16);
    overflow_gather_kernel<<<grid, 256, 0, s>>>(runs, count, run_base, total, keys, vals, kmask, ck, cs, cv);
    return cudaGetLastError();
}

cudaError_t launch_overflow_scatter(const RunEntry *runs, const unsigned long long *run_base, uint64_t total,
                                    const uint64_t *ck, const uint32_t *cs, const uint32_t *cv, uint64_t *keys,
                                    void *perm, int perm_u64, cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64((total + 255) / 256, 152ull * 16);
    if (perm_u64)
        overflow_scatter_kernel<uint64_t><<<grid, 256, 0, s>>>(runs, run_base, total, ck, cs, cv, keys,
                                                               static_cast<uint64_t *>(perm));
    else
        overflow_scatter_kernel<uint32_t><<<grid, 256, 0, s>>>(runs, run_base, total, ck, cs, cv, keys,
                                                               static_cast<uint32_t *>(perm));
    return cudaGetLastError();
}

cudaError_t launch_rmi_compose(uint64_t *keys, uint64_t n, const RmiModel *model, int bits, int kb,
                               unsigned long long *hist, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (bits < 1 || bits > 3 * kRadixBits || kb < 1 || kb + bits > 64) return cudaErrorInvalidValue;
    const uint64_t groups = (n + (uint64_t)kCmpThreads * kCmpItems - 1) / ((uint64_t)kCmpThreads * kCmpItems);
    const unsigned grid = (unsigned)umin64(groups, (uint64_t)num_sms);  // one CTA per SM (shared memory)
    constexpr size_t smem = kRmiLeaves * sizeof(LeafPk) + kRmiLeaves * 4 + (kAccel + 8) * 2 + 3 * kBins * 4;
    static_assert(((kAccel + 8) * 2) % 16 == 0, "the histogram stays 4-byte aligned");
    static bool configured = false;
    if (!configured) {
        const cudaError_t e =
            cudaFuncSetAttribute(rmi_compose_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    rmi_compose_kernel<<<grid, kCmpThreads, smem, s>>>(keys, n, model, bits, kb, hist);
    return cudaGetLastError();
}

template <class S, typename K64, typename K32>
cudaError_t set_smem_once(bool &done, K64 k64, K32 k32) {
    if (done) return cudaSuccess;
    const int smem = (int)sizeof(typename S::Smem);
    cudaError_t e = cudaFuncSetAttribute(k64, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_bucket_tile_sort(const TileSortArgs &a, int perm_u64, int num_sms, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (a.kb < 1 || a.kb > kTsMaxKeyBits) return cudaErrorInvalidValue;
    static bool configured = false;
    cudaError_t e = set_smem_once<TsMain>(configured, bucket_tile_sort_kernel<uint64_t>,
                                          bucket_tile_sort_kernel<uint32_t>);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(TsMain::Smem);
    const uint64_t ranges = (a.n + kTsRange - 1) / kTsRange;
    const unsigned grid = (unsigned)umin64(ranges, (uint64_t)num_sms * TsMain::kMinBlocks);
    if (perm_u64)
        bucket_tile_sort_kernel<uint64_t><<<grid, TsMain::kThreads, smem, s>>>(a);
    else
        bucket_tile_sort_kernel<uint32_t><<<grid, TsMain::kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bucket_run_sort(const RunSortArgs &a, int perm_u64, int num_sms, cudaStream_t s) {
    if (a.count == 0) return cudaSuccess;
    if (a.kb < 1 || a.kb > kTsMaxKeyBits) return cudaErrorInvalidValue;
    static bool configured = false;
    cudaError_t e = set_smem_once<TsBig>(configured, bucket_run_sort_kernel<uint64_t>,
                                         bucket_run_sort_kernel<uint32_t>);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(TsBig::Smem);
    const unsigned grid = (unsigned)umin64(a.count, (uint64_t)num_sms);
    if (perm_u64)
        bucket_run_sort_kernel<uint64_t><<<grid, TsBig::kThreads, smem, s>>>(a);
    else
        bucket_run_sort_kernel<uint32_t><<<grid, TsBig::kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_oversize_ties(const RunEntry *runs, uint64_t count, const uint64_t *keys, const RunQueues &q,
                                 DevFlags *flags, int num_sms, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64(count, (uint64_t)num_sms * 4);
    oversize_ties_kernel<<<grid, kOtThreads, 0, s>>>(runs, count, keys, q, flags);
    return cudaGetLastError();
}

}  // namespace hs
