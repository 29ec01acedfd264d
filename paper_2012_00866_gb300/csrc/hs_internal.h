// Host-side internal interface between the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "hs_device.cuh"

namespace hs {

// ---- encode.cu -----------------------------------------------------------
// Step 1 over n strings.  Writes per string either the husky code or, with
// key_flag (ASCII7 only), the sort key (code << 1) | not_exact; optionally
// the non-exact bitmask (bit i of word i/32) and the 8 digit histograms of
// what it wrote (8 x kBins u64, accumulated); sets flags.
// Batched packing for the encoder (byte-range coder only): the instance id
// of string i goes above its key (key_bits + seg_bits <= 64), vals[i] gets
// its local index; tile_seg[t] = instance of string t * 1024 (t <= tiles).
struct EncPack {
    const uint64_t *seg_offsets;  // nullptr: no packing
    uint64_t num_segs;
    int seg_bits;
    uint32_t *vals;
    const uint32_t *tile_seg;
    int spec_range;               // byte-range coder: use flags->alpha_spec_* (the range of a first chunk)
    // Single sorts, byte-range coder: when 8w + idx_bits <= 64 the encoder
    // writes (code << idx_bits) | (idx_base + i) -- the string's index below
    // its code, no not-exact bit in the key (it goes to nonexact_bits) --
    // and sets flags->idx_packed.  0: never.
    int idx_bits;
    uint64_t idx_base;            // index of the launch's first string
    // Sorted-input test after the encode (single sorts): see launch_sorted_test.
    int sorted_check;
    uint64_t *pairs;
    uint64_t pairs_cap;
};
// Sorted-input test over n encoded keys: flags->descent |= 1 if some key is
// below its predecessor's (the code above a packed index when the encoder set
// flags->idx_packed); otherwise the equal-key pairs not both exact (the
// not-exact bit in the key when flag_in_key and unpacked, else in the bitmap)
// are queued in pairs[] by the index of their first string, counted in
// flags->pairs.
cudaError_t launch_sorted_test(const uint64_t *keys, const uint32_t *nonexact_bits, uint64_t n, bool flag_in_key,
                               int idx_bits, uint64_t *pairs, uint64_t pairs_cap, DevFlags *flags, int num_sms,
                               cudaStream_t s);
// Numeric coders: codes[i] of values[i] (type as hs_numeric), or for a
// 32-bit type with pack_bits > 0 the word (code << pack_bits) | i; with hist
// the 8 digit histograms of the codes (accumulated).
cudaError_t launch_numeric_encode(const void *values, uint64_t n, int type, uint64_t *codes,
                                  unsigned long long *hist, int num_sms, cudaStream_t s, int pack_bits = 0);
// flags->descent |= 1 if some queued pair i (strings pairs[i], pairs[i] + 1)
// is out of order; count = flags->pairs as the host read it.
cudaError_t launch_pairs_ordered(const uint8_t *bytes, const uint64_t *offsets, const uint64_t *pairs,
                                 uint64_t count, DevFlags *flags, int num_sms, cudaStream_t s);
// tile_seg[t] for t = 0 .. ceil(n / 1024): the instance holding string
// min(t * 1024, n - 1).
cudaError_t launch_tile_segs(const uint64_t *seg_offsets, uint64_t num_segs, uint64_t n, uint32_t *tile_seg,
                             cudaStream_t s);
// coder 3 (byte range): values from flags->alpha_lo_inv / alpha_hi; writes
// alpha_w / alpha_k (keys of at most alpha_max_bits bits) and, when the range
// needs more than alpha_max_w bits or 9 chars do not fit, encodes as ASCII7.
// Digit histograms count the key without a packed index.
cudaError_t launch_encode(int coder, bool key_flag, const uint8_t *bytes,
                          const uint64_t *offsets, uint64_t n, uint64_t *codes,
                          uint32_t *nonexact_bits, unsigned long long *hist,
                          DevFlags *flags, int num_sms, cudaStream_t s, int alpha_max_w = 6,
                          int alpha_max_bits = 64, EncPack pack = EncPack{});
// Smallest / largest byte of bytes[offsets[0] .. offsets[n]) max-reduced into
// flags->alpha_lo_inv (as 255 - min) and flags->alpha_hi; cut short once the
// range is known to exceed max_span values.
cudaError_t launch_alphabet(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, int max_span,
                            DevFlags *flags, int num_sms, cudaStream_t s);

// ---- sort.cu -------------------------------------------------------------
constexpr int kSortThreads = 512;  // threads per onesweep CTA
constexpr int kSortMinBlocks = 2;  // onesweep CTAs resident per SM (register budget)
constexpr int kSortTile = 4096;    // elements per onesweep tile
inline uint64_t sort_tiles(uint64_t n) { return (n + kSortTile - 1) / kSortTile; }

// Digit plan.  A 64-bit key has 8 digits: seven of 9 bits (bits 0..62) and
// the top bit alone; a 32-bit segment id has 4 digits of 9 bits.  Histogram
// index p: 0..7 key digits, 8..11 segment digits.
constexpr int kKeyPasses = 8;
constexpr int kSegPasses = 4;
constexpr int kHistPasses = kKeyPasses + kSegPasses;
__host__ __device__ inline int digit_shift(int p) {
    return p < 7 ? kRadixBits * p : (p == 7 ? 63 : kRadixBits * (p - 8));
}
__host__ __device__ inline unsigned digit_mask(int p) { return p == 7 ? 1u : (unsigned)(kBins - 1); }

enum OutMode { kOutVals = 0, kOutPerm32 = 1, kOutPerm64 = 2 };

struct OnesweepArgs {
    const uint64_t *keys_in;
    uint64_t *keys_out;          // nullable: keys not needed downstream
    const uint32_t *segs_in;     // segmented sorts only
    uint32_t *segs_out;
    const uint32_t *vals_in;     // nullable when vals are synthesised
    void *vals_out;
    const uint32_t *flag_bits;   // synthesised vals: bit 31 source (nullable)
    uint64_t n;
    int pack_bits;               // > 0: elements are (key << pack_bits) | index, no vals
    int shift;                   // digit = (source >> shift) & mask
    unsigned mask;
    const unsigned long long *bucket_base;  // kBins entries for this pass
    uint64_t *lookback;          // sort_tiles(n) * kBins words
    uint32_t epoch;              // look-back epoch of this launch (1..63)
    unsigned int *tile_counter;  // zeroed
    DevFlags *flags;
};

// One stable LSD pass.  has_seg: elements carry a u32 segment id; digit_seg:
// the digit comes from the segment id instead of the key; synth: vals are
// generated as i | flag_bit(i) << 31; out: what vals_out receives.  With
// a.pack_bits > 0 the keys are packed (key, index) words and nothing else
// moves: kOutVals writes the words to keys_out, kOutPerm32/64 the indices
// to vals_out (and the words to keys_out as well when it is set).
// items: keys per thread, 0 (the default shape) or one of onesweep_shapes()
// (segmented passes always use 8).
cudaError_t launch_onesweep(const OnesweepArgs &a, bool has_seg,
                            bool digit_seg, bool synth, OutMode out,
                            cudaStream_t s, int items = 0);
// Bounded-wait test support on the current device: the onesweep look-back's
// poll budget (0: the default kSpinLimit) and a tile id whose look-back words
// are never published (-1: none).
cudaError_t set_wait_test(uint32_t spin_limit, long long withhold_tile);
// The tile shapes (keys per thread) unsegmented passes can run with; [0] is
// the default.
constexpr int kOnesweepShapes[2] = {12, 8};

// Digit histograms of keys (8 digits) and optionally segs (4 digits):
// hist[p * kBins + d], p < 8 for keys, 8..11 for segs; accumulated.
cudaError_t launch_histogram(const uint64_t *keys, const uint32_t *segs,
                             uint64_t n, unsigned long long *hist,
                             int num_sms, cudaStream_t s);

// Exclusive scans of npass histograms into bucket_base, and
// flags->active[p] = (no single digit holds all n elements).
cudaError_t launch_plan(const unsigned long long *hist, int npass, uint64_t n,
                        unsigned long long *bucket_base, DevFlags *flags,
                        cudaStream_t s);

// vals[i] = i | flag_bit(i) << 31 (or perm output), used when no pass runs.
cudaError_t launch_identity(const uint32_t *flag_bits, uint64_t n,
                            void *out, OutMode mode, cudaStream_t s);

// Batched sorts: segs[i] = instance of string i (seg_offsets holds the
// num_segs + 1 string-index boundaries), vals[i] = local index of i
// (| flag_bit(i) << 31 when flag_bits is given), and the instance-id digit
// histograms (hist rows kKeyPasses..kHistPasses-1, accumulated).
cudaError_t launch_seg_fill(const uint64_t *seg_offsets, uint64_t num_segs,
                            uint64_t n, const uint32_t *flag_bits,
                            uint32_t *segs, uint32_t *vals,
                            unsigned long long *hist, DevFlags *flags,
                            int num_sms, cudaStream_t s);

// flags->error |= kErrOffsets unless seg_offsets[0] == 0, seg_offsets is
// non-decreasing, seg_offsets[num_segs] == n and no instance holds more than
// 2^31 - 1 strings (local indices are 31-bit).
cudaError_t launch_validate_segments(const uint64_t *seg_offsets, uint64_t num_segs,
                                     uint64_t n, DevFlags *flags, cudaStream_t s);

// Instance boundaries used by the fix-up kernels of a batched sort: a run at
// permutation position p belongs to instance s with seg_offsets[s] <= p <
// seg_offsets[s+1], and its entries are local indices of that instance.
struct Instances {
    const uint64_t *seg_offsets;  // NULL for a single sort
    uint64_t num_segs;
    // The call's device error word (nullable).  Once an earlier kernel has
    // set it (a wait that gave up leaves positions unwritten) the fix-up
    // kernels do nothing: they would read string indices from those
    // positions.
    const unsigned int *stop = nullptr;
};

__device__ __forceinline__ bool stopped(const Instances &in) {
    return in.stop != nullptr && *reinterpret_cast<const volatile unsigned int *>(in.stop) != 0u;
}

__device__ __forceinline__ uint64_t instance_base(const Instances &in, uint64_t pos) {
    if (in.seg_offsets == nullptr) return 0;
    uint64_t lo = 0, hi = in.num_segs;  // seg_offsets[lo] <= pos < seg_offsets[hi]
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (in.seg_offsets[mid] <= pos) lo = mid; else hi = mid;
    }
    return in.seg_offsets[lo];
}

// ---- fixup.cu ------------------------------------------------------------
enum QueueId { kQSmall = 0, kQMedium = 1, kQLargeA = 2, kQLargeB = 3, kQOverflow = 4, kQMixed = 5, kQOverflow2 = 6 };
constexpr uint32_t kSmallMax = 32;     // warp per run
constexpr uint32_t kMediumMax = 2048;  // block per run

// Tie-detection modes: where the "needs work" flag of an element lives and
// what is written to the permutation.
enum TieMode {
    kTieKeyFlag = 0,   // flag = key bit 0 (ASCII7 sort key); perm already written
    kTieValFlag = 1,   // flag = payload bit 31; perm[j] = payload & kIdxMask
    kTieRefine = 2,    // flag = window tag "continues"; perm[pos(j)] = payload
    kTiePacked = 3     // keys are (code << pack_bits) | index; flag = bits[index], looked up
                       // only where the code's last char is not padding; perm[j] = index
};

struct TieArgs {
    const uint64_t *keys;
    const uint32_t *segs;           // refinement run ids, or instance ids (batched); NULL otherwise
    const uint32_t *vals;
    const uint32_t *bits;           // kTiePacked: not-exact bit of string i (bit i of word i/32)
    int pack_bits;                  // kTiePacked: index bits below the code
    uint64_t last_char_mask;        // kTiePacked: the code's last char (0: shorter string, exact)
    uint64_t n;
    int prefix_len;                 // bytes covered by the husky code
    void *perm;                     // output permutation
    int perm_u64;
    uint64_t perm_n;                // length of perm (every run must fit)
    const RunEntry *runs;           // refinement: runs being refined
    const unsigned long long *run_base;  // refinement: compacted starts
    RunEntry *q_small, *q_medium, *q_large;
    uint64_t cap_small, cap_medium, cap_large;
    int q_large_id;                 // which DevFlags::qcount slot q_large uses
    uint64_t *lookback;             // sort_tiles(n) words
    uint32_t epoch;                 // look-back epoch (1..63)
    unsigned int *tile_counter;     // zeroed
    DevFlags *flags;
};

// Equal-key runs of a sorted sequence that still need work, pushed to the
// size-class queues; writes the permutation as the mode says.
cudaError_t launch_tie_detect(const TieArgs &a, TieMode mode, cudaStream_t s);

// dirty (nullable): flags whose dirty_lo / dirty_hi widen over the positions
// a launch rewrites (the small and medium kernels alike).
cudaError_t launch_small_runs(const uint8_t *bytes, const uint64_t *offsets,
                              void *perm, int perm_u64, const RunEntry *q,
                              const unsigned long long *qcount, uint64_t first, uint64_t cap,
                              uint64_t perm_n, Instances inst, int prefix_len,
                              int num_sms, cudaStream_t s, DevFlags *dirty = nullptr);

// Large runs that are not all copies of one string, copied from q to q_out
// (count in *qcount_out, which the caller zeroes).  diff (cap entries) and
// base (cap + 1) are scratch; done2 points at two zeroed counters.
cudaError_t launch_distinct_large(const uint8_t *bytes, const uint64_t *offsets, const void *perm, int perm_u64,
                                  const RunEntry *q, const unsigned long long *qcount, uint64_t cap,
                                  uint64_t perm_n, Instances inst, int prefix_len, uint32_t *diff,
                                  unsigned long long *base, RunEntry *q_out, unsigned long long *qcount_out,
                                  uint64_t cap_out, DevFlags *flags, unsigned int *done2, int num_sms,
                                  cudaStream_t s);
// Runs of q[0 .. min(*qcount, cap)) (CTA-sized) whose members are all copies
// of one string get length 0, which launch_medium_runs skips.
cudaError_t launch_copies_filter(const uint8_t *bytes, const uint64_t *offsets, const void *perm, int perm_u64,
                                 RunEntry *q, const unsigned long long *qcount, uint64_t cap, uint64_t perm_n,
                                 Instances inst, int prefix_len, int num_sms, cudaStream_t s);

cudaError_t launch_medium_runs(const uint8_t *bytes, const uint64_t *offsets,
                               void *perm, int perm_u64, const RunEntry *q,
                               const unsigned long long *qcount, uint64_t first, uint64_t cap,
                               uint64_t perm_n, Instances inst, int prefix_len,
                               int num_sms, cudaStream_t s, DevFlags *dirty = nullptr);

// Large-run refinement helpers.
cudaError_t launch_run_scan(const RunEntry *runs, uint64_t count,
                            unsigned long long *run_base, cudaStream_t s);

cudaError_t launch_refine_keys(const uint8_t *bytes, const uint64_t *offsets,
                               const void *perm, int perm_u64,
                               const RunEntry *runs, uint64_t count,
                               const unsigned long long *run_base,
                               uint64_t total, Instances inst, int prefix_len,
                               uint64_t *keys, uint32_t *segs, uint32_t *vals,
                               DevFlags *flags, cudaStream_t s);

cudaError_t launch_push_constant_runs(const RunEntry *runs, uint64_t count,
                                      const unsigned long long *run_base,
                                      const uint64_t *keys, int prefix_len,
                                      RunEntry *q_small, RunEntry *q_medium,
                                      RunEntry *q_large, uint64_t cap_small,
                                      uint64_t cap_medium, uint64_t cap_large,
                                      int q_large_id, uint64_t perm_n,
                                      DevFlags *flags, cudaStream_t s);

// ---- rmi.cu (learned bucketing) --------------------------------------------
constexpr int kRmiHidden = 32;
constexpr int kRmiParams = 32 + 32 + 32 * 32 + 32 + 32 + 1;  // W1 b1 W2 b2 w3 b3
constexpr int kRmiLeaves = 4096;
constexpr int kRmiTrain = 2048;       // training-point capacity (hs_rmi_grad)
constexpr int kRmiTrainPoints = 512;  // points the learned path trains on
constexpr int kRmiSteps = 8;          // projected gradient steps after the quantile init
constexpr float kRmiLr = 0.02f;
constexpr int kRmiFeatureBits = 24;
constexpr uint64_t kRmiStride = 100;  // one sample per 100 keys (a 1% sample)
constexpr uint64_t kRmiSeed = 0x5DEECE66Dull;
constexpr int kBucketCap = 4096;      // largest bucket sorted inside one CTA
constexpr int kRmiAccelBits = 12;     // leaf index over the top 12 feature bits

// Model state (device, in the workspace).  thresh[l-1] = least feature X
// routed to leaf >= l (l = 1..L-1); thresh[L-1] = 2^24.
struct RmiModel {
    float p[kRmiParams];
    float pad0[3];
    uint32_t thresh[kRmiLeaves];
    uint32_t leaf_start[kRmiLeaves + 4];
    float slope[kRmiLeaves], icept[kRmiLeaves], lo[kRmiLeaves], hi[kRmiLeaves];
    // leaf l evaluates its line on (key - kbase[l]) * kscale[l]
    unsigned long long kbase[kRmiLeaves];
    float kscale[kRmiLeaves];
    unsigned long long kmin;
    int shift;
    int pad1;
    float loss0, loss1;  // training loss before / after the gradient steps
    // For the bucket kernels: leaf l's parameters in one 32-byte record, and
    // accel[s] = the leaf of feature s << (24 - kRmiAccelBits) (s up to
    // 2^kRmiAccelBits inclusive), so the leaf of feature X lies in
    // [accel[X >> 12], accel[(X >> 12) + 1]].
    struct alignas(32) LeafPk {
        unsigned long long kbase;
        float kscale, slope, icept, lo, hi, pad;
    } leafpk[kRmiLeaves];
    uint16_t accel[(1 << kRmiAccelBits) + 8];
};

cudaError_t launch_rmi_sample(const uint64_t *keys, uint64_t n, uint64_t seed,
                              uint64_t *out, uint32_t m, cudaStream_t s);
cudaError_t launch_sample_indices(uint64_t n, uint64_t seed, uint64_t *out,
                                  uint32_t m, cudaStream_t s);
// Features of the sorted sample and training (quantile init + steps).
cudaError_t launch_rmi_train(const uint64_t *sorted_sample, uint32_t m,
                             RmiModel *model, uint64_t kmin, int shift,
                             uint32_t *Xi, float *xf, float *tf, int steps,
                             float lr, cudaStream_t s);
// Leaf table (bisection of the root) made non-decreasing.
cudaError_t launch_rmi_table(RmiModel *model, cudaStream_t s);
// Leaf ranges of the sorted sample, leaf bases, leaf-relative sample
// inputs (written over xf), least-squares leaves.
cudaError_t launch_rmi_leaves(const uint64_t *sorted_sample, const uint32_t *Xi,
                              float *xf, const float *tf, uint32_t m,
                              RmiModel *model, cudaStream_t s);
// Oversize buckets (from the bucket sort's queue): copy payload to perm and
// flag buckets whose keys are not all equal (mixed[r] = 1, zeroed by caller).
// keys_out (nullable): also write key & kmask there.
cudaError_t launch_big_buckets(const RunEntry *big, uint64_t count,
                               const unsigned long long *base, uint64_t total,
                               const uint64_t *keys, const uint32_t *vals,
                               void *perm, int perm_u64, uint32_t *mixed,
                               uint64_t *keys_out, uint64_t kmask,
                               cudaStream_t s);
// Push the mixed ones to q_mixed (DevFlags::qcount[kQMixed]).
cudaError_t launch_collect_mixed(const RunEntry *big, uint64_t count,
                                 const uint32_t *mixed, RunEntry *q_mixed,
                                 uint64_t cap, DevFlags *flags, cudaStream_t s);
cudaError_t launch_rmi_grad(const float *params, const float *x, const float *t,
                            int T, float *grad, float *loss, cudaStream_t s);
cudaError_t launch_leaf_fit(const float *x, const float *t,
                            const uint32_t *leaf_start, uint32_t m, int leaves,
                            float *slope, float *icept, float *lo, float *hi,
                            cudaStream_t s);
cudaError_t launch_rmi_bucket(const uint64_t *keys, uint64_t n,
                              const RmiModel *model, int bits, int linear,
                              uint32_t *buckets, uint32_t *vals,
                              unsigned long long *hist, int num_sms,
                              cudaStream_t s);
cudaError_t launch_bucket_bounds(const uint32_t *bk, uint64_t n,
                                 unsigned long long *first,
                                 unsigned long long *last, int num_sms,
                                 cudaStream_t s);
cudaError_t launch_bucket_sort(const unsigned long long *first,
                               const unsigned long long *last,
                               uint64_t num_buckets, uint64_t *keys,
                               const uint32_t *vals, void *perm, int perm_u64,
                               RunEntry *overflow, uint64_t cap_overflow,
                               DevFlags *flags, int num_sms, cudaStream_t s);
cudaError_t launch_overflow_gather(const RunEntry *runs, uint64_t count,
                                   const unsigned long long *run_base,
                                   uint64_t total, const uint64_t *keys,
                                   const uint32_t *vals, uint64_t kmask,
                                   uint64_t *ck, uint32_t *cs, uint32_t *cv,
                                   cudaStream_t s);
// Composite keys: keys[i] |= bucket(keys[i]) << kb (the trained model's
// bucket of `bits` bits, kb + bits <= 64, every key below 2^kb), with the
// bucket ids' 9-bit digit histograms accumulated into hist rows
// 0..ceil(bits/9)-1.
cudaError_t launch_rmi_compose(uint64_t *keys, uint64_t n, const RmiModel *model,
                               int bits, int kb, unsigned long long *hist,
                               int num_sms, cudaStream_t s);
// Size-class run queues the fix-up reads (DevFlags::qcount[kQSmall],
// [kQMedium], [kQLargeA]).
struct RunQueues {
    RunEntry *small, *medium, *large;
    uint64_t cap_small, cap_medium, cap_large;
    uint64_t perm_n;
};
// Widest key (bits below the bucket id) the in-bucket sorts take.
constexpr int kTsMaxKeyBits = 50;
// In-bucket sorts of composite keys grouped by bucket (key bits below kb,
// kb <= kTsMaxKeyBits): writes the payload in key order to perm; with ties
// set, queues every run of equal keys whose bit 0 (not exact) is set; buckets
// longer than one window are queued in overflow (DevFlags::qcount[kQOverflow])
// and left to the caller.
struct TileSortArgs {
    const uint64_t *keys_in;
    const uint32_t *vals_in;
    void *perm;
    uint64_t n;
    int kb;
    int ties;
    unsigned int *range_counter;  // zeroed
    RunEntry *overflow;
    uint64_t cap_overflow;
    RunQueues q;
    DevFlags *flags;
};
cudaError_t launch_bucket_tile_sort(const TileSortArgs &a, int perm_u64,
                                    int num_sms, cudaStream_t s);
// The queued buckets, each sorted whole in a window of 12288 (as above);
// longer ones go to rest (DevFlags::qcount[kQOverflow2]).
struct RunSortArgs {
    const uint64_t *keys_in;
    const uint32_t *vals_in;
    void *perm;
    int kb;
    int ties;
    const RunEntry *runs;
    uint64_t count;
    RunEntry *rest;
    uint64_t cap_rest;
    RunQueues q;
    DevFlags *flags;
};
cudaError_t launch_bucket_run_sort(const RunSortArgs &a, int perm_u64,
                                   int num_sms, cudaStream_t s);
// Tie runs inside the runs of `runs` (sorted keys, bit 0 = not exact).
cudaError_t launch_oversize_ties(const RunEntry *runs, uint64_t count,
                                 const uint64_t *keys, const RunQueues &q,
                                 DevFlags *flags, int num_sms, cudaStream_t s);
cudaError_t launch_overflow_scatter(const RunEntry *runs,
                                    const unsigned long long *run_base,
                                    uint64_t total, const uint64_t *ck,
                                    const uint32_t *cs, const uint32_t *cv,
                                    uint64_t *keys, void *perm, int perm_u64,
                                    cudaStream_t s);

}  // namespace hs
