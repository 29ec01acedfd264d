// C ABI entry points and host-side orchestration of the three steps.
//
// hs_argsort(PLAIN):
//   encode (codes, non-exact bits, digit histograms)   -- Step 1
//   plan   (bucket bases, which digits vary)            -- host reads flags
//   onesweep passes over the varying digits             -- Step 2
//   if not perfect: tie detection, then large-run
//   refinement rounds, then CTA and warp run sorts       -- Step 3
// The caller owns every device buffer; scratch is carved from d_ws.
#include <atomic>
#include <cstdio>
#include <cstring>

#include <cuda.h>
#include <mutex>
#include <string>
#include <vector>

#include "husky.h"
#include "husky_learned.h"
#include "hs_internal.h"
#include "hs_bignum.h"
#include "hs_fixup.h"

namespace hs {
namespace {

thread_local std::string g_last_error;

hs_status fail(hs_status st, const char *msg) {
    g_last_error = msg;
    return st;
}

hs_status fail_cuda(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return HS_ERR_CUDA;
}

// ---- per-kernel timing (hs_stats_*) ----------------------------------------

enum KernelKind {
    kKEncode, kKPlan, kKOnesweep, kKIdentity, kKTieDetect, kKSmallRuns, kKMediumRuns,
    kKRunScan, kKRefineKeys, kKPushConstant, kKHistogram, kKSegFill, kKRmiSample, kKRmiFit, kKRmiBucket,
    kKBucketBounds, kKBucketSort, kKOverflow, kKRmiTable, kKRmiLeaves, kKDistinctLarge, kKCollectMixed, kKValidate, kKAlphabet, kKPairs, kKSorted, kKCopies,
    kKBucketRun, kKBigBuckets, kKOversizeTies, kKDecimal, kKWindowDense, kKNumKinds
};
const char *const kKindNames[kKNumKinds] = {
    "encode", "plan", "onesweep", "identity", "tie_detect", "small_runs", "medium_runs",
    "run_scan", "refine_keys", "push_constant_runs", "histogram", "seg_fill", "rmi_sample", "rmi_train",
    "rmi_bucket", "bucket_bounds", "bucket_sort", "overflow", "rmi_table", "rmi_leaves", "distinct_large", "collect_mixed", "validate", "alphabet", "pairs_ordered", "sorted_test", "copies_filter",
    "bucket_run_sort", "big_buckets", "oversize_ties", "decimal_encode", "window_dense"};

struct StatsTable {
    std::mutex mu;
    bool enabled = false;
    uint64_t launches[kKNumKinds] = {};
    double ms[kKNumKinds] = {};
    double bytes[kKNumKinds] = {};
    std::vector<cudaEvent_t> pool;   // reused events
};
StatsTable g_stats;

struct PendingStat {
    int kind;
    double bytes;
    cudaEvent_t a, b;
    int launches;
};

cudaEvent_t pooled_event() {
    std::lock_guard<std::mutex> g(g_stats.mu);
    if (!g_stats.pool.empty()) {
        cudaEvent_t e = g_stats.pool.back();
        g_stats.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

constexpr size_t kAlign = 256;
constexpr int kNumCounters = 4096;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Carver {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    }
};

// Workspace layout of hs_argsort / hs_encode for n strings.
struct Layout {
    size_t flags, hist, bucket, counters;  // control block (zeroed per call)
    size_t control_end;
    size_t codes_a, codes_b, vals_a, vals_b, segs_a, segs_b, bits;
    size_t lb;
    size_t q_small, q_medium, q_large_a, q_large_b, run_base, large_diff;
    uint64_t cap_small, cap_medium, cap_large;
    // learned mode only
    bool learned;
    int bucket_bits;
    uint32_t m;  // sample size
    size_t model, samp_keys_a, samp_keys_b, samp_vals_a, samp_vals_b, samp_X, samp_x, samp_t;
    size_t b_first, b_last, q_over, q_over2, over_base, keys_extra, big_mixed, q_mixed, mixed_base;
    uint64_t cap_over;
    // hs_argsort_host only: device copies of the host inputs and output
    size_t dev_bytes, dev_offsets, dev_perm;
    size_t total;
};

constexpr uint64_t kLearnedMinN = 1ull << 16;  // below this the plain path is used

// Bucket-id bits: about n/256 buckets, rounded to whole 9-bit partition
// passes -- 18 bits (two passes) up to ~2.7e8 keys, 23-24 bits (three)
// above.  g_forced_bucket_bits (hs_learned_force_bucket_bits) overrides the
// choice so that the wider branches can be checked at small n.
std::atomic<int> g_forced_bucket_bits{0};

int learned_bits(uint64_t n) {
    const int forced = g_forced_bucket_bits.load();
    if (forced > 0) return forced;
    int want = 1;
    while (want < 30 && (1ull << want) * 256 < n) ++want;
    return want <= 20 ? 18 : (want + 2 < 24 ? want + 2 : 24);
}

Layout make_layout(uint64_t n, bool learned = false) {
    Layout L{};
    Carver c;
    L.flags = c.take(sizeof(DevFlags));
    L.hist = c.take(kHistPasses * kBins * sizeof(unsigned long long));
    L.bucket = c.take(kHistPasses * kBins * sizeof(unsigned long long));
    L.counters = c.take(kNumCounters * sizeof(unsigned int));
    L.control_end = c.off;
    L.codes_a = c.take(n * 8);
    L.codes_b = c.take(n * 8);
    L.vals_a = c.take(n * 4);
    L.vals_b = c.take(n * 4);
    L.segs_a = c.take(n * 4);
    L.segs_b = c.take(n * 4);
    L.bits = c.take(((n + 31) / 32) * 4);
    L.lb = c.take(sort_tiles(n) * kBins * 8);
    L.cap_small = n / 2 + 1;
    L.cap_medium = n / (kSmallMax + 1) + 1;
    L.cap_large = n / (kMediumMax + 1) + 1;
    L.q_small = c.take(L.cap_small * sizeof(RunEntry));
    L.q_medium = c.take(L.cap_medium * sizeof(RunEntry));
    L.q_large_a = c.take(L.cap_large * sizeof(RunEntry));
    L.q_large_b = c.take(L.cap_large * sizeof(RunEntry));
    L.run_base = c.take((L.cap_large + 1) * 8);
    L.large_diff = c.take(L.cap_large * 4);
    L.learned = learned && n >= kLearnedMinN;
    if (L.learned) {
        L.bucket_bits = learned_bits(n);
        L.m = (uint32_t)(n / kRmiStride);
        L.model = c.take(sizeof(RmiModel));
        L.samp_keys_a = c.take((size_t)L.m * 8);
        L.samp_keys_b = c.take((size_t)L.m * 8);
        L.samp_vals_a = c.take((size_t)L.m * 4);
        L.samp_vals_b = c.take((size_t)L.m * 4);
        L.samp_X = c.take((size_t)L.m * 4);
        L.samp_x = c.take((size_t)L.m * 4);
        L.samp_t = c.take((size_t)L.m * 4);
        const uint64_t B = 1ull << L.bucket_bits;
        L.b_first = c.take(B * 8);
        L.b_last = c.take(B * 8);
        L.cap_over = n / (kBucketCap + 1) + 1;
        L.q_over = c.take(L.cap_over * sizeof(RunEntry));
        L.q_over2 = c.take(L.cap_over * sizeof(RunEntry));
        L.over_base = c.take((L.cap_over + 1) * 8);
        L.big_mixed = c.take(L.cap_over * 4);
        L.q_mixed = c.take(L.cap_over * sizeof(RunEntry));
        L.mixed_base = c.take((L.cap_over + 1) * 8);
        L.keys_extra = c.take(n * 8);
    }
    L.total = c.off;
    return L;
}

// hs_argsort_host: the hs_argsort layout followed by device copies of the
// bytes (plus 16 bytes of slack), the offsets and the permutation.
Layout make_host_layout(uint64_t n, uint64_t total_bytes, bool learned, size_t isz) {
    Layout L = make_layout(n, learned);
    Carver c{L.total};
    L.dev_bytes = c.take(total_bytes + 16);
    L.dev_offsets = c.take((n + 1) * 8);
    L.dev_perm = c.take(n * isz);
    L.total = c.off;
    return L;
}

// Library-owned copy stream per device (non-blocking, created once) and a
// pool of timing-free events for the chunk hand-offs.
constexpr int kMaxDevices = 64;
std::mutex g_copy_mu;
cudaStream_t g_copy_stream[kMaxDevices] = {};
std::vector<cudaEvent_t> g_sync_events;

cudaError_t copy_stream(cudaStream_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_copy_mu);
    if (!g_copy_stream[dev]) {
        e = cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    *out = g_copy_stream[dev];
    return cudaSuccess;
}

cudaError_t sync_event(cudaEvent_t *out) {
    std::lock_guard<std::mutex> g(g_copy_mu);
    if (!g_sync_events.empty()) {
        *out = g_sync_events.back();
        g_sync_events.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreateWithFlags(out, cudaEventDisableTiming);
}

void release_sync_events(std::vector<cudaEvent_t> &v) {
    std::lock_guard<std::mutex> g(g_copy_mu);
    for (cudaEvent_t e : v) g_sync_events.push_back(e);
    v.clear();
}

// Pinned host copies of the control block: a device-to-host copy into
// pageable memory is staged and blocking, into pinned memory it is one DMA.
std::vector<DevFlags *> g_pinned_flags;

cudaError_t pinned_flags(DevFlags **out) {
    std::lock_guard<std::mutex> g(g_copy_mu);
    if (!g_pinned_flags.empty()) {
        *out = g_pinned_flags.back();
        g_pinned_flags.pop_back();
        return cudaSuccess;
    }
    return cudaHostAlloc(reinterpret_cast<void **>(out), sizeof(DevFlags), cudaHostAllocDefault);
}

void release_pinned_flags(DevFlags *p) {
    if (p == nullptr) return;
    std::lock_guard<std::mutex> g(g_copy_mu);
    g_pinned_flags.push_back(p);
}

// Tile-shape tuner.  The first sort of a layout (packed words, or key and
// payload pairs) in a size class (floor(log2 n), n >= 2^20) runs its second
// and third radix passes with the two shapes of kOnesweepShapes, timed with
// events, and keeps the faster for that class.  The shape only changes how a
// pass is tiled, never its result.
struct ShapeTuner {
    std::mutex mu;
    bool enabled = true;
    int choice[2][64] = {};  // keys per thread, 0 = not tuned yet
};
ShapeTuner g_tuner;

int size_class(uint64_t n) {
    int c = 0;
    while (c < 63 && (2ull << c) <= n) ++c;
    return c;
}

// Host source of hs_argsort_host: where the inputs are and where their
// device copies go.
struct HostSrc {
    const uint8_t *h_bytes;
    const uint64_t *h_offsets;
    uint8_t *d_bytes;
    uint64_t *d_offsets;
    uint64_t total;
};

// Strings per transfer chunk: whole 1024-string encoder tiles, about eight
// chunks per call, at least 2^18 strings so small calls stay one chunk.
uint64_t host_chunk(uint64_t n) {
    uint64_t c = n / 8;
    if (c < (1ull << 18)) c = 1ull << 18;
    return (c + 1023) / 1024 * 1024;
}

int num_sms_cached() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    return sms;
}

// Per-call execution context.
struct Ctx {
    cudaStream_t s;
    char *ws;
    Layout L;
    int sms;
    DevFlags *d_flags;
    unsigned int *d_counters;
    int next_counter = 0;
    DevFlags h;  // last host copy of the flags
    const HostSrc *host = nullptr;    // hs_argsort_host: inputs still on the host
    int alpha_k = 9;                  // chars the alphabet coder covered (its prefix length)
    int alpha_w = 0;                  // its bits per char
    bool idx_packed = false;          // the encoder packed each string's index below its code
    int idx_bits = 0;                 // ... in this many bits
    // hs_argsort_host: the permutation's copy to h_out may start once it is
    // written (packed words: by the last radix pass, or by tie detection
    // when no pass ran); early_copy marks its end, and the fix-up's
    // rewrites (DevFlags::dirty_lo / dirty_hi, or all of it after refinement
    // rounds) are copied again afterwards.
    void *h_out = nullptr;
    size_t h_out_isz = 0;
    cudaEvent_t early_copy = nullptr;
    bool dirty_all = false;
    std::vector<cudaEvent_t> events;  // chunk hand-off events in use

    template <typename T> T *at(size_t off) { return reinterpret_cast<T *>(ws + off); }

    cudaError_t counter(unsigned int **out) {
        if (next_counter >= kNumCounters) {
            cudaError_t e = cudaMemsetAsync(d_counters, 0, kNumCounters * sizeof(unsigned int), s);
            if (e != cudaSuccess) return e;
            next_counter = 0;
        }
        *out = d_counters + next_counter++;
        return cudaSuccess;
    }

    // Look-back epochs: each look-back launch gets its own; the array is
    // cleared when they run out.
    uint32_t epoch = kLbEpochs;  // forces a clear before the first use
    uint64_t lb_words = 0;       // words to clear (sort_tiles(n) * kBins)
    cudaError_t next_epoch(uint32_t *out) {
        if (epoch >= kLbEpochs) {
            cudaError_t e = cudaMemsetAsync(ws + L.lb, 0, lb_words * 8, s);
            if (e != cudaSuccess) return e;
            epoch = 0;
        }
        *out = ++epoch;
        return cudaSuccess;
    }

    DevFlags *h_pinned = nullptr;  // staging for h
    bool pinned_ok = true;         // may take a pinned buffer (not on the allocation-free path)
    cudaError_t read_flags() {
        cudaError_t e = cudaSuccess;
        if (!pinned_ok) {
            e = cudaMemcpyAsync(&h, d_flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return e;
            return cudaStreamSynchronize(s);
        }
        if (!h_pinned && (e = pinned_flags(&h_pinned)) != cudaSuccess) {
            h_pinned = nullptr;
            return e;
        }
        e = cudaMemcpyAsync(h_pinned, d_flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        h = *h_pinned;
        return cudaSuccess;
    }

    // Launch through f(), bracketed by events when timing is enabled.
    std::vector<PendingStat> pending;
    bool timing = false;
    template <typename F> cudaError_t timed(int kind, double bytes, F f, int launches = 1) {
        if (!timing) return f();
        PendingStat p{kind, bytes, pooled_event(), pooled_event(), launches};
        cudaEventRecord(p.a, s);
        cudaError_t e = f();
        cudaEventRecord(p.b, s);
        pending.push_back(p);
        return e;
    }

    // Called once the stream is idle: fold event times into the table.
    void flush_stats() {
        if (pending.empty()) return;
        cudaStreamSynchronize(s);
        std::lock_guard<std::mutex> g(g_stats.mu);
        for (auto &p : pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess && g_stats.enabled) {
                g_stats.launches[p.kind] += p.launches;
                g_stats.ms[p.kind] += ms;
                g_stats.bytes[p.kind] += p.bytes;
            }
            g_stats.pool.push_back(p.a);
            g_stats.pool.push_back(p.b);
        }
        pending.clear();
    }
    ~Ctx() {
        flush_stats();
        if (early_copy) cudaEventSynchronize(early_copy);  // the caller's buffer is not written after return
        if (!events.empty() || h_pinned) cudaStreamSynchronize(s);  // no copy or wait still uses them
        if (!events.empty()) release_sync_events(events);
        release_pinned_flags(h_pinned);
    }
};

#define HS_TRY(expr, where)                               \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return fail_cuda(_e, where); \
    } while (0)

hs_status device_error_status(const DevFlags &h) {
    if (h.error & kErrOffsets) return fail(HS_ERR_INVALID_ARG, "offsets are decreasing or exceed offsets[n]");
    if (h.error & kErrTimeout) return fail(HS_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (h.error) return fail(HS_ERR_INTERNAL, "device-side consistency check failed");
    return HS_OK;
}

// Step 1 into ctx buffers; resolves HS_CODER_AUTO.  On return ctx.h holds the
// flags and *used the coder actually used.
hs_status run_encode(Ctx &c, const uint8_t *bytes, const uint64_t *offsets, uint64_t n, int coder,
                     uint64_t *codes, uint32_t *bits, bool hist, bool sort_key, int *used, int max_key_bits = 64,
                     EncPack pack = EncPack{}) {
    int u = coder == HS_CODER_BYTE8 ? HS_CODER_BYTE8 : (coder == HS_CODER_ASCII7 ? HS_CODER_ASCII7 : HS_CODER_ALPHA);
    c.idx_packed = false;
    c.idx_bits = pack.idx_bits;
    for (int attempt = 0; attempt < 3; ++attempt) {
        HS_TRY(cudaMemsetAsync(c.ws, 0, c.L.control_end, c.s), "memset control");
        HS_TRY(cudaMemsetAsync(&c.d_flags->kmin, 0xFF, sizeof(unsigned long long), c.s), "memset kmin");
        c.next_counter = 0;
        const double enc_bytes = 8.0 * (n + 1) + 8.0 * n + (bits ? n / 8.0 : 0.0);
        const bool kflag = sort_key && u != HS_CODER_BYTE8;
        // a packed index leaves the not-exact bit out of the key: the bitmap holds it
        uint32_t *ebits = (kflag && !(u == HS_CODER_ALPHA && pack.idx_bits > 0)) ? nullptr : bits;
        unsigned long long *ehist = hist ? c.at<unsigned long long>(c.L.hist) : nullptr;
        const bool from_host = c.host && attempt == 0;
        // AUTO takes the byte-range coder only where it saves a radix pass
        // over ASCII7 (w <= 5: a range of at most 31 values); asked for, up
        // to 6 bits.
        const int max_w = coder == HS_CODER_ALPHA ? 6 : 5;
        bool spec = false;
        if (from_host) {
            // Inputs still on the host: copy them chunk by chunk on the
            // library's copy stream; each chunk is encoded once it is in.
            // The byte-range coder scans each chunk's range as well and
            // encodes with the first chunk's range, checked against the
            // whole range after the last chunk (re-encoded on a mismatch).
            const HostSrc &h = *c.host;
            cudaStream_t cs = nullptr;
            HS_TRY(copy_stream(&cs), "copy stream");
            cudaEvent_t start = nullptr;
            HS_TRY(sync_event(&start), "event");
            c.events.push_back(start);
            HS_TRY(cudaEventRecord(start, c.s), "record start");  // after the caller's earlier work
            HS_TRY(cudaStreamWaitEvent(cs, start, 0), "copy waits");
            const uint64_t chunk = host_chunk(n);
            for (uint64_t s0 = 0; s0 < n; s0 += chunk) {
                const uint64_t s1 = umin64(n, s0 + chunk);
                HS_TRY(cudaMemcpyAsync(h.d_offsets + s0, h.h_offsets + s0, (s1 - s0 + 1) * 8,
                                       cudaMemcpyHostToDevice, cs),
                       "copy offsets");
                const uint64_t b0 = h.h_offsets[s0], b1 = h.h_offsets[s1];
                if (b1 > b0)
                    HS_TRY(cudaMemcpyAsync(h.d_bytes + b0, h.h_bytes + b0, b1 - b0, cudaMemcpyHostToDevice, cs),
                           "copy bytes");
                cudaEvent_t ev = nullptr;
                HS_TRY(sync_event(&ev), "event");
                c.events.push_back(ev);
                HS_TRY(cudaEventRecord(ev, cs), "record chunk");
                HS_TRY(cudaStreamWaitEvent(c.s, ev, 0), "encode waits");
                const uint64_t m = s1 - s0;
                if (u == HS_CODER_ALPHA) {
                    HS_TRY(c.timed(kKAlphabet, (double)(b1 - b0), [&] {
                               return launch_alphabet(h.d_bytes, h.d_offsets + s0, m, (1 << max_w) - 1, c.d_flags,
                                                      c.sms, c.s);
                           }),
                           "alphabet chunk");
                    if (s0 == 0)
                        HS_TRY(cudaMemcpyAsync(&c.d_flags->alpha_spec_lo_inv, &c.d_flags->alpha_lo_inv,
                                               2 * sizeof(unsigned int), cudaMemcpyDeviceToDevice, c.s),
                               "speculative range");
                    spec = true;
                }
                EncPack pk = pack;
                pk.spec_range = spec ? 1 : 0;
                pk.idx_base = s0;
                HS_TRY(c.timed(kKEncode, enc_bytes * ((double)m / (double)n), [&] {
                           return launch_encode(u, kflag, h.d_bytes, h.d_offsets + s0, m, codes + s0,
                                                ebits ? ebits + s0 / 32 : nullptr, ehist, c.d_flags, c.sms, c.s,
                                                max_w, max_key_bits, pk);
                       }),
                       "encode chunk");
            }
        } else if (u == HS_CODER_ALPHA) {
            HS_TRY(c.timed(kKAlphabet, 0.0, [&] {
                       return launch_alphabet(bytes, offsets, n, (1 << max_w) - 1, c.d_flags, c.sms, c.s);
                   }),
                   "alphabet");
        }
        if (!from_host)
            HS_TRY(c.timed(kKEncode, enc_bytes, [&] {
                       return launch_encode(u, kflag, bytes, offsets, n, codes, ebits, ehist, c.d_flags, c.sms, c.s,
                                            max_w, max_key_bits, pack);
                   }),
                   "encode");
        if (pack.sorted_check)
            HS_TRY(c.timed(kKSorted, 0.0, [&] {
                       return launch_sorted_test(codes, ebits, n, kflag, pack.idx_bits, pack.pairs, pack.pairs_cap,
                                                 c.d_flags, c.sms, c.s);
                   }),
                   "sorted test");
        if (hist)
            HS_TRY(c.timed(kKPlan, 8.0 * kBins * 16, [&] {
                       return launch_plan(c.at<unsigned long long>(c.L.hist), kKeyPasses, n,
                                          c.at<unsigned long long>(c.L.bucket), c.d_flags, c.s);
                   }),
                   "plan");
        HS_TRY(c.read_flags(), "encode sync");
        hs_status st = device_error_status(c.h);
        if (st != HS_OK) return st;
        if (spec && (c.h.alpha_spec_lo_inv != c.h.alpha_lo_inv || c.h.alpha_spec_hi != c.h.alpha_hi))
            continue;  // a later chunk widened the byte range: encode again from the device copies
        if (u == HS_CODER_ALPHA) {
            // the encoder's own test: w within max_w and the 8-char key within max_key_bits
            if ((int)c.h.alpha_w <= max_w && 8 * (int)c.h.alpha_w + 1 <= max_key_bits) {
                c.alpha_k = (int)c.h.alpha_k;
                c.alpha_w = (int)c.h.alpha_w;
                c.idx_packed = c.h.idx_packed != 0;
                break;
            }
            if (coder == HS_CODER_ALPHA)
                return fail(HS_ERR_CODER_DOMAIN, "byte-range coder: the strings span more than 63 byte values");
            u = HS_CODER_ASCII7;  // the kernel encoded as ASCII7
        }
        if (u == HS_CODER_ASCII7 && c.h.domain) {
            if (coder == HS_CODER_ASCII7)
                return fail(HS_ERR_CODER_DOMAIN, "ASCII7 coder: a byte >= 0x80 among the first 9 bytes");
            u = HS_CODER_BYTE8;  // the byte coder is order preserving on all bytes
            continue;
        }
        break;
    }
    *used = u;
    return HS_OK;
}

// Bytes of each string the sort key's code covers (the fix-up starts after).
int coded_prefix(const Ctx &c, int used) {
    return used == HS_CODER_BYTE8 ? 8 : (used == HS_CODER_ALPHA ? c.alpha_k : 9);
}

// Runs the active radix passes over (keys, vals) pairs.  Returns the index
// (0 or 1) of the buffers holding the result when the result is not written
// to `final_out`.
struct SortBufs {
    uint64_t *keys[2];
    uint32_t *vals[2];
    uint32_t *segs[2];
};

hs_status run_passes(Ctx &c, SortBufs &b, int *cur, uint64_t n, const int *passes, int npasses,
                     bool segmented, const uint32_t *flag_bits, bool synth_first, void *final_out,
                     OutMode final_mode, bool keep_keys, int pack_bits = 0, int digit_base = 0) {
    uint64_t *lb = c.at<uint64_t>(c.L.lb);
    const int layout = segmented ? -1 : (pack_bits > 0 ? 0 : 1);
    const int cls = size_class(n);
    int items = 0;
    bool tune = false;
    if (layout >= 0 && n >= (1ull << 20)) {
        std::lock_guard<std::mutex> g(g_tuner.mu);
        items = g_tuner.choice[layout][cls];
        tune = g_tuner.enabled && items == 0 && npasses >= 4;
    }
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (tune)
        for (auto &e : tev)
            if ((e = pooled_event()) == nullptr) tune = false;
    if (pack_bits > 0) {  // (key << pack_bits) | index words: nothing else moves
        if (segmented || (!keep_keys && final_out == nullptr)) return fail(HS_ERR_INTERNAL, "packed passes");
        synth_first = false;
        flag_bits = nullptr;
    }
    for (int i = 0; i < npasses; ++i) {
        const int p = passes[i];
        const bool first = i == 0, last = i == npasses - 1;
        const bool digit_seg = p >= kKeyPasses;
        OnesweepArgs a{};
        a.keys_in = b.keys[*cur];
        a.keys_out = (last && !keep_keys) ? nullptr : b.keys[*cur ^ 1];
        a.segs_in = segmented ? b.segs[*cur] : nullptr;
        a.segs_out = segmented ? b.segs[*cur ^ 1] : nullptr;
        a.vals_in = ((first && synth_first) || pack_bits > 0) ? nullptr : b.vals[*cur];
        const bool to_final = last && final_out != nullptr;
        a.vals_out = to_final ? final_out : (pack_bits > 0 ? nullptr : b.vals[*cur ^ 1]);
        a.flag_bits = flag_bits;
        a.n = n;
        a.pack_bits = pack_bits;
        a.shift = digit_shift(p) + pack_bits + digit_base;
        a.mask = digit_mask(p);
        a.bucket_base = c.at<unsigned long long>(c.L.bucket) + (size_t)p * kBins;
        a.lookback = lb;
        HS_TRY(c.next_epoch(&a.epoch), "epoch");
        HS_TRY(c.counter(&a.tile_counter), "counter");
        a.flags = c.d_flags;
        const OutMode om = to_final ? final_mode : kOutVals;
        double ob = 8.0 * n;                                   // keys read
        if (pack_bits > 0) {
            ob += a.keys_out ? 8.0 * n : 0.0;                  // words written
            ob += om == kOutPerm32 ? 4.0 * n : (om == kOutPerm64 ? 8.0 * n : 0.0);  // indices written
        } else {
            ob += (first && synth_first) ? (flag_bits ? n / 8.0 : 0.0) : 4.0 * n;  // vals read
            ob += a.keys_out ? 8.0 * n : 0.0;                  // keys written
            ob += om == kOutPerm64 ? 8.0 * n : 4.0 * n;        // vals written
            ob += segmented ? 8.0 * n : 0.0;                   // segs read + written
        }
        const bool timed_shape = tune && (i == 1 || i == 2);
        const int shape = timed_shape ? kOnesweepShapes[i - 1] : items;
        if (timed_shape) HS_TRY(cudaEventRecord(tev[2 * (i - 1)], c.s), "tuner event");
        HS_TRY(c.timed(kKOnesweep, ob, [&] {
                   return launch_onesweep(a, segmented, digit_seg, first && synth_first, om, c.s, shape);
               }),
               "onesweep");
        if (timed_shape) HS_TRY(cudaEventRecord(tev[2 * (i - 1) + 1], c.s), "tuner event");
        if (tune && i == 2) {
            float ms0 = 0.f, ms1 = 0.f;
            HS_TRY(cudaEventSynchronize(tev[3]), "tuner sync");
            HS_TRY(cudaEventElapsedTime(&ms0, tev[0], tev[1]), "tuner time");
            HS_TRY(cudaEventElapsedTime(&ms1, tev[2], tev[3]), "tuner time");
            items = ms1 < ms0 ? kOnesweepShapes[1] : kOnesweepShapes[0];
            std::lock_guard<std::mutex> g(g_tuner.mu);
            g_tuner.choice[layout][cls] = items;
        }
        *cur ^= 1;
    }
    if (tune) {
        std::lock_guard<std::mutex> g(g_stats.mu);
        for (auto e : tev) g_stats.pool.push_back(e);
    }
    return HS_OK;
}

struct Input {
    const uint8_t *bytes;
    const uint64_t *offsets;
    uint64_t n;
    int prefix_len;
    void *perm;
    int perm_u64;
};

// Step 3 on the sorted keys.  When it returns HS_OK with *synced set, every
// launch has finished and c.h holds the final flags.
// perm_written: packed words whose last radix pass wrote the permutation
// beside them (tie detection then only finds the runs).
hs_status run_fixup(Ctx &c, const Input &in, SortBufs &b, int cur, TieMode mode, const Instances &inst0,
                    bool *synced = nullptr, bool instance_in_key = false, bool perm_written = false,
                    bool runs_queued = false) {
    if (synced) *synced = false;
    Instances inst = inst0;
    inst.stop = &c.d_flags->error;  // after a give-up the fix-up kernels do nothing
    const uint64_t n = in.n;
    RunEntry *q_small = c.at<RunEntry>(c.L.q_small);
    RunEntry *q_medium = c.at<RunEntry>(c.L.q_medium);
    RunEntry *q_large[2] = {c.at<RunEntry>(c.L.q_large_a), c.at<RunEntry>(c.L.q_large_b)};
    unsigned long long *run_base = c.at<unsigned long long>(c.L.run_base);
    uint64_t *lb = c.at<uint64_t>(c.L.lb);

    TieArgs t{};
    t.keys = b.keys[cur];
    // batched: runs end at instance boundaries (implied by the key when the
    // instance id is packed into it)
    t.segs = (inst.seg_offsets && !instance_in_key) ? b.segs[cur] : nullptr;
    t.vals = b.vals[cur];
    if (mode == kTiePacked) {
        t.bits = c.at<uint32_t>(c.L.bits);
        t.pack_bits = c.idx_bits;
        t.last_char_mask = (1ull << c.alpha_w) - 1;
    }
    t.n = n;
    t.prefix_len = in.prefix_len;
    t.perm = (mode == kTiePacked && perm_written) ? nullptr : in.perm;
    t.perm_u64 = in.perm_u64;
    t.perm_n = n;
    t.q_small = q_small;
    t.q_medium = q_medium;
    t.q_large = q_large[0];
    t.cap_small = c.L.cap_small;
    t.cap_medium = c.L.cap_medium;
    t.cap_large = c.L.cap_large;
    t.q_large_id = kQLargeA;
    t.lookback = lb;
    t.flags = c.d_flags;
    HS_TRY(c.next_epoch(&t.epoch), "epoch");
    HS_TRY(c.counter(&t.tile_counter), "counter");
    // Packed words: the permutation is final but for the fix-up's runs once
    // written (by the last radix pass, or by tie detection), and those runs
    // are few (the byte-range code covers 8 chars).  With (key, payload)
    // pairs the fix-up's rewrites spread over the whole permutation
    // (measured: the copy then goes twice), so the copy waits for the end.
    const bool early = c.h_out != nullptr && !inst.seg_offsets && mode == kTiePacked;
    cudaEvent_t perm_done = nullptr;
    if (early) {
        HS_TRY(cudaMemsetAsync(&c.d_flags->dirty_lo, 0xFF, sizeof(unsigned long long), c.s), "memset dirty");
        HS_TRY(sync_event(&perm_done), "event");
        c.events.push_back(perm_done);
        if (perm_written) HS_TRY(cudaEventRecord(perm_done, c.s), "record last pass");
    }
    const double tie_bytes = mode == kTieKeyFlag ? 8.0 * n
                             : mode == kTiePacked ? 8.0 * n + (t.perm ? (in.perm_u64 ? 8.0 : 4.0) * n : 0.0)
                                                  : 8.0 * n + 4.0 * n + (in.perm_u64 ? 8.0 : 4.0) * n;
    if (!runs_queued)  // else the caller's kernels queued the runs already
        HS_TRY(c.timed(kKTieDetect, tie_bytes, [&] { return launch_tie_detect(t, mode, c.s); }), "tie detect");
    if (early && !perm_written) HS_TRY(cudaEventRecord(perm_done, c.s), "record tie detect");
    // Runs of copies of one string are final already; only the others go on
    // to refinement (queue B).
    HS_TRY(cudaMemsetAsync(&c.d_flags->qcount[kQLargeB], 0, sizeof(unsigned long long), c.s), "memset q");
    unsigned int *done2 = nullptr, *done2b = nullptr;
    HS_TRY(c.counter(&done2), "counter");
    HS_TRY(c.counter(&done2b), "counter");
    if (done2b != done2 + 1) {  // the pair wrapped past the end of the counter block: take a fresh pair
        HS_TRY(c.counter(&done2), "counter");
        HS_TRY(c.counter(&done2b), "counter");
    }
    HS_TRY(c.timed(kKDistinctLarge, 0.0, [&] {
               return launch_distinct_large(in.bytes, in.offsets, in.perm, in.perm_u64, q_large[0],
                                            &c.d_flags->qcount[kQLargeA], c.L.cap_large, n, inst, in.prefix_len,
                                            c.at<uint32_t>(c.L.large_diff), run_base, q_large[1],
                                            &c.d_flags->qcount[kQLargeB], c.L.cap_large, c.d_flags, done2, c.sms,
                                            c.s);
           }, 2),
           "distinct large runs");
    // The warp- and CTA-sized runs tie detection queued need nothing from
    // the host: their kernels read the queue counts on the device.  Launch
    // them now; refinement (if any) appends more, handled after it.
    const double isz = in.perm_u64 ? 8.0 : 4.0;
    auto launch_med_small = [&](uint64_t med0, uint64_t small0, bool known) -> hs_status {
        const uint64_t med = c.h.qcount[kQMedium], sm = c.h.qcount[kQSmall];
        if (!known)
            HS_TRY(c.timed(kKCopies, 0.0, [&] {
                       return launch_copies_filter(in.bytes, in.offsets, in.perm, in.perm_u64, q_medium,
                                                   &c.d_flags->qcount[kQMedium], c.L.cap_medium, n, inst,
                                                   in.prefix_len, c.sms, c.s);
                   }),
                   "copies filter");
        if (!known || med > med0)
            HS_TRY(c.timed(kKMediumRuns, known ? (double)(med - med0) * 16.0 * (2 * isz + 16.0) : 0.0, [&] {
                       return launch_medium_runs(in.bytes, in.offsets, in.perm, in.perm_u64, q_medium,
                                                 &c.d_flags->qcount[kQMedium], med0, c.L.cap_medium, n, inst,
                                                 in.prefix_len, c.sms, c.s, early ? c.d_flags : nullptr);
                   }),
                   "medium runs");
        if (!known || sm > small0)
            HS_TRY(c.timed(kKSmallRuns, known ? (double)(sm - small0) * (16.0 + 2.0 * (2 * isz + 16.0)) : 0.0, [&] {
                       return launch_small_runs(in.bytes, in.offsets, in.perm, in.perm_u64, q_small,
                                                &c.d_flags->qcount[kQSmall], small0, c.L.cap_small, n, inst,
                                                in.prefix_len, c.sms, c.s, early ? c.d_flags : nullptr);
                   }, 2),
                   "small runs");
        return HS_OK;
    };
    hs_status st = launch_med_small(0, 0, false);
    if (st != HS_OK) return st;
    if (early) {
        // the permutation leaves while the fix-up runs (issued after the
        // fix-up launches: a copy to pageable memory blocks the host)
        cudaStream_t cs = nullptr;
        HS_TRY(copy_stream(&cs), "copy stream");
        HS_TRY(cudaStreamWaitEvent(cs, perm_done, 0), "copy waits");
        HS_TRY(cudaMemcpyAsync(c.h_out, in.perm, n * c.h_out_isz, cudaMemcpyDeviceToHost, cs), "early copy");
        HS_TRY(sync_event(&c.early_copy), "event");
        c.events.push_back(c.early_copy);
        HS_TRY(cudaEventRecord(c.early_copy, cs), "record early copy");
    }
    HS_TRY(c.read_flags(), "tie sync");
    st = device_error_status(c.h);
    if (st != HS_OK) return st;
    const uint64_t med0 = c.h.qcount[kQMedium], small0 = c.h.qcount[kQSmall];
    if (c.h.qcount[kQLargeB] == 0) {
        if (synced) *synced = true;
        return HS_OK;
    }

    // Large runs: refine 7 bytes per round until every run is constant-and-
    // resolved or has been split into CTA / warp sized pieces.
    int li = 1;
    uint64_t large = c.h.qcount[kQLargeB];
    int rounds = 0;
    if (early) c.dirty_all = true;  // refinement rewrites positions all over
    while (large > 0) {
        if (++rounds > (1 << 26)) return fail(HS_ERR_INTERNAL, "refinement did not terminate");
        if (large > c.L.cap_large) return fail(HS_ERR_INTERNAL, "large-run queue overflow");
        const int next = li ^ 1;
        const int next_id = next ? kQLargeB : kQLargeA;
        const int cur_id = li ? kQLargeB : kQLargeA;
        HS_TRY(cudaMemsetAsync(&c.d_flags->qcount[next_id], 0, sizeof(unsigned long long), c.s), "memset q");
        HS_TRY(cudaMemsetAsync(&c.d_flags->nonconst, 0, sizeof(unsigned int), c.s), "memset nonconst");
        HS_TRY(c.timed(kKRunScan, 24.0 * large, [&] { return launch_run_scan(q_large[li], large, run_base, c.s); }),
               "run scan");
        unsigned long long total = 0;
        HS_TRY(cudaMemcpyAsync(&total, run_base + large, 8, cudaMemcpyDeviceToHost, c.s), "read total");
        HS_TRY(cudaStreamSynchronize(c.s), "scan sync");
        if (total > n) return fail(HS_ERR_INTERNAL, "large runs overlap (run descriptors inconsistent)");
        SortBufs r = b;
        int rc = 0;
        // Every run of a round is at the same depth: runs enter at depth 0
        // and each round moves the ones it keeps one window on.  When the
        // runs hold most of the strings, one pass in string order writes
        // every string's window key to a dense array (r.keys[1], free until
        // the sort below), and the refinement gathers one word a member
        // from it instead of the member's offsets and bytes.
        const uint32_t depth = (uint32_t)(rounds - 1);
        uint64_t *win = nullptr;
        if (total * 5 >= n * 2) {
            win = r.keys[1];
            HS_TRY(c.timed(kKWindowDense, 32.0 * n, [&] {
                       return launch_window_dense(in.bytes, in.offsets, n, in.prefix_len, depth, win, c.sms, c.s);
                   }),
                   "window keys");
        }
        HS_TRY(c.timed(kKRefineKeys, (win ? 28.0 : 32.0) * total, [&] {
                   return launch_refine_keys_win(in.bytes, in.offsets, in.perm, in.perm_u64, q_large[li], large,
                                                 run_base, total, inst, in.prefix_len, win, depth, r.keys[0],
                                                 r.segs[0], r.vals[0], c.d_flags, c.s);
               }),
               "refine keys");
        HS_TRY(c.read_flags(), "refine sync");
        st = device_error_status(c.h);
        if (st != HS_OK) return st;
        if (!c.h.nonconst) {
            HS_TRY(c.timed(kKPushConstant, 32.0 * large, [&] {
                       return launch_push_constant_runs(q_large[li], large, run_base, r.keys[0], in.prefix_len,
                                                        q_small, q_medium, q_large[next], c.L.cap_small,
                                                        c.L.cap_medium, c.L.cap_large, next_id, n, c.d_flags,
                                                        c.s);
                   }),
                   "push constant runs");
        } else {
            unsigned long long *hist = c.at<unsigned long long>(c.L.hist);
            HS_TRY(cudaMemsetAsync(hist, 0, kHistPasses * kBins * 8, c.s), "memset hist");
            HS_TRY(c.timed(kKHistogram, 12.0 * total,
                           [&] { return launch_histogram(r.keys[0], r.segs[0], total, hist, c.sms, c.s); }),
                   "histogram");
            HS_TRY(c.timed(kKPlan, 8.0 * kBins * 24, [&] {
                       return launch_plan(hist, kHistPasses, total, c.at<unsigned long long>(c.L.bucket), c.d_flags,
                                          c.s);
                   }),
                   "plan");
            HS_TRY(c.read_flags(), "plan sync");
            int passes[kHistPasses], np = 0;
            for (int p = 0; p < kHistPasses; ++p)
                if (c.h.active[p]) passes[np++] = p;
            st = run_passes(c, r, &rc, total, passes, np, true, nullptr, false, nullptr, kOutVals, true);
            if (st != HS_OK) return st;
            TieArgs u = t;
            u.keys = r.keys[rc];
            u.segs = r.segs[rc];
            u.vals = r.vals[rc];
            u.n = total;
            u.runs = q_large[li];
            u.run_base = run_base;
            u.q_large = q_large[next];
            u.q_large_id = next_id;
            HS_TRY(c.next_epoch(&u.epoch), "epoch");
            HS_TRY(c.counter(&u.tile_counter), "counter");
            HS_TRY(c.timed(kKTieDetect, 20.0 * total, [&] { return launch_tie_detect(u, kTieRefine, c.s); }),
                   "refine tie detect");
        }
        (void)cur_id;
        HS_TRY(c.read_flags(), "round sync");
        st = device_error_status(c.h);
        if (st != HS_OK) return st;
        large = c.h.qcount[next_id];
        li = next;
    }

    return launch_med_small(med0, small0, true);
}

hs_status argsort_plain(Ctx &c, const Input &in0, int coder) {
    Input in = in0;
    const uint64_t n = in.n;
    SortBufs b{{c.at<uint64_t>(c.L.codes_a), c.at<uint64_t>(c.L.codes_b)},
               {c.at<uint32_t>(c.L.vals_a), c.at<uint32_t>(c.L.vals_b)},
               {c.at<uint32_t>(c.L.segs_a), c.at<uint32_t>(c.L.segs_b)}};
    uint32_t *bits = c.at<uint32_t>(c.L.bits);
    c.lb_words = sort_tiles(n) * kBins;
    int used = 0;
    // Up to 2^idx_bits strings: the byte-range coder's 8w-bit codes and
    // their indices share one word when they fit, so a pass moves 8 bytes
    // a string instead of 12 and the not-exact bit rides in the bitmap.
    int idx_bits = 0;
    while (idx_bits < 63 && (1ull << idx_bits) < n) ++idx_bits;
    EncPack pk{};
    pk.idx_bits = n >= 2 ? idx_bits : 0;
    // Already-sorted inputs (the partially-sorted case the paper's appendix
    // discusses, at its extreme): the encoder compares neighbours' order
    // keys on the way, so an ordered input costs the encode, a comparison
    // of the pairs it could not decide and the identity permutation.
    pk.sorted_check = n >= 2 ? 1 : 0;
    pk.pairs = b.keys[1];
    pk.pairs_cap = n;
    hs_status st = run_encode(c, in.bytes, in.offsets, n, coder, b.keys[0], bits, true, true, &used, 64, pk);
    if (st != HS_OK) return st;
    in.prefix_len = coded_prefix(c, used);
    const OutMode pmode = in.perm_u64 ? kOutPerm64 : kOutPerm32;
    if (pk.sorted_check && !c.h.descent && c.h.pairs <= pk.pairs_cap) {
        if (c.h.pairs > 0) {
            const uint64_t pairs = c.h.pairs;
            HS_TRY(c.timed(kKPairs, 24.0 * pairs, [&] {
                       return launch_pairs_ordered(in.bytes, in.offsets, b.keys[1], pairs, c.d_flags, c.sms, c.s);
                   }),
                   "pairs ordered");
            HS_TRY(c.read_flags(), "pairs sync");
            st = device_error_status(c.h);
            if (st != HS_OK) return st;
        }
        if (!c.h.descent) {
            HS_TRY(c.timed(kKIdentity, 4.0 * n, [&] { return launch_identity(nullptr, n, in.perm, pmode, c.s); }),
                   "identity");
            HS_TRY(c.read_flags(), "final sync");
            return device_error_status(c.h);
        }
    }
    if (used == HS_CODER_ALPHA && c.idx_packed) {
        const bool perfect = c.h.nonexact == 0;
        int passes[kKeyPasses], np = 0;
        for (int p = 0; p < kKeyPasses; ++p)
            if (c.h.active[p]) passes[np++] = p;
        int cur = 0;
        if (np == 0) {
            if (perfect)
                HS_TRY(c.timed(kKIdentity, 4.0 * n, [&] { return launch_identity(nullptr, n, in.perm, pmode, c.s); }),
                       "identity");
        }
        // Host output: the last pass writes the permutation beside the
        // words, so its copy leaves before tie detection.
        const bool perm_written = np > 0 && (perfect || c.h_out != nullptr);
        if (np > 0) {
            st = run_passes(c, b, &cur, n, passes, np, false, nullptr, false, perm_written ? in.perm : nullptr, pmode,
                            !perfect, c.idx_bits);
            if (st != HS_OK) return st;
        }
        bool synced = false;
        if (!perfect) {
            st = run_fixup(c, in, b, cur, kTiePacked, Instances{nullptr, 0}, &synced, false, perm_written);
            if (st != HS_OK) return st;
        }
        if (!synced) HS_TRY(c.read_flags(), "final sync");
        return device_error_status(c.h);
    }
    // ASCII7: the sort key carries the not-exact bit, so the permutation is
    // final after the last pass and runs needing work are read off the keys.
    // BYTE8: the bit rides in the payload and tie detection writes the
    // permutation.
    const bool key_flag = used != HS_CODER_BYTE8;
    const bool perfect = c.h.nonexact == 0;
    int passes[kKeyPasses], np = 0;
    for (int p = 0; p < kKeyPasses; ++p)
        if (c.h.active[p]) passes[np++] = p;
    const OutMode perm_mode = in.perm_u64 ? kOutPerm64 : kOutPerm32;
    const bool final_is_perm = key_flag || perfect;
    const uint32_t *flag_bits = key_flag ? nullptr : bits;
    int cur = 0;
    if (np == 0) {
        HS_TRY(c.timed(kKIdentity, n / 8.0 + 4.0 * n, [&] {
                   return launch_identity(flag_bits, n, final_is_perm ? in.perm : (void *)b.vals[0],
                                          final_is_perm ? perm_mode : kOutVals, c.s);
               }),
               "identity");
    } else {
        st = run_passes(c, b, &cur, n, passes, np, false, flag_bits, true, final_is_perm ? in.perm : nullptr,
                        perm_mode, !perfect);
        if (st != HS_OK) return st;
    }
    bool synced = false;
    if (!perfect) {
        st = run_fixup(c, in, b, cur, key_flag ? kTieKeyFlag : kTieValFlag, Instances{nullptr, 0}, &synced);
        if (st != HS_OK) return st;
    }
    if (!synced) HS_TRY(c.read_flags(), "final sync");
    return device_error_status(c.h);
}

// Learned: a monotone model maps sort keys to buckets; a stable partition by
// bucket (two or three 9-bit passes) plus a sort inside each bucket gives the
// sort by key.  Oversize buckets are copied when constant, sorted by a
// segmented radix sort otherwise.  Returns HS_OK with *fallback = true when
// the plain path must be used instead (BYTE8 coder).
struct LearnedProfile {
    uint64_t *keys;      // out: sort keys
    uint32_t *buckets;   // out: bucket per string
    int linear;          // untrained linear map instead of the model
    double info[4];
};

// Runs of the learned path too long for an in-CTA sort, `big` of them in
// q_over (positions in keys/vals): the payload goes
// to the permutation as it stands (and key & kmask to big_keys_out when
// given); the runs holding more than one key are gathered into ov.*[0],
// sorted by a segmented radix sort over (run, key & kmask) and scattered
// back: keys to sorted_keys_out, payload to the permutation.  The ov.*[1]
// buffers are the passes' other side and may alias keys/vals (read only by
// the gather).
hs_status sort_oversize(Ctx &c, const Input &in, const RunEntry *q_over, uint64_t big, const uint64_t *keys,
                        const uint32_t *vals, uint64_t kmask, uint64_t *big_keys_out, uint64_t *sorted_keys_out,
                        SortBufs ov) {
    const uint64_t n = in.n;
    const Layout &L = c.L;
    if (big == 0) return HS_OK;
    if (big > L.cap_over) return fail(HS_ERR_INTERNAL, "overflow queue full");
    RunEntry *q_mixed = c.at<RunEntry>(L.q_mixed);
    unsigned long long *hist = c.at<unsigned long long>(L.hist);
    unsigned long long *bucket = c.at<unsigned long long>(L.bucket);
    unsigned long long *bb = c.at<unsigned long long>(L.over_base);
    HS_TRY(c.timed(kKRunScan, 0.0, [&] { return launch_run_scan(q_over, big, bb, c.s); }), "big scan");
    unsigned long long big_total = 0;
    HS_TRY(cudaMemcpyAsync(&big_total, bb + big, 8, cudaMemcpyDeviceToHost, c.s), "big total");
    HS_TRY(cudaStreamSynchronize(c.s), "big sync");
    if (big_total > n) return fail(HS_ERR_INTERNAL, "oversize buckets overlap");
    uint32_t *mixed = c.at<uint32_t>(L.big_mixed);
    HS_TRY(cudaMemsetAsync(mixed, 0, big * 4, c.s), "memset mixed");
    HS_TRY(c.timed(kKBigBuckets, 20.0 * big_total, [&] {
               return launch_big_buckets(q_over, big, bb, big_total, keys, vals, in.perm, in.perm_u64, mixed,
                                         big_keys_out, kmask, c.s);
           }),
           "big buckets");
    HS_TRY(c.timed(kKCollectMixed, 0.0, [&] { return launch_collect_mixed(q_over, big, mixed, q_mixed, L.cap_over, c.d_flags, c.s); }), "collect mixed");
    HS_TRY(c.read_flags(), "mixed sync");
    hs_status st = device_error_status(c.h);
    if (st != HS_OK) return st;
    const uint64_t over = c.h.qcount[kQMixed];
    if (over == 0) return HS_OK;
    unsigned long long *ob = c.at<unsigned long long>(L.mixed_base);
    HS_TRY(c.timed(kKRunScan, 0.0, [&] { return launch_run_scan(q_mixed, over, ob, c.s); }), "overflow scan");
    unsigned long long total = 0;
    HS_TRY(cudaMemcpyAsync(&total, ob + over, 8, cudaMemcpyDeviceToHost, c.s), "overflow total");
    HS_TRY(cudaStreamSynchronize(c.s), "overflow sync");
    if (total > n) return fail(HS_ERR_INTERNAL, "overflow buckets overlap");
    HS_TRY(c.timed(kKOverflow, 28.0 * total, [&] {
               return launch_overflow_gather(q_mixed, over, ob, total, keys, vals, kmask, ov.keys[0], ov.segs[0],
                                             ov.vals[0], c.s);
           }),
           "overflow gather");
    HS_TRY(cudaMemsetAsync(hist, 0, kHistPasses * kBins * 8, c.s), "memset hist");
    HS_TRY(c.timed(kKHistogram, 0.0, [&] { return launch_histogram(ov.keys[0], ov.segs[0], total, hist, c.sms, c.s); }), "overflow histogram");
    HS_TRY(c.timed(kKPlan, 0.0, [&] { return launch_plan(hist, kHistPasses, total, bucket, c.d_flags, c.s); }), "overflow plan");
    HS_TRY(c.read_flags(), "overflow plan sync");
    int passes[kHistPasses], np = 0;
    for (int p = 0; p < kHistPasses; ++p)
        if (c.h.active[p]) passes[np++] = p;
    int oc = 0;
    st = run_passes(c, ov, &oc, total, passes, np, true, nullptr, false, nullptr, kOutVals, true);
    if (st != HS_OK) return st;
    HS_TRY(c.timed(kKOverflow, 28.0 * total, [&] {
               return launch_overflow_scatter(q_mixed, ob, total, ov.keys[oc], ov.segs[oc], ov.vals[oc],
                                              sorted_keys_out, in.perm, in.perm_u64, c.s);
           }),
           "overflow scatter");
    return HS_OK;
}

// Bucket-id bits when the id sits above the key: an average bucket of at
// most about 2048 keys (windows of the in-bucket sort hold 6144), and at
// most 18 bits, two 9-bit partition passes.
int composite_bits(uint64_t n) {
    int bits = 1;
    while (bits < 18 && (n >> bits) > 2048) ++bits;
    return bits;
}

// Learned partition with the bucket id above a sort key of kb bits: compose,
// one to three partition passes on the bucket digits (one word per element),
// in-bucket sorts over windows of whole buckets (which write the
// permutation and the sorted keys), the overflow sort for longer buckets,
// then tie detection and the fix-up on the sorted keys.
hs_status learned_composite(Ctx &c, const Input &in, SortBufs &b, RmiModel *model, int kb, int bits, bool perfect) {
    const uint64_t n = in.n;
    const Layout &L = c.L;
    unsigned long long *hist = c.at<unsigned long long>(L.hist);
    unsigned long long *bucket = c.at<unsigned long long>(L.bucket);
    HS_TRY(cudaMemsetAsync(hist, 0, kHistPasses * kBins * 8, c.s), "memset hist");
    HS_TRY(c.timed(kKRmiBucket, 16.0 * n, [&] {
               return launch_rmi_compose(b.keys[0], n, model, bits, kb, hist, c.sms, c.s);
           }),
           "rmi compose");
    const int nparts = (bits + kRadixBits - 1) / kRadixBits;
    HS_TRY(c.timed(kKPlan, 0.0, [&] { return launch_plan(hist, nparts, n, bucket, c.d_flags, c.s); }), "bucket plan");
    HS_TRY(c.read_flags(), "bucket plan sync");
    hs_status st = device_error_status(c.h);
    if (st != HS_OK) return st;
    int passes[3], np = 0;
    for (int p = 0; p < nparts; ++p)
        if (c.h.active[p]) passes[np++] = p;
    if (np == 0) passes[np++] = 0;  // one pass still writes the payload (the string index)
    int cur = 0;
    st = run_passes(c, b, &cur, n, passes, np, false, nullptr, true, nullptr, kOutVals, true, 0, kb);
    if (st != HS_OK) return st;
    unsigned int *ranges = nullptr;
    HS_TRY(c.counter(&ranges), "counter");
    const RunQueues rq{c.at<RunEntry>(L.q_small), c.at<RunEntry>(L.q_medium), c.at<RunEntry>(L.q_large_a),
                       L.cap_small, L.cap_medium, L.cap_large, n};
    const TileSortArgs t{b.keys[cur], b.vals[cur], in.perm, n, kb, perfect ? 0 : 1, ranges,
                         c.at<RunEntry>(L.q_over), L.cap_over, rq, c.d_flags};
    HS_TRY(c.timed(kKBucketSort, 12.0 * n + (in.perm_u64 ? 8.0 : 4.0) * n, [&] {
               return launch_bucket_tile_sort(t, in.perm_u64, c.sms, c.s);
           }),
           "bucket tile sort");
    HS_TRY(c.read_flags(), "tile sort sync");
    st = device_error_status(c.h);
    if (st != HS_OK) return st;
    // Buckets longer than a window: sorted whole in windows twice as long
    // where they fit; the rest by the overflow sort, whose sorted keys (bucket
    // bits cleared) land in the other key buffer, then their tie runs.
    const uint64_t big = c.h.qcount[kQOverflow];
    uint64_t big2 = 0;
    RunEntry *q_rest = c.at<RunEntry>(L.q_over2);
    if (big > 0) {
        if (big > L.cap_over) return fail(HS_ERR_INTERNAL, "overflow queue full");
        const RunSortArgs ra{b.keys[cur], b.vals[cur], in.perm, kb, perfect ? 0 : 1, c.at<RunEntry>(L.q_over), big,
                             q_rest, L.cap_over, rq, c.d_flags};
        HS_TRY(c.timed(kKBucketRun, 0.0, [&] { return launch_bucket_run_sort(ra, in.perm_u64, c.sms, c.s); }),
               "bucket run sort");
        HS_TRY(c.read_flags(), "run sort sync");
        st = device_error_status(c.h);
        if (st != HS_OK) return st;
        big2 = c.h.qcount[kQOverflow2];
    }
    const uint64_t kmask = (1ull << kb) - 1;
    st = sort_oversize(c, in, q_rest, big2, b.keys[cur], b.vals[cur], kmask, b.keys[cur ^ 1], b.keys[cur ^ 1],
                       SortBufs{{c.at<uint64_t>(L.keys_extra), b.keys[cur]},
                                {b.vals[cur ^ 1], b.vals[cur]},
                                {b.segs[0], b.segs[1]}});
    if (st != HS_OK) return st;
    if (!perfect && big2 > 0)
        HS_TRY(c.timed(kKOversizeTies, 0.0, [&] {
                   return launch_oversize_ties(q_rest, big2, b.keys[cur ^ 1], rq, c.d_flags, c.sms, c.s);
               }),
               "oversize ties");
    if (!perfect) {
        st = run_fixup(c, in, b, cur ^ 1, kTieKeyFlag, Instances{nullptr, 0}, nullptr, false, false, true);
        if (st != HS_OK) return st;
    }
    HS_TRY(c.read_flags(), "final sync");
    return device_error_status(c.h);
}

hs_status argsort_learned(Ctx &c, const Input &in0, int coder, bool *fallback, LearnedProfile *prof = nullptr) {
    Input in = in0;
    const uint64_t n = in.n;
    const Layout &L = c.L;
    SortBufs b{{c.at<uint64_t>(L.codes_a), c.at<uint64_t>(L.codes_b)},
               {c.at<uint32_t>(L.vals_a), c.at<uint32_t>(L.vals_b)},
               {c.at<uint32_t>(L.segs_a), c.at<uint32_t>(L.segs_b)}};
    c.lb_words = sort_tiles(n) * kBins;
    int used = 0;
    hs_status st = run_encode(c, in.bytes, in.offsets, n, coder, b.keys[0], c.at<uint32_t>(L.bits), false, true,
                              &used);
    if (st != HS_OK) return st;
    if (used == HS_CODER_BYTE8) {
        *fallback = true;
        return HS_OK;
    }
    in.prefix_len = coded_prefix(c, used);
    const bool perfect = c.h.nonexact == 0;
    const uint64_t kmin = c.h.kmin, kmax = c.h.kmax;
    int shift = 0;
    while (((kmax - kmin) >> shift) >= (1ull << kRmiFeatureBits)) ++shift;
    RmiModel *model = c.at<RmiModel>(L.model);
    unsigned long long *hist = c.at<unsigned long long>(L.hist);
    unsigned long long *bucket = c.at<unsigned long long>(L.bucket);

    // 1% sample, sorted with the plain radix sort
    const uint32_t m = L.m;
    SortBufs sb{{c.at<uint64_t>(L.samp_keys_a), c.at<uint64_t>(L.samp_keys_b)},
                {c.at<uint32_t>(L.samp_vals_a), c.at<uint32_t>(L.samp_vals_b)},
                {nullptr, nullptr}};
    HS_TRY(c.timed(kKRmiSample, 16.0 * m, [&] { return launch_rmi_sample(b.keys[0], n, kRmiSeed, sb.keys[0], m, c.s); }),
           "rmi sample");
    HS_TRY(cudaMemsetAsync(hist, 0, kHistPasses * kBins * 8, c.s), "memset hist");
    HS_TRY(c.timed(kKHistogram, 0.0, [&] { return launch_histogram(sb.keys[0], nullptr, m, hist, c.sms, c.s); }), "sample histogram");
    HS_TRY(c.timed(kKPlan, 0.0, [&] { return launch_plan(hist, kKeyPasses, m, bucket, c.d_flags, c.s); }), "sample plan");
    HS_TRY(c.read_flags(), "sample plan sync");
    int passes[kHistPasses], np = 0;
    for (int p = 0; p < kKeyPasses; ++p)
        if (c.h.active[p]) passes[np++] = p;
    int sc = 0;
    st = run_passes(c, sb, &sc, m, passes, np, false, nullptr, true, nullptr, kOutVals, true);
    if (st != HS_OK) return st;

    // model: quantile init, gradient steps, leaf table, leaf fits
    {
        const unsigned long long km = kmin;
        const int sh = shift;
        HS_TRY(cudaMemcpyAsync(&model->kmin, &km, sizeof(km), cudaMemcpyHostToDevice, c.s), "model kmin");
        HS_TRY(cudaMemcpyAsync(&model->shift, &sh, sizeof(sh), cudaMemcpyHostToDevice, c.s), "model shift");
    }
    HS_TRY(c.timed(kKRmiFit, 20.0 * m, [&] {
               return launch_rmi_train(sb.keys[sc], m, model, kmin, shift, c.at<uint32_t>(L.samp_X),
                                       c.at<float>(L.samp_x), c.at<float>(L.samp_t), kRmiSteps, kRmiLr, c.s);
           }, 2),
           "rmi train");
    HS_TRY(c.timed(kKRmiTable, 0.0, [&] { return launch_rmi_table(model, c.s); }, 2), "rmi table");
    HS_TRY(c.timed(kKRmiLeaves, 12.0 * m, [&] {
               return launch_rmi_leaves(sb.keys[sc], c.at<uint32_t>(L.samp_X), c.at<float>(L.samp_x),
                                        c.at<float>(L.samp_t), m, model, c.s);
           }, 4),
           "rmi leaves");

    // buckets, then the stable partition by bucket digits
    const int bits = L.bucket_bits;
    const uint64_t B = 1ull << bits;
    if (prof) {
        HS_TRY(launch_rmi_bucket(b.keys[0], n, model, bits, prof->linear, prof->buckets, nullptr, nullptr, c.sms, c.s),
               "profile buckets");
        HS_TRY(cudaMemcpyAsync(prof->keys, b.keys[0], n * 8, cudaMemcpyDeviceToDevice, c.s), "profile keys");
        float losses[2] = {0.f, 0.f};
        HS_TRY(cudaMemcpyAsync(losses, &model->loss0, sizeof(losses), cudaMemcpyDeviceToHost, c.s), "profile loss");
        HS_TRY(cudaStreamSynchronize(c.s), "profile sync");
        prof->info[0] = bits;
        prof->info[1] = m;
        prof->info[2] = losses[0];
        prof->info[3] = losses[1];
        return HS_OK;
    }
    // Byte-range keys leave room above them: the bucket id goes there and
    // each partition pass moves one word and the payload.
    if (used == HS_CODER_ALPHA) {
        const int kb = kmax ? 64 - __builtin_clzll(kmax) : 1;
        const int forced = g_forced_bucket_bits.load();
        const int cbits = forced > 0 ? forced : composite_bits(n);
        if (kb + cbits <= 64 && cbits <= 3 * kRadixBits && kb <= kTsMaxKeyBits)
            return learned_composite(c, in, b, model, kb, cbits, perfect);
    }
    HS_TRY(cudaMemsetAsync(hist, 0, kHistPasses * kBins * 8, c.s), "memset hist");
    HS_TRY(c.timed(kKRmiBucket, 16.0 * n, [&] {
               return launch_rmi_bucket(b.keys[0], n, model, bits, 0, b.segs[0], b.vals[0], hist, c.sms, c.s);
           }),
           "rmi bucket");
    HS_TRY(c.timed(kKPlan, 0.0, [&] { return launch_plan(hist, kHistPasses, n, bucket, c.d_flags, c.s); }), "bucket plan");
    HS_TRY(c.read_flags(), "bucket plan sync");
    st = device_error_status(c.h);
    if (st != HS_OK) return st;
    np = 0;
    for (int p = kKeyPasses; p < kKeyPasses + (bits + kRadixBits - 1) / kRadixBits; ++p)
        if (c.h.active[p]) passes[np++] = p;
    int cur = 0;
    st = run_passes(c, b, &cur, n, passes, np, true, nullptr, false, nullptr, kOutVals, true);
    if (st != HS_OK) return st;

    // per-bucket sorts
    unsigned long long *first = c.at<unsigned long long>(L.b_first), *last = c.at<unsigned long long>(L.b_last);
    HS_TRY(cudaMemsetAsync(first, 0xFF, B * 8, c.s), "memset bucket bounds");
    HS_TRY(c.timed(kKBucketBounds, 4.0 * n, [&] { return launch_bucket_bounds(b.segs[cur], n, first, last, c.sms, c.s); }),
           "bucket bounds");
    RunEntry *q_over = c.at<RunEntry>(L.q_over);
    HS_TRY(c.timed(kKBucketSort, 12.0 * n + (in.perm_u64 ? 16.0 : 12.0) * n, [&] {
               return launch_bucket_sort(first, last, B, b.keys[cur], b.vals[cur], in.perm, in.perm_u64, q_over,
                                         L.cap_over, c.d_flags, c.sms, c.s);
           }),
           "bucket sort");
    HS_TRY(c.read_flags(), "bucket sort sync");
    st = device_error_status(c.h);
    if (st != HS_OK) return st;
    st = sort_oversize(c, in, c.at<RunEntry>(L.q_over), c.h.qcount[kQOverflow], b.keys[cur], b.vals[cur], ~0ull,
                       nullptr, b.keys[cur],
                       SortBufs{{c.at<uint64_t>(L.keys_extra), b.keys[cur ^ 1]},
                                {b.vals[cur ^ 1], b.vals[cur]},
                                {b.segs[cur ^ 1], b.segs[cur]}});
    if (st != HS_OK) return st;
    if (!perfect) {
        st = run_fixup(c, in, b, cur, kTieKeyFlag, Instances{nullptr, 0});
        if (st != HS_OK) return st;
    }
    HS_TRY(c.read_flags(), "final sync");
    return device_error_status(c.h);
}

// Batched: one segmented sort by (instance, sort key) over all strings; the
// payload is the local index, so the last pass writes the local permutation.
hs_status argsort_batched(Ctx &c, const Input &in0, const uint64_t *seg_offsets, uint64_t num_segs, int coder) {
    Input in = in0;
    const uint64_t n = in.n;
    SortBufs b{{c.at<uint64_t>(c.L.codes_a), c.at<uint64_t>(c.L.codes_b)},
               {c.at<uint32_t>(c.L.vals_a), c.at<uint32_t>(c.L.vals_b)},
               {c.at<uint32_t>(c.L.segs_a), c.at<uint32_t>(c.L.segs_b)}};
    uint32_t *bits = c.at<uint32_t>(c.L.bits);
    c.lb_words = sort_tiles(n) * kBins;
    HS_TRY(cudaMemsetAsync(c.ws, 0, c.L.control_end, c.s), "memset control");
    HS_TRY(c.timed(kKValidate, 0.0, [&] { return launch_validate_segments(seg_offsets, num_segs, n, c.d_flags, c.s); }), "validate segments");
    HS_TRY(c.read_flags(), "validate sync");
    if (c.h.error & kErrOffsets)
        return fail(HS_ERR_INVALID_ARG,
                    "seg_offsets must start at 0, not decrease, end at n, and give no instance 2^31 or more strings");
    // With the byte-range coder the key leaves room above it for the
    // instance id: one key, no separate instance array in the radix passes.
    int seg_bits = 1;
    while (seg_bits < 63 && (1ull << seg_bits) < num_segs) ++seg_bits;
    // the instance of every 1024-string tile's first string, for the encoder
    uint32_t *tile_seg = b.segs[0];
    HS_TRY(c.timed(kKSegFill, 0.0, [&] { return launch_tile_segs(seg_offsets, num_segs, n, tile_seg, c.s); }),
           "tile instances");
    int used = 0;
    hs_status st = run_encode(c, in.bytes, in.offsets, n, coder, b.keys[0], bits, true, true, &used, 64 - seg_bits,
                              EncPack{seg_offsets, num_segs, seg_bits, b.vals[0], tile_seg});
    if (st != HS_OK) return st;
    in.prefix_len = coded_prefix(c, used);
    const bool key_flag = used != HS_CODER_BYTE8;
    const bool perfect = c.h.nonexact == 0;
    unsigned long long *hist = c.at<unsigned long long>(c.L.hist);
    const Instances inst{seg_offsets, num_segs};
    if (used == HS_CODER_ALPHA) {
        // the encoder packed the instance ids, wrote the local indices and
        // planned the passes over the packed keys
        const int key_bits = (int)(c.h.alpha_k * c.h.alpha_w) + 1;
        if (key_bits + seg_bits > 64) return fail(HS_ERR_INTERNAL, "packed batched key does not fit");
        int passes[kKeyPasses], np = 0;
        for (int p = 0; p < kKeyPasses; ++p)
            if (c.h.active[p]) passes[np++] = p;
        if (np == 0) passes[np++] = 0;  // a no-op pass still writes the permutation
        int cur = 0;
        st = run_passes(c, b, &cur, n, passes, np, false, nullptr, false, in.perm, kOutPerm32, !perfect);
        if (st != HS_OK) return st;
        bool synced = false;
        if (!perfect) {
            st = run_fixup(c, in, b, cur, kTieKeyFlag, inst, &synced, true);
            if (st != HS_OK) return st;
        }
        if (!synced) HS_TRY(c.read_flags(), "final sync");
        return device_error_status(c.h);
    }
    HS_TRY(c.timed(kKSegFill, 8.0 * n + 8.0 * n, [&] {
               return launch_seg_fill(seg_offsets, num_segs, n, key_flag ? nullptr : bits, b.segs[0], b.vals[0],
                                      hist, c.d_flags, c.sms, c.s);
           }),
           "seg fill");
    HS_TRY(c.timed(kKPlan, 0.0, [&] { return launch_plan(hist, kHistPasses, n, c.at<unsigned long long>(c.L.bucket), c.d_flags, c.s); }), "plan");
    HS_TRY(c.read_flags(), "plan sync");
    st = device_error_status(c.h);
    if (st != HS_OK) return st;
    int passes[kHistPasses], np = 0;
    for (int p = 0; p < kHistPasses; ++p)
        if (c.h.active[p]) passes[np++] = p;
    if (np == 0) passes[np++] = 0;  // a no-op pass still writes the permutation
    const bool final_is_perm = key_flag || perfect;
    int cur = 0;
    st = run_passes(c, b, &cur, n, passes, np, true, nullptr, false, final_is_perm ? in.perm : nullptr, kOutPerm32,
                    !perfect);
    if (st != HS_OK) return st;
    if (!perfect) {
        st = run_fixup(c, in, b, cur, key_flag ? kTieKeyFlag : kTieValFlag, inst);
        if (st != HS_OK) return st;
    }
    HS_TRY(c.read_flags(), "final sync");
    return device_error_status(c.h);
}

bool make_ctx(Ctx &c, void *ws, size_t ws_bytes, uint64_t n, void *stream, hs_status *st, bool learned = false,
              const Layout *layout = nullptr) {
    c.L = layout ? *layout : make_layout(n, learned);
    if (ws == nullptr || ws_bytes < c.L.total) {
        *st = fail(HS_ERR_WORKSPACE, "workspace missing or smaller than hs_workspace_size()");
        return false;
    }
    if ((reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) {
        *st = fail(HS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        return false;
    }
    c.s = static_cast<cudaStream_t>(stream);
    c.ws = static_cast<char *>(ws);
    c.sms = num_sms_cached();
    c.d_flags = c.at<DevFlags>(c.L.flags);
    c.d_counters = c.at<unsigned int>(c.L.counters);
    {
        std::lock_guard<std::mutex> g(g_stats.mu);
        c.timing = g_stats.enabled;
    }
    return true;
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" {

hs_status hs_workspace_size(uint64_t n, uint64_t total_bytes, int mode, int out_t, size_t *out) {
    (void)total_bytes;
    (void)out_t;
    g_last_error.clear();
    if (!out) return fail(HS_ERR_INVALID_ARG, "out is NULL");
    if (mode != HS_MODE_PLAIN && mode != HS_MODE_LEARNED && mode != HS_MODE_AUTO) return fail(HS_ERR_INVALID_ARG, "bad mode");
    if (mode == HS_MODE_AUTO) mode = HS_MODE_PLAIN;  // see hs_mode
    *out = make_layout(n, mode == HS_MODE_LEARNED).total;
    return HS_OK;
}

hs_status hs_encode(const uint8_t *d_bytes, const uint64_t *d_offsets, uint64_t n, int coder, uint64_t *d_codes,
                    int *h_all_exact, int *h_coder_used, void *d_ws, size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (coder < HS_CODER_AUTO || coder > HS_CODER_ALPHA) return fail(HS_ERR_INVALID_ARG, "bad coder");
    if (!d_offsets || (n > 0 && !d_codes)) return fail(HS_ERR_INVALID_ARG, "null pointer");
    Ctx c;
    hs_status st;
    if (!make_ctx(c, d_ws, ws_bytes, 0, stream, &st)) return st;
    if (n == 0) {
        if (h_all_exact) *h_all_exact = 1;
        if (h_coder_used) *h_coder_used = coder == HS_CODER_BYTE8 ? HS_CODER_BYTE8 : HS_CODER_ASCII7;
        return HS_OK;
    }
    if (!d_bytes) return fail(HS_ERR_INVALID_ARG, "null bytes");
    int used = 0;
    st = run_encode(c, d_bytes, d_offsets, n, coder, d_codes, nullptr, false, false, &used);
    if (st != HS_OK) return st;
    if (h_all_exact) *h_all_exact = c.h.nonexact ? 0 : 1;
    if (h_coder_used) *h_coder_used = used;
    return HS_OK;
}

hs_status hs_argsort(const uint8_t *d_bytes, const uint64_t *d_offsets, uint64_t n, int mode, int coder, int out_t,
                     void *d_perm, void *d_ws, size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (mode != HS_MODE_PLAIN && mode != HS_MODE_LEARNED && mode != HS_MODE_AUTO) return fail(HS_ERR_INVALID_ARG, "bad mode");
    if (mode == HS_MODE_AUTO) mode = HS_MODE_PLAIN;  // see hs_mode
    if (coder < HS_CODER_AUTO || coder > HS_CODER_ALPHA) return fail(HS_ERR_INVALID_ARG, "bad coder");
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    if (n > HS_MAX_N) return fail(HS_ERR_INVALID_ARG, "n exceeds HS_MAX_N");
    if (n == 0) return HS_OK;
    if (!d_bytes || !d_offsets || !d_perm) return fail(HS_ERR_INVALID_ARG, "null pointer");
    Ctx c;
    hs_status st;
    if (!make_ctx(c, d_ws, ws_bytes, n, stream, &st, mode == HS_MODE_LEARNED)) return st;
    Input in{d_bytes, d_offsets, n, 9, d_perm, out_t == HS_U64 ? 1 : 0};
    if (c.L.learned) {
        bool fallback = false;
        st = argsort_learned(c, in, coder, &fallback);
        if (st != HS_OK || !fallback) return st;
    }
    return argsort_plain(c, in, coder);
}

// Workspace of hs_argsort_bigint: the string sort's, then the encoded
// strings (total_bytes + 2n) and their offsets.
struct BigLayout {
    size_t sort_bytes, enc_bytes, enc_offsets, total;
    uint64_t enc_cap;
};
BigLayout bigint_layout(uint64_t n, uint64_t total_bytes) {
    auto up = [](size_t x) { return (x + kAlign - 1) / kAlign * kAlign; };
    BigLayout b{};
    b.sort_bytes = up(make_layout(n).total);
    b.enc_cap = total_bytes + 2 * n;
    b.enc_bytes = b.sort_bytes;
    b.enc_offsets = b.enc_bytes + up(b.enc_cap + 16);
    b.total = b.enc_offsets + up(8 * (n + 1));
    return b;
}

// BigDecimal: the sort workspace, then the encoded strings (at most 7 bytes
// longer than the text: class byte, 5 exponent bytes, terminator; the sign,
// point and exponent characters are not copied), their offsets and the tile
// totals of the length pass.
struct DecLayout {
    size_t sort_bytes, enc_bytes, enc_offsets, tile_sum, total;
    uint64_t enc_cap;
};
DecLayout bigdecimal_layout(uint64_t n, uint64_t total_bytes) {
    auto up = [](size_t x) { return (x + kAlign - 1) / kAlign * kAlign; };
    DecLayout d{};
    d.sort_bytes = up(make_layout(n).total);
    d.enc_cap = total_bytes + 7 * n;
    d.enc_bytes = d.sort_bytes;
    d.enc_offsets = d.enc_bytes + up(d.enc_cap + 16);
    d.tile_sum = d.enc_offsets + up(8 * (n + 1));
    d.total = d.tile_sum + up(8 * (bigdecimal_tiles(n) + 1));
    return d;
}

hs_status hs_bigdecimal_workspace_size(uint64_t n, uint64_t total_bytes, int out_t, size_t *out) {
    g_last_error.clear();
    if (!out) return fail(HS_ERR_INVALID_ARG, "out is NULL");
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    *out = bigdecimal_layout(n, total_bytes).total;
    return HS_OK;
}

hs_status hs_argsort_bigdecimal(const uint8_t *d_bytes, const uint64_t *d_offsets, uint64_t n, uint64_t total_bytes,
                                int out_t, void *d_perm, void *d_ws, size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    if (n > HS_MAX_N) return fail(HS_ERR_INVALID_ARG, "n exceeds HS_MAX_N");
    if (n == 0) return HS_OK;
    if (!d_bytes || !d_offsets || !d_perm) return fail(HS_ERR_INVALID_ARG, "null pointer");
    const DecLayout dl = bigdecimal_layout(n, total_bytes);
    if (d_ws == nullptr || ws_bytes < dl.total)
        return fail(HS_ERR_WORKSPACE, "workspace smaller than hs_bigdecimal_workspace_size()");
    Ctx c;
    hs_status st;
    if (!make_ctx(c, d_ws, dl.sort_bytes, n, stream, &st)) return st;
    uint8_t *eb = c.at<uint8_t>(dl.enc_bytes);
    uint64_t *eo = c.at<uint64_t>(dl.enc_offsets);
    unsigned long long *ts = c.at<unsigned long long>(dl.tile_sum);
    HS_TRY(cudaMemsetAsync(c.ws, 0, c.L.control_end, c.s), "memset control");
    // algorithmic bytes: each pass reads the offsets and the text; the second
    // also writes the encoded strings (at most 7 bytes longer) and offsets
    HS_TRY(c.timed(kKDecimal, 8.0 * (n + 1) + (double)total_bytes, [&] {
               return launch_bigdecimal_lengths(d_bytes, d_offsets, n, total_bytes, ts, c.d_flags, c.s);
           }, 2),
           "bigdecimal lengths");
    HS_TRY(c.read_flags(), "bigdecimal sync");
    if (c.h.error & kErrOffsets)
        return fail(HS_ERR_INVALID_ARG,
                    "a value is not a decimal text, is longer than 32767 bytes, or its offsets decrease or pass "
                    "total_bytes");
    st = device_error_status(c.h);
    if (st != HS_OK) return st;
    HS_TRY(c.timed(kKDecimal, 16.0 * (n + 1) + 2.0 * (double)total_bytes, [&] {
               return launch_bigdecimal_write(d_bytes, d_offsets, n, total_bytes, ts, eb, dl.enc_cap, eo, c.d_flags,
                                              c.s);
           }),
           "bigdecimal write");
    Input in{eb, eo, n, 9, d_perm, out_t == HS_U64 ? 1 : 0};
    return argsort_plain(c, in, HS_CODER_BYTE8);
}

hs_status hs_bigint_workspace_size(uint64_t n, uint64_t total_bytes, int out_t, size_t *out) {
    g_last_error.clear();
    if (!out) return fail(HS_ERR_INVALID_ARG, "out is NULL");
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    *out = bigint_layout(n, total_bytes).total;
    return HS_OK;
}

hs_status hs_argsort_bigint(const uint8_t *d_bytes, const uint64_t *d_offsets, uint64_t n, uint64_t total_bytes,
                            int out_t, void *d_perm, void *d_ws, size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    if (n > HS_MAX_N) return fail(HS_ERR_INVALID_ARG, "n exceeds HS_MAX_N");
    if (n == 0) return HS_OK;
    if (!d_bytes || !d_offsets || !d_perm) return fail(HS_ERR_INVALID_ARG, "null pointer");
    const BigLayout bl = bigint_layout(n, total_bytes);
    if (d_ws == nullptr || ws_bytes < bl.total) return fail(HS_ERR_WORKSPACE, "workspace smaller than hs_bigint_workspace_size()");
    Ctx c;
    hs_status st;
    if (!make_ctx(c, d_ws, bl.sort_bytes, n, stream, &st)) return st;
    uint8_t *eb = c.at<uint8_t>(bl.enc_bytes);
    uint64_t *eo = c.at<uint64_t>(bl.enc_offsets);
    HS_TRY(cudaMemsetAsync(c.ws, 0, c.L.control_end, c.s), "memset control");
    HS_TRY(launch_bigint_encode(d_bytes, d_offsets, n, eb, bl.enc_cap, eo, c.d_flags, c.sms, c.s), "bigint encode");
    HS_TRY(c.read_flags(), "bigint sync");
    if (c.h.error & kErrOffsets)
        return fail(HS_ERR_INVALID_ARG, "a value is empty, not minimal, longer than 32767 bytes or past total_bytes");
    st = device_error_status(c.h);
    if (st != HS_OK) return st;
    Input in{eb, eo, n, 9, d_perm, out_t == HS_U64 ? 1 : 0};
    return argsort_plain(c, in, HS_CODER_BYTE8);
}

hs_status hs_encode_numeric(const void *d_values, uint64_t n, int type, uint64_t *d_codes, void *stream) {
    g_last_error.clear();
    if (type < HS_NUM_U64 || type > HS_NUM_DATETIME) return fail(HS_ERR_INVALID_ARG, "bad numeric type");
    if (n == 0) return HS_OK;
    if (!d_values || !d_codes) return fail(HS_ERR_INVALID_ARG, "null pointer");
    const cudaError_t e = launch_numeric_encode(d_values, n, type, d_codes, nullptr, num_sms_cached(),
                                                static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HS_OK : fail_cuda(e, "numeric encode");
}

hs_status hs_numeric_workspace_size(uint64_t n, int out_t, size_t *out) {
    g_last_error.clear();
    if (!out) return fail(HS_ERR_INVALID_ARG, "out is NULL");
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    *out = make_layout(n).total;
    return HS_OK;
}

hs_status hs_argsort_numeric(const void *d_values, uint64_t n, int type, int out_t, void *d_perm, void *d_ws,
                             size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (type < HS_NUM_U64 || type > HS_NUM_DATETIME) return fail(HS_ERR_INVALID_ARG, "bad numeric type");
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    if (n > HS_MAX_N) return fail(HS_ERR_INVALID_ARG, "n exceeds HS_MAX_N");
    if (n == 0) return HS_OK;
    if (!d_values || !d_perm) return fail(HS_ERR_INVALID_ARG, "null pointer");
    Ctx c;
    hs_status st;
    if (!make_ctx(c, d_ws, ws_bytes, n, stream, &st)) return st;
    SortBufs b{{c.at<uint64_t>(c.L.codes_a), c.at<uint64_t>(c.L.codes_b)},
               {c.at<uint32_t>(c.L.vals_a), c.at<uint32_t>(c.L.vals_b)},
               {c.at<uint32_t>(c.L.segs_a), c.at<uint32_t>(c.L.segs_b)}};
    c.lb_words = sort_tiles(n) * kBins;
    unsigned long long *hist = c.at<unsigned long long>(c.L.hist);
    HS_TRY(cudaMemsetAsync(c.ws, 0, c.L.control_end, c.s), "memset control");
    // Perfect codes (distinct values, distinct codes): Step 2 alone, the last
    // pass writing the permutation; no tie detection or fix-up.  A 32-bit
    // code and the index share one word (32 + 31 bits at most), so those
    // passes move 8 bytes a value instead of 12.
    const bool narrow = type == HS_NUM_I32 || type == HS_NUM_F32;
    int idx_bits = 1;
    while (idx_bits < 32 && (1ull << idx_bits) < n) ++idx_bits;
    const int pack_bits = narrow ? idx_bits : 0;
    HS_TRY(c.timed(kKEncode, (narrow ? 4.0 : 8.0) * n + 8.0 * n, [&] {
               return launch_numeric_encode(d_values, n, type, b.keys[0], hist, c.sms, c.s, pack_bits);
           }),
           "numeric encode");
    HS_TRY(c.timed(kKPlan, 8.0 * kBins * 16, [&] {
               return launch_plan(hist, kKeyPasses, n, c.at<unsigned long long>(c.L.bucket), c.d_flags, c.s);
           }),
           "plan");
    HS_TRY(c.read_flags(), "plan sync");
    int passes[kKeyPasses], np = 0;
    for (int p = 0; p < kKeyPasses; ++p)
        if (c.h.active[p]) passes[np++] = p;
    const OutMode pmode = out_t == HS_U64 ? kOutPerm64 : kOutPerm32;
    int cur = 0;
    if (np == 0) {
        HS_TRY(c.timed(kKIdentity, 4.0 * n, [&] { return launch_identity(nullptr, n, d_perm, pmode, c.s); }),
               "identity");
    } else {
        st = run_passes(c, b, &cur, n, passes, np, false, nullptr, pack_bits == 0, d_perm, pmode, false, pack_bits);
        if (st != HS_OK) return st;
    }
    HS_TRY(c.read_flags(), "final sync");
    return device_error_status(c.h);
}

hs_status hs_host_workspace_size(uint64_t n, uint64_t total_bytes, int mode, int out_t, size_t *out) {
    g_last_error.clear();
    if (!out) return fail(HS_ERR_INVALID_ARG, "out is NULL");
    if (mode != HS_MODE_PLAIN && mode != HS_MODE_LEARNED && mode != HS_MODE_AUTO) return fail(HS_ERR_INVALID_ARG, "bad mode");
    if (mode == HS_MODE_AUTO) mode = HS_MODE_PLAIN;  // see hs_mode
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    *out = make_host_layout(n, total_bytes, mode == HS_MODE_LEARNED, out_t == HS_U64 ? 8 : 4).total;
    return HS_OK;
}

hs_status hs_argsort_host(const uint8_t *h_bytes, const uint64_t *h_offsets, uint64_t n, int mode, int coder,
                          int out_t, void *h_perm, void *d_ws, size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (mode != HS_MODE_PLAIN && mode != HS_MODE_LEARNED && mode != HS_MODE_AUTO) return fail(HS_ERR_INVALID_ARG, "bad mode");
    if (mode == HS_MODE_AUTO) mode = HS_MODE_PLAIN;  // see hs_mode
    if (coder < HS_CODER_AUTO || coder > HS_CODER_ALPHA) return fail(HS_ERR_INVALID_ARG, "bad coder");
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    if (n > HS_MAX_N) return fail(HS_ERR_INVALID_ARG, "n exceeds HS_MAX_N");
    if (n == 0) return HS_OK;
    if (!h_bytes || !h_offsets || !h_perm) return fail(HS_ERR_INVALID_ARG, "null pointer");
    for (const void *p : {(const void *)h_bytes, (const void *)h_offsets, (const void *)h_perm}) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();  // unregistered host memory on older runtimes
            continue;
        }
        if (a.type == cudaMemoryTypeDevice) return fail(HS_ERR_INVALID_ARG, "hs_argsort_host needs host pointers");
    }
    // Chunk boundaries must not decrease (the copies are sized from them);
    // every other offset is checked on the device.
    const uint64_t total = h_offsets[n];
    const uint64_t chunk = host_chunk(n);
    uint64_t prev = h_offsets[0];
    for (uint64_t s1 = chunk; ; s1 += chunk) {
        const uint64_t b = h_offsets[umin64(s1, n)];
        if (b < prev) return fail(HS_ERR_INVALID_ARG, "offsets are decreasing");
        prev = b;
        if (s1 >= n) break;
    }
    const bool learned = mode == HS_MODE_LEARNED;
    const size_t isz = out_t == HS_U64 ? 8 : 4;
    const Layout L = make_host_layout(n, total, learned, isz);
    Ctx c;
    hs_status st;
    if (!make_ctx(c, d_ws, ws_bytes, n, stream, &st, learned, &L)) return st;
    HostSrc hsrc{h_bytes, h_offsets, c.at<uint8_t>(L.dev_bytes), c.at<uint64_t>(L.dev_offsets), total};
    void *d_perm = c.at<void>(L.dev_perm);
    Input in{hsrc.d_bytes, hsrc.d_offsets, n, 9, d_perm, out_t == HS_U64 ? 1 : 0};
    if (learned) {
        // the learned path reads the inputs before and after its own encode:
        // copy them whole first
        HS_TRY(cudaMemcpyAsync(hsrc.d_offsets, h_offsets, (n + 1) * 8, cudaMemcpyHostToDevice, c.s), "copy offsets");
        if (total > h_offsets[0])
            HS_TRY(cudaMemcpyAsync(hsrc.d_bytes + h_offsets[0], h_bytes + h_offsets[0], total - h_offsets[0],
                                   cudaMemcpyHostToDevice, c.s),
                   "copy bytes");
        bool fallback = false;
        st = argsort_learned(c, in, coder, &fallback);
        if (st == HS_OK && fallback) st = argsort_plain(c, in, coder);
    } else {
        c.host = &hsrc;
        c.h_out = h_perm;
        c.h_out_isz = isz;
        st = argsort_plain(c, in, coder);
        c.host = nullptr;
    }
    if (st != HS_OK) return st;
    if (c.early_copy) {
        // the copy issued once the permutation was written has to finish
        // first; then the positions the fix-up rewrote go again
        HS_TRY(cudaStreamWaitEvent(c.s, c.early_copy, 0), "wait early copy");
        uint64_t lo = 0, hi = n - 1;
        bool again = c.dirty_all;
        if (!again && c.h.dirty_lo <= c.h.dirty_hi && c.h.dirty_hi < n) {
            again = true;
            lo = c.h.dirty_lo;
            hi = c.h.dirty_hi;
        }
        if (again)
            HS_TRY(cudaMemcpyAsync(static_cast<char *>(h_perm) + lo * isz, static_cast<char *>(d_perm) + lo * isz,
                                   (hi - lo + 1) * isz, cudaMemcpyDeviceToHost, c.s),
                   "copy rewritten positions");
    } else {
        HS_TRY(cudaMemcpyAsync(h_perm, d_perm, n * isz, cudaMemcpyDeviceToHost, c.s), "copy permutation");
    }
    HS_TRY(cudaStreamSynchronize(c.s), "final sync");
    return HS_OK;
}

hs_status hs_argsort_batched(const uint8_t *d_bytes, const uint64_t *d_offsets, const uint64_t *d_seg_offsets,
                             uint64_t num_segs, uint64_t n, int coder, uint32_t *d_perm, void *d_ws,
                             size_t ws_bytes, void *stream) {
    g_last_error.clear();
    if (coder < HS_CODER_AUTO || coder > HS_CODER_ALPHA) return fail(HS_ERR_INVALID_ARG, "bad coder");
    if (num_segs > 0xFFFFFFFFull) return fail(HS_ERR_INVALID_ARG, "num_segs must fit 32 bits");
    if (n == 0) return HS_OK;
    if (num_segs == 0) return fail(HS_ERR_INVALID_ARG, "n > 0 strings but no instances");
    // Local indices are 31-bit: more strings than num_segs instances of
    // 2^31 - 1 means some instance is too large (the device checks each one).
    if (n > num_segs * (uint64_t)kIdxMask)
        return fail(HS_ERR_INVALID_ARG, "an instance holds 2^31 or more strings");
    if (!d_bytes || !d_offsets || !d_seg_offsets || !d_perm) return fail(HS_ERR_INVALID_ARG, "null pointer");
    Ctx c;
    hs_status st;
    if (!make_ctx(c, d_ws, ws_bytes, n, stream, &st)) return st;
    Input in{d_bytes, d_offsets, n, 9, d_perm, 0};
    return argsort_batched(c, in, d_seg_offsets, num_segs, coder);
}

hs_status hs_batched_workspace_size(uint64_t n, uint64_t num_segs, size_t *out) {
    (void)num_segs;
    g_last_error.clear();
    if (!out) return fail(HS_ERR_INVALID_ARG, "out is NULL");
    *out = make_layout(n).total;
    return HS_OK;
}

hs_status hs_autotune(int mode) {
    g_last_error.clear();
    if (mode < 0 || mode > 2) return fail(HS_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
    std::lock_guard<std::mutex> g(g_tuner.mu);
    if (mode == 2) {
        for (auto &row : g_tuner.choice)
            for (auto &v : row) v = 0;
        g_tuner.enabled = true;
    } else {
        g_tuner.enabled = mode == 1;
    }
    return HS_OK;
}

hs_status hs_autotune_choice(int layout, uint64_t n, int *items) {
    g_last_error.clear();
    if (layout < 0 || layout > 1 || !items) return fail(HS_ERR_INVALID_ARG, "bad layout or NULL");
    std::lock_guard<std::mutex> g(g_tuner.mu);
    *items = n >= (1ull << 20) ? g_tuner.choice[layout][size_class(n)] : 0;
    return HS_OK;
}

hs_status hs_shutdown(void) {
    g_last_error.clear();
    bool ok = true;
    {
        std::lock_guard<std::mutex> g(g_copy_mu);
        int cur = -1;
        const bool have_dev = cudaGetDevice(&cur) == cudaSuccess;
        for (int d = 0; d < kMaxDevices; ++d) {
            if (!g_copy_stream[d]) continue;
            if (have_dev) cudaSetDevice(d);
            ok &= cudaStreamDestroy(g_copy_stream[d]) == cudaSuccess;
            g_copy_stream[d] = nullptr;
        }
        if (have_dev && cur >= 0) cudaSetDevice(cur);
        for (cudaEvent_t e : g_sync_events) ok &= cudaEventDestroy(e) == cudaSuccess;
        g_sync_events.clear();
        for (DevFlags *p : g_pinned_flags) ok &= cudaFreeHost(p) == cudaSuccess;
        g_pinned_flags.clear();
    }
    {
        std::lock_guard<std::mutex> g(g_stats.mu);
        for (cudaEvent_t e : g_stats.pool) ok &= cudaEventDestroy(e) == cudaSuccess;
        g_stats.pool.clear();
        g_stats.enabled = false;
        for (int k = 0; k < kKNumKinds; ++k) {
            g_stats.launches[k] = 0;
            g_stats.ms[k] = 0.0;
            g_stats.bytes[k] = 0.0;
        }
    }
    cudaGetLastError();  // leave no sticky error from the destroys behind
    return ok ? HS_OK : fail(HS_ERR_CUDA, "a stream or event could not be destroyed");
}

hs_status hs_stats_enable(int on) {
    g_last_error.clear();
    std::lock_guard<std::mutex> g(g_stats.mu);
    g_stats.enabled = on != 0;
    if (on) {
        for (int k = 0; k < kKNumKinds; ++k) {
            g_stats.launches[k] = 0;
            g_stats.ms[k] = 0;
            g_stats.bytes[k] = 0;
        }
    }
    return HS_OK;
}

hs_status hs_stats_read(hs_kernel_stat *out, int max, int *count) {
    g_last_error.clear();
    if (!count || (max > 0 && !out)) return fail(HS_ERR_INVALID_ARG, "null pointer");
    std::lock_guard<std::mutex> g(g_stats.mu);
    for (int k = 0; k < kKNumKinds && k < max; ++k) {
        std::memset(&out[k], 0, sizeof(hs_kernel_stat));
        std::strncpy(out[k].name, kKindNames[k], sizeof(out[k].name) - 1);
        out[k].launches = g_stats.launches[k];
        out[k].total_ms = g_stats.ms[k];
        out[k].algo_bytes = g_stats.bytes[k];
    }
    *count = kKNumKinds;
    return HS_OK;
}

hs_status hs_rmi_grad(const float *d_params, const float *d_x, const float *d_t, uint32_t T, float *d_grad,
                      float *d_loss, void *stream) {
    g_last_error.clear();
    if (T < 1 || T > HS_RMI_MAX_POINTS) return fail(HS_ERR_INVALID_ARG, "T must be 1..HS_RMI_MAX_POINTS");
    if (!d_params || !d_x || !d_t || !d_grad || !d_loss) return fail(HS_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HS_TRY(launch_rmi_grad(d_params, d_x, d_t, (int)T, d_grad, d_loss, s), "rmi grad");
    HS_TRY(cudaStreamSynchronize(s), "rmi grad sync");
    return HS_OK;
}

hs_status hs_rmi_leaf_fit(const float *d_x, const float *d_t, const uint32_t *d_leaf_start, uint32_t m,
                          uint32_t leaves, float *d_slope, float *d_icept, float *d_lo, float *d_hi, void *stream) {
    g_last_error.clear();
    if (leaves == 0) return HS_OK;
    if (!d_x || !d_t || !d_leaf_start || !d_slope || !d_icept || !d_lo || !d_hi)
        return fail(HS_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HS_TRY(launch_leaf_fit(d_x, d_t, d_leaf_start, m, (int)leaves, d_slope, d_icept, d_lo, d_hi, s), "leaf fit");
    HS_TRY(cudaStreamSynchronize(s), "leaf fit sync");
    return HS_OK;
}

hs_status hs_rmi_sample_indices(uint64_t n, uint64_t seed, uint64_t *d_out, void *stream) {
    g_last_error.clear();
    const uint64_t m = n / kRmiStride;
    if (m == 0) return HS_OK;
    if (!d_out) return fail(HS_ERR_INVALID_ARG, "null pointer");
    if (m > 0xFFFFFFFFull) return fail(HS_ERR_INVALID_ARG, "n too large");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HS_TRY(launch_sample_indices(n, seed, d_out, (uint32_t)m, s), "sample indices");
    HS_TRY(cudaStreamSynchronize(s), "sample sync");
    return HS_OK;
}

hs_status hs_learned_profile(const uint8_t *d_bytes, const uint64_t *d_offsets, uint64_t n, int linear,
                             uint64_t *d_keys, uint32_t *d_buckets, double *h_info, void *d_ws, size_t ws_bytes,
                             void *stream) {
    g_last_error.clear();
    if (n < kLearnedMinN || n > HS_MAX_N) return fail(HS_ERR_INVALID_ARG, "n must be 65536..HS_MAX_N");
    if (!d_bytes || !d_offsets || !d_keys || !d_buckets) return fail(HS_ERR_INVALID_ARG, "null pointer");
    Ctx c;
    hs_status st;
    if (!make_ctx(c, d_ws, ws_bytes, n, stream, &st, true)) return st;
    Input in{d_bytes, d_offsets, n, 9, nullptr, 0};
    LearnedProfile prof{d_keys, d_buckets, linear, {0, 0, 0, 0}};
    bool fallback = false;
    st = argsort_learned(c, in, HS_CODER_ASCII7, &fallback, &prof);
    if (st != HS_OK) return st;
    if (fallback) return fail(HS_ERR_CODER_DOMAIN, "learned profile needs ASCII7 input");
    if (h_info)
        for (int i = 0; i < 4; ++i) h_info[i] = prof.info[i];
    return HS_OK;
}

hs_status hs_test_bounded_waits(uint32_t spin_limit, int64_t withhold_tile) {
    g_last_error.clear();
    if (withhold_tile < -1) return fail(HS_ERR_INVALID_ARG, "withhold_tile must be -1 or a tile id");
    HS_TRY(set_wait_test(spin_limit, (long long)withhold_tile), "bounded-wait test setting");
    return HS_OK;
}

hs_status hs_learned_force_bucket_bits(int bits) {
    g_last_error.clear();
    if (bits < 0 || bits > 24) return fail(HS_ERR_INVALID_ARG, "bucket bits must be 0 or 1..24");
    g_forced_bucket_bits.store(bits);
    return HS_OK;
}

const char *hs_last_error(void) { return g_last_error.c_str(); }

int hs_version(void) { return 100; }

}  // extern "C"

// ---- allocation-free variant (hs_argsort_noalloc) -----------------------------
//
// The scratch of hs_argsort, carved from one static device array instead of
// a caller-supplied workspace.  Host code must not use the array's name as a
// device address: its device address is looked up with cudaGetSymbolAddress
// once per CUDA context, while that context's device is current, and that
// pointer is what the kernels receive.

static __device__ __align__(256) unsigned char hs_noalloc_scratch[HS_NOALLOC_SCRATCH_BYTES];

namespace hs {
namespace {

// One cached address per CUDA context.  The key is the context's id, not the
// device number: after a device reset the module is loaded again in a new
// context, possibly at another address, and the lookup must be repeated.
struct NoAllocEntry {
    unsigned long long ctx_id;
    void *ptr;
};
std::mutex g_noalloc_mu;
std::vector<NoAllocEntry> g_noalloc_cache;

// The two driver calls, found through the runtime (the library does not
// link the driver, so that it loads on machines without one).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

hs_status driver_calls() {
    if (g_ctx_get_current && g_ctx_get_id) return HS_OK;
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa{}, qb{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
        return fail(HS_ERR_CUDA, "hs_argsort_noalloc: driver entry points cuCtxGetCurrent / cuCtxGetId not found");
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(b);
    return HS_OK;
}

// Device address of the static scratch in the current context (looked up on
// the first call in each context, with that context's device current).
hs_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "hs_argsort_noalloc: cudaGetDevice");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    hs_status st = driver_calls();
    if (st != HS_OK) return st;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) {
        // no context bound to this thread yet: bind the device's primary one
        e = cudaSetDevice(dev);
        if (e != cudaSuccess) return fail_cuda(e, "hs_argsort_noalloc: cudaSetDevice");
        if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr)
            return fail(HS_ERR_CUDA, "hs_argsort_noalloc: no current CUDA context");
    }
    unsigned long long id = 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return fail(HS_ERR_CUDA, "hs_argsort_noalloc: cuCtxGetId failed");
    for (const NoAllocEntry &en : g_noalloc_cache)
        if (en.ctx_id == id) {
            *out = en.ptr;
            return HS_OK;
        }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, hs_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
        return fail_cuda(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "hs_argsort_noalloc: cudaGetSymbolAddress");
    g_noalloc_cache.push_back(NoAllocEntry{id, p});
    *out = p;
    return HS_OK;
}

}  // namespace
}  // namespace hs

extern "C" hs_status hs_argsort_noalloc(const uint8_t *d_bytes, const uint64_t *d_offsets, uint64_t n, int coder,
                                        int out_t, void *d_perm, void *stream) {
    g_last_error.clear();
    if (coder < HS_CODER_AUTO || coder > HS_CODER_ALPHA) return fail(HS_ERR_INVALID_ARG, "bad coder");
    if (out_t != HS_U32 && out_t != HS_U64) return fail(HS_ERR_INVALID_ARG, "bad index type");
    if (n > HS_NOALLOC_MAX_N)
        return fail(HS_ERR_INVALID_ARG, "hs_argsort_noalloc: n exceeds HS_NOALLOC_MAX_N (262144 strings)");
    if (n == 0) return HS_OK;
    if (!d_bytes || !d_offsets || !d_perm) return fail(HS_ERR_INVALID_ARG, "null pointer");
    if (make_layout(n).total > HS_NOALLOC_SCRATCH_BYTES)
        return fail(HS_ERR_INTERNAL, "hs_argsort_noalloc: scratch layout exceeds the static array");
    void *ws = nullptr;
    hs_status st = noalloc_scratch(&ws);
    if (st != HS_OK) return st;
    Ctx c;
    if (!make_ctx(c, ws, HS_NOALLOC_SCRATCH_BYTES, n, stream, &st)) return st;
    c.timing = false;      // no event objects on this path
    c.pinned_ok = false;   // and no host allocation
    Input in{d_bytes, d_offsets, n, 9, d_perm, out_t == HS_U64 ? 1 : 0};
    return argsort_plain(c, in, coder);
}
