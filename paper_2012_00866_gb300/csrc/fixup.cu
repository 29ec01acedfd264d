// Step 3: fix the inversions the code sort leaves (Section 3.1 Step 3,
// Algorithm 1; skipped entirely when the coding is perfect, Section 3.4).
//
// With an order-preserving coder, code(a) < code(b) implies a < b (Section
// 3.2 with p confined to ties), so after a stable sort by code only runs of
// equal codes can be out of order, and only if some member was not exactly
// represented.  The paper re-sorts the whole array with Timsort; here only
// those runs are sorted, by size class:
//   tie detection   one chained-scan pass finds each run of equal keys and
//                   whether any member needs work (decoupled look-back);
//   2..32           a warp per run ranks its members by full comparison;
//   33..2048        a CTA per run sorts (window key, index) in shared memory,
//                   refining 7 bytes at a time until every tie is resolved;
//   larger          refined globally: window keys for all members, a
//                   segmented radix sort by (run, key), and tie detection
//                   again on the result (driven from the host).
#include "hs_internal.h"
#include "hs_fixup.h"

namespace hs {
namespace {

// ---- tie detection ----------------------------------------------------------
//
// Scan state over positions: has_head, position of the last run head, OR of
// the "needs work" flags since that head.  (a then b) = b if b has a head,
// else (a.has, a.last, a.or | b.or).  Held packed in one word, as the 56-bit
// look-back value: bit 55 has, bit 54 or, bits 0..53 last; so combining is a
// select and an OR, and a shuffle moves one word.

constexpr uint64_t kRunLastMask = (1ull << 54) - 1;
constexpr uint64_t kRunHas = 1ull << 55;
constexpr uint64_t kRunOr = 1ull << 54;
static_assert((kRunHas | kRunOr | kRunLastMask) <= kLbValueMask, "packed run state must fit the look-back value");

struct RunState {
    uint64_t v;
    __device__ __forceinline__ uint64_t last() const { return v & kRunLastMask; }
    __device__ __forceinline__ bool orf() const { return (v & kRunOr) != 0; }
};

__device__ __forceinline__ RunState run_state(uint64_t last, bool has, bool orf) {
    return RunState{(has ? kRunHas : 0ull) | (orf ? kRunOr : 0ull) | (last & kRunLastMask)};
}

__device__ __forceinline__ RunState combine(const RunState &a, const RunState &b) {
    return (b.v & kRunHas) ? b : RunState{a.v | (b.v & kRunOr)};
}

__device__ __forceinline__ uint64_t pack(const RunState &s) { return s.v; }
__device__ __forceinline__ RunState unpack(uint64_t v) { return RunState{v}; }

constexpr int kTieThreads = 256;
constexpr int kTieItems = 16;
constexpr int kTieTile = kTieThreads * kTieItems;

__device__ __forceinline__ void push_run(const TieArgs &a, uint64_t start, uint64_t len, uint32_t depth) {
    if (start >= a.perm_n || len > a.perm_n - start) {  // a run must lie inside perm
        atomicOr(&a.flags->error, kErrInternal);
        return;
    }
    RunEntry e;
    e.start = start;
    e.len = (uint32_t)umin64(len, 0xFFFFFFFFull);
    e.depth = depth;
    if (len <= kSmallMax) {
        const unsigned long long i = atomicAdd(&a.flags->qcount[kQSmall], 1ull);
        if (i < a.cap_small) a.q_small[i] = e; else atomicOr(&a.flags->error, kErrInternal);
    } else if (len <= kMediumMax) {
        const unsigned long long i = atomicAdd(&a.flags->qcount[kQMedium], 1ull);
        if (i < a.cap_medium) a.q_medium[i] = e; else atomicOr(&a.flags->error, kErrInternal);
    } else {
        const unsigned long long i = atomicAdd(&a.flags->qcount[a.q_large_id], 1ull);
        if (i < a.cap_large && len < 0xFFFFFFFFull) a.q_large[i] = e;
        else atomicOr(&a.flags->error, kErrInternal);
    }
}

// Keys of the tile (plus one neighbour on each side) are staged through
// shared memory with coalesced loads; each thread then scans 16 consecutive
// positions.  Staging slot x lives at tie_slot(x) = x + x / 16: the 16
// threads of a half-warp read words 17 apart, in distinct bank pairs (without
// the gap all sixteen would hit the same pair).
constexpr int kTieSlots = kTieTile + 2;
__device__ __forceinline__ int tie_slot(int x) { return x + (x >> 4); }
constexpr size_t kTieSmem = (size_t)(kTieSlots + kTieSlots / 16 + 1) * 8;

template <int MODE>
__global__ void __launch_bounds__(kTieThreads, MODE == kTiePacked || MODE == kTieRefine ? 4 : 6)
tie_detect_kernel(const TieArgs a) {
    constexpr bool REFINE = MODE == kTieRefine;
    constexpr bool PACKED = MODE == kTiePacked;  // s_key holds (code << pack_bits) | index
    extern __shared__ __align__(16) unsigned char tie_smem[];
    uint64_t *s_key = reinterpret_cast<uint64_t *>(tie_smem);  // s_key[tie_slot(i + 1)] = keys[t0 + i]
    __shared__ uint64_t s_state[kTieThreads / 32];
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t n = a.n;
    const uint64_t t0 = tile * kTieTile;
    const uint32_t cont_tag = (uint32_t)a.prefix_len + 8;

    for (int i = tid; i < kTieSlots; i += kTieThreads) {
        const uint64_t j = t0 + i;  // position t0 + i - 1
        const bool in = j >= 1 && j - 1 < n;
        cp_async8(&s_key[tie_slot(i)], in ? a.keys + (j - 1) : a.keys, in ? 8u : 0u);
    }
    cp_async_wait_all();
    __syncthreads();

    const int i0 = tid * kTieItems;
    const uint64_t j0 = t0 + i0;
    const bool SEGS = REFINE || a.segs != nullptr;  // runs also break where the segment changes
    uint32_t seg_prev = 0;
    if (SEGS && j0 > 0 && j0 - 1 < n) seg_prev = a.segs[j0 - 1];
    uint32_t heads = 0, flagsb = 0;
    RunState mine{0};
    if (PACKED) {
        // Words (code << pack_bits) | index.  Heads from the codes; only
        // strings with a neighbour of equal code and all coded chars present
        // can be longer than the code, and their not-exact bits are looked
        // up, four loads in flight at a time.
        const int pb = a.pack_bits;
        const uint64_t imask = (1ull << pb) - 1;
        uint32_t need = 0;
        uint64_t kp = s_key[tie_slot(i0)] >> pb, kc = s_key[tie_slot(i0 + 1)] >> pb;
#pragma unroll 4
        for (int i = 0; i < kTieItems; ++i) {
            const uint64_t j = j0 + i;
            const uint64_t kn = s_key[tie_slot(i0 + i + 2)] >> pb;
            const bool head = j == 0 || kc != kp;
            const bool tied = j < n && (!head || (j + 1 < n && kn == kc));
            heads |= (uint32_t)(j < n && head) << i;
            if (tied && (kc & a.last_char_mask) != 0) need |= 1u << i;
            kp = kc;
            kc = kn;
        }
#pragma unroll
        for (int g = 0; g < kTieItems; g += 4) {
            if (((need >> g) & 0xFu) == 0) continue;
            uint32_t word[4], sh[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t idx = (uint32_t)(s_key[tie_slot(i0 + g + q + 1)] & imask);
                sh[q] = idx & 31u;
                word[q] = ((need >> (g + q)) & 1u) ? __ldg(&a.bits[idx >> 5]) : 0u;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) flagsb |= ((word[q] >> sh[q]) & 1u) << (g + q);
        }
#pragma unroll
        for (int i = 0; i < kTieItems; ++i)
            if (j0 + i < n) mine = combine(mine, run_state(j0 + i, (heads >> i) & 1u, (flagsb >> i) & 1u));
        // The permutation is the words' index fields in tile order:
        // written with coalesced stores (unless the last radix pass wrote it).
        const int cnt = a.perm ? (int)umin64(kTieTile, n - t0) : 0;
        for (int i = tid; i < cnt; i += kTieThreads) {
            const uint64_t idx = s_key[tie_slot(i + 1)] & imask;
            if (a.perm_u64)
                static_cast<uint64_t *>(a.perm)[t0 + i] = idx;
            else
                static_cast<uint32_t *>(a.perm)[t0 + i] = (uint32_t)idx;
        }
    } else {
        uint64_t k_prev = s_key[tie_slot(i0)];
#pragma unroll
        for (int i = 0; i < kTieItems; ++i) {
            const uint64_t j = j0 + i;
            if (j < n) {
                const uint64_t k = s_key[tie_slot(i0 + i + 1)];
                const uint32_t sg = SEGS ? a.segs[j] : 0;
                const bool head = (j == 0) || k != k_prev || (SEGS && sg != seg_prev);
                k_prev = k;
                bool f;
                if (MODE == kTieKeyFlag) f = (k & 1u) != 0;
                else if (MODE == kTieValFlag) f = (a.vals[j] >> 31) != 0;
                else f = window_tag(k) == cont_tag;
                heads |= (uint32_t)head << i;
                flagsb |= (uint32_t)f << i;
                mine = combine(mine, run_state(j, head, f));
                seg_prev = sg;
            }
        }
    }

    // Exclusive scan of thread states across the block.
    RunState x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const RunState y{__shfl_up_sync(kFull, x.v, o)};
        if (lane >= o) x = combine(y, x);
    }
    if (lane == 31) s_state[warp] = pack(x);
    __syncthreads();
    RunState wpre{0};
    for (int w = 0; w < warp; ++w) wpre = combine(wpre, unpack(s_state[w]));
    RunState excl;
    {
        const RunState xp{__shfl_up_sync(kFull, x.v, 1)};
        excl = lane == 0 ? wpre : combine(wpre, xp);
    }

    // Tile aggregate and look-back (warp 0).  Lane i reads the word of tile
    // t - i, 32 predecessors per round trip; the ready words before the first
    // inclusive one (or before the first unwritten one) are folded in
    // position order by a shuffle reduction.
    if (warp == 0) {
        RunState agg{0};
        for (int w = 0; w < kTieThreads / 32; ++w) agg = combine(agg, unpack(s_state[w]));
        uint64_t *lb = a.lookback + tile;
        const uint32_t epoch = a.epoch;
        RunState prefix{0};
        if (tile == 0) {
            if (lane == 0) st_relaxed(lb, lb_word(epoch, kLbInclusive, pack(agg)));
        } else {
            if (lane == 0) st_relaxed(lb, lb_word(epoch, kLbAggregate, pack(agg)));
            int64_t t = (int64_t)tile - 1;
            uint32_t spins = 0;
            while (t >= 0) {
                const int64_t tt = t - lane;
                const uint64_t v = tt >= 0 ? ld_relaxed(&a.lookback[tt]) : 0;
                const bool ready = tt >= 0 && (uint32_t)(v >> 58) == epoch;
                const bool incl = ready && (v & (3ull << 56)) == kLbInclusive;
                const unsigned not_ready = __ballot_sync(kFull, !ready && tt >= 0);
                const unsigned inclusive = __ballot_sync(kFull, incl);
                const int first_nr = not_ready ? __ffs(not_ready) - 1 : 32;
                const int first_in = inclusive ? __ffs(inclusive) - 1 : 32;
                const int stop = first_in < first_nr ? first_in : first_nr - 1;  // last lane to fold
                const int avail = t + 1 < 32 ? (int)(t + 1) : 32;               // lanes with tt >= 0
                const int last = stop < avail - 1 ? stop : avail - 1;
                if (last >= 0) {
                    // fold lanes 0..last; lane i holds the word of an earlier tile than lane i-1
                    RunState x = lane <= last ? unpack(v & kLbValueMask) : RunState{0};
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const RunState y{__shfl_down_sync(kFull, x.v, o)};
                        if (lane + o < 32) x = combine(y, x);
                    }
                    const RunState folded{__shfl_sync(kFull, x.v, 0)};
                    prefix = combine(folded, prefix);
                }
                if (first_in < first_nr) break;  // folded through an inclusive prefix
                if (last >= 0) {
                    t -= last + 1;
                } else {
                    if (++spins > kSpinLimit) {
                        if (lane == 0) atomicOr(&a.flags->error, kErrTimeout);
                        break;
                    }
                    if (spins > 8) __nanosleep(32);
                }
            }
            if (lane == 0) st_relaxed(lb, lb_word(epoch, kLbInclusive, pack(combine(prefix, agg))));
        }
        if (lane == 0) s_prefix = pack(prefix);
    }
    __syncthreads();
    RunState st = combine(unpack(s_prefix), excl);

    // Replay my items: write the permutation, emit runs at their tails.
    uint32_t next_seg = 0;
    const uint64_t jn = j0 + kTieItems;
    if (SEGS && jn < n) next_seg = a.segs[jn];
#pragma unroll
    for (int i = 0; i < kTieItems; ++i) {
        const uint64_t j = j0 + i;
        if (j >= n) break;
        const bool head = (heads >> i) & 1u;
        const bool f = (flagsb >> i) & 1u;
        st = combine(st, run_state(j, head, f));
        uint64_t pos = j, run_start = st.last();
        uint32_t depth = 0;
        if (REFINE) {
            const uint32_t sg = a.segs[j];
            const RunEntry r = a.runs[sg];
            pos = r.start + (j - a.run_base[sg]);
            run_start = r.start + (st.last() - a.run_base[sg]);
            depth = r.depth + 1;
        }
        if (MODE == kTieValFlag || REFINE) {
            const uint32_t v = a.vals[j];
            const uint32_t out = REFINE ? v : (v & kIdxMask);
            if (a.perm_u64)
                static_cast<uint64_t *>(a.perm)[pos] = out;
            else
                static_cast<uint32_t *>(a.perm)[pos] = out;
        }
        bool tail;
        if (i + 1 < kTieItems) {
            tail = (j + 1 >= n) || ((heads >> (i + 1)) & 1u);
        } else if (jn >= n) {
            tail = true;
        } else {
            const int pb = PACKED ? a.pack_bits : 0;
            tail = (s_key[tie_slot(i0 + i + 2)] >> pb) != (s_key[tie_slot(i0 + i + 1)] >> pb) ||
                   (SEGS && next_seg != a.segs[j]);
        }
        if (tail) {
            const uint64_t len = j - st.last() + 1;
            if (len >= 2 && st.orf()) push_run(a, run_start, len, depth);
        }
    }
}

// ---- tie detection without a scan (unsegmented keys, flag in bit 0) ------------
// A run needing work is a run of two or more equal keys with bit 0 (not
// exact) set; all its members share bit 0.  Its head is the position whose
// key differs from the predecessor's and equals the successor's.  Each head's
// thread finds the run's end by a galloping search over the sorted keys (the
// first larger key) and queues the run; every other position costs one
// comparison with a neighbour, so the pass is one streaming read of the keys
// with no look-back.  Used when the permutation is already written and no
// segment ids break runs (instance ids, when there are any, are in the key).

constexpr int kHeadThreads = 256;
constexpr int kHeadItems = 8;  // keys a thread; a warp takes 256 consecutive keys, all loads in flight together

// The end of the run of key k that starts at j (keys[j + 1] == k): the first
// position after it, by a galloping search and a bisection.
__device__ uint64_t run_end(const uint64_t *__restrict__ keys, uint64_t n, uint64_t j, uint64_t k) {
    uint64_t lo = j + 1, hi, step = 2;
    for (;;) {
        hi = lo + step;
        if (hi >= n) {
            hi = n;
            break;
        }
        if (keys[hi] != k) break;
        lo = hi;
        step <<= 1;
    }
    while (hi - lo > 1) {  // keys[lo] == k; hi == n or keys[hi] != k
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (keys[mid] == k) lo = mid; else hi = mid;
    }
    return hi;
}

// Small runs (the common kind) are gathered in shared memory and queued a
// batch at a time, one counter update per batch: with millions of runs, one
// atomic per run on the queue's single counter serialises.
constexpr int kHeadBatch = 2048;  // buffered small runs; a block iteration finds at most 1024

__device__ void flush_small(const TieArgs &a, RunEntry *s_runs, unsigned int *s_cnt, unsigned long long *s_base) {
    __syncthreads();
    const unsigned int cnt = *s_cnt;
    if (cnt) {
        if (threadIdx.x == 0) *s_base = atomicAdd(&a.flags->qcount[kQSmall], (unsigned long long)cnt);
        __syncthreads();
        const unsigned long long base = *s_base;
        for (unsigned int t = threadIdx.x; t < cnt; t += kHeadThreads) {
            if (base + t < a.cap_small) a.q_small[base + t] = s_runs[t];
            else atomicOr(&a.flags->error, kErrInternal);
        }
        __syncthreads();
        if (threadIdx.x == 0) *s_cnt = 0;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kHeadThreads) tie_heads_kernel(const TieArgs a) {
    __shared__ RunEntry s_runs[kHeadBatch];
    __shared__ unsigned int s_cnt;
    __shared__ unsigned long long s_base;
    const uint64_t n = a.n;
    const uint64_t *__restrict__ keys = a.keys;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint64_t kChunk = 32 * kHeadItems;
    constexpr uint64_t kBlockKeys = kChunk * (kHeadThreads / 32);
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (uint64_t bb = (uint64_t)blockIdx.x * kBlockKeys; bb < n; bb += (uint64_t)gridDim.x * kBlockKeys) {
        const uint64_t base = bb + (uint64_t)warp * kChunk;
        uint64_t key[kHeadItems];
#pragma unroll
        for (int k = 0; k < kHeadItems; ++k) {
            const uint64_t j = base + k * 32 + lane;
            key[k] = j < n ? keys[j] : 0ull;
        }
        // the neighbours just outside the warp's chunk
        const uint64_t before = (lane == 0 && base > 0 && base - 1 < n) ? keys[base - 1] : 0ull;
        const uint64_t after = (lane == 31 && base + kChunk < n) ? keys[base + kChunk] : 0ull;
#pragma unroll
        for (int k = 0; k < kHeadItems; ++k) {
            const uint64_t j = base + k * 32 + lane;
            uint64_t prev = __shfl_up_sync(kFull, key[k], 1);
            const uint64_t wrap_prev = __shfl_sync(kFull, key[k > 0 ? k - 1 : 0], 31);
            uint64_t next = __shfl_down_sync(kFull, key[k], 1);
            const uint64_t wrap_next = __shfl_sync(kFull, key[k + 1 < kHeadItems ? k + 1 : k], 0);
            if (lane == 0) prev = k > 0 ? wrap_prev : before;
            if (lane == 31) next = k + 1 < kHeadItems ? wrap_next : after;
            if (j >= n) continue;
            const uint64_t kk = key[k];
            if (!(kk & 1ull)) continue;                        // exact: copies, already in index order
            if (j > 0 && prev == kk) continue;                 // not the head of its run
            if (j + 1 >= n || next != kk) continue;            // a single key
            const uint64_t len = run_end(keys, n, j, kk) - j;
            if (len <= kSmallMax) s_runs[atomicAdd(&s_cnt, 1u)] = RunEntry{j, (unsigned)len, 0u};
            else push_run(a, j, len, 0);
        }
        // at most kHeadBatch / 2 runs an iteration: flush once half full
        __syncthreads();
        if (s_cnt >= kHeadBatch / 2) flush_small(a, s_runs, &s_cnt, &s_base);
    }
    flush_small(a, s_runs, &s_cnt, &s_base);
}

// ---- 2: thread per run ------------------------------------------------------
// Pairs are most of the small runs on long text (two strings that share the
// coded prefix), and each is a chain of dependent loads (the entry, the two
// indices, their offsets, the bytes), so a thread per pair keeps 32 times as
// many of them in flight as a warp per run.  The order is the warp kernel's:
// by the strings from the window offset on, then by index.

template <typename IdxT>
__global__ void __launch_bounds__(256)
pair_runs_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                 IdxT *__restrict__ perm, const RunEntry *__restrict__ q,
                 const unsigned long long *__restrict__ qcount, uint64_t first, uint64_t cap, uint64_t perm_n,
                 Instances inst, int prefix_len, DevFlags *dirty) {
    if (stopped(inst)) return;
    const uint64_t count = umin64(*qcount, cap);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = first + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += stride) {
        const RunEntry e = q[r];
        if (e.len != 2 || e.start >= perm_n || perm_n - e.start < 2) continue;
        const uint64_t base = instance_base(inst, e.start);
        const IdxT i0 = perm[e.start], i1 = perm[e.start + 1];
        const uint64_t o0 = offsets[base + i0], l0 = offsets[base + i0 + 1] - o0;
        const uint64_t o1 = offsets[base + i1], l1 = offsets[base + i1 + 1] - o1;
        const uint64_t from = min(window_offset(prefix_len, e.depth), min(l0, l1));
        const int c = compare_from(bytes + o0, l0, bytes + o1, l1, from);
        if (c > 0 || (c == 0 && i1 < i0)) {
            perm[e.start] = i1;
            perm[e.start + 1] = i0;
            mark_dirty(dirty, e.start, 2);
        }
    }
}

// ---- 3..32: warp per run ----------------------------------------------------

template <typename IdxT>
__global__ void __launch_bounds__(256)
small_runs_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                  IdxT *__restrict__ perm, const RunEntry *__restrict__ q,
                  const unsigned long long *__restrict__ qcount, uint64_t first, uint64_t cap, uint64_t perm_n,
                  Instances inst, int prefix_len, DevFlags *dirty) {
    if (stopped(inst)) return;
    const int lane = threadIdx.x & 31;
    const uint64_t warp_id = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t count = umin64(*qcount, cap);
    for (uint64_t r = first + warp_id; r < count; r += nwarps) {
        const RunEntry e = q[r];
        if (e.len > kSmallMax || e.start >= perm_n || e.len > perm_n - e.start) continue;  // never queued
        if (e.len == 2) continue;  // pair_runs_kernel's
        const bool mine = (uint32_t)lane < e.len;
        const uint64_t base = instance_base(inst, e.start);  // string index of local index 0
        IdxT idx = 0;
        uint64_t off = 0, len = 0;
        if (mine) {
            idx = perm[e.start + lane];
            off = offsets[base + idx];
            len = offsets[base + idx + 1] - off;
        }
        const uint64_t o = window_offset(prefix_len, e.depth);
        {
            // copies of one string are already in index order: nothing to do
            const uint64_t o0 = __shfl_sync(kFull, off, 0), l0 = __shfl_sync(kFull, len, 0);
            const bool eq = !mine || equal_from(bytes + off, len, bytes + o0, l0, min(o, l0));
            if (__all_sync(kFull, eq)) continue;
        }
        uint32_t rank = 0;
        for (uint32_t m = 0; m < e.len; ++m) {
            const IdxT im = __shfl_sync(kFull, idx, m);
            const uint64_t om = __shfl_sync(kFull, off, m);
            const uint64_t lm = __shfl_sync(kFull, len, m);
            if (mine && m != (uint32_t)lane) {
                const uint64_t from = min(o, min(len, lm));
                const int c = compare_from(bytes + off, len, bytes + om, lm, from);
                if (c > 0 || (c == 0 && im < idx)) ++rank;
            }
        }
        __syncwarp();
        if (mine) perm[e.start + rank] = idx;
        if (lane == 0) mark_dirty(dirty, e.start, e.len);
        __syncwarp();
    }
}

// ---- >2048: runs of copies of one string ------------------------------------
// A run whose members are all the same string is already in index order
// (the stable sort kept input order), so it needs no refinement.  Two
// launches with fixed grids, every count read on the device:
//   sample  CTA per run: 64 members spread over the run against the first;
//           a difference (or a malformed entry, left for the later checks)
//           marks the run distinct.  The last CTA to finish computes the
//           exclusive sum of the lengths of the unmarked runs;
//   full    every member of those runs, flattened over the grid, against its
//           run's first member.  The last CTA to finish copies the distinct
//           runs to q_out.
// "Last CTA" is the usual fence-and-count hand-off: no CTA waits on another.

template <typename IdxT>
__device__ __forceinline__ bool member_equals_first(const uint8_t *bytes, const uint64_t *offsets,
                                                    const IdxT *perm, const RunEntry &e, uint64_t base,
                                                    uint64_t j, int prefix_len) {
    const uint64_t g0 = base + perm[e.start];
    const uint64_t g = base + perm[e.start + j];
    const uint64_t o0 = offsets[g0], l0 = offsets[g0 + 1] - o0;
    const uint64_t off = offsets[g], len = offsets[g + 1] - off;
    const uint64_t from = min(window_offset(prefix_len, e.depth), l0);
    return len == l0 && same_from(bytes + off, bytes + o0, l0, from, suffix_word(bytes + off, l0, from),
                                  suffix_word(bytes + o0, l0, from));
}

__device__ __forceinline__ bool odd_run(const RunEntry &e, uint64_t perm_n) {
    return e.len < 2 || e.start >= perm_n || e.len > perm_n - e.start;
}

// True in every thread of the CTA that finishes last among gridDim.x.
__device__ __forceinline__ bool last_cta(unsigned int *done) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    const bool last = s_last != 0;
    if (last) __threadfence();
    return last;
}

template <typename IdxT>
__global__ void __launch_bounds__(256)
distinct_sample_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                       const IdxT *__restrict__ perm, const RunEntry *__restrict__ q,
                       const unsigned long long *__restrict__ qcount, uint64_t cap, uint64_t perm_n,
                       Instances inst, int prefix_len, uint32_t *diff, unsigned long long *base,
                       unsigned int *done) {
    if (stopped(inst)) return;
    __shared__ unsigned long long s_warp[8];
    __shared__ unsigned long long s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t count = umin64(*qcount, cap);
    for (uint64_t r = blockIdx.x; r < count; r += gridDim.x) {
        const RunEntry e = q[r];
        bool d = odd_run(e, perm_n);  // uniform over the CTA
        if (!d && tid < 64) {
            const uint64_t j = (uint64_t)tid * (e.len - 1) / 63;
            d = !member_equals_first(bytes, offsets, perm, e, instance_base(inst, e.start), j, prefix_len);
        }
        d = __syncthreads_or(d);
        if (tid == 0) diff[r] = d ? 1u : 0u;
    }
    if (!last_cta(done)) return;
    // exclusive sum of the unmarked runs' lengths; base[count] = total
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t b0 = 0; b0 < count; b0 += blockDim.x) {
        const uint64_t r = b0 + tid;
        const unsigned long long v = (r < count && !((volatile uint32_t *)diff)[r]) ? q[r].len : 0;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        unsigned long long wsum = 0;
        for (int w = 0; w < warp; ++w) wsum += s_warp[w];
        const unsigned long long carry = s_carry;
        if (r < count) base[r] = carry + wsum + x - v;
        __syncthreads();
        if (tid == blockDim.x - 1) s_carry = carry + wsum + x;
        __syncthreads();
    }
    if (tid == 0) base[count] = s_carry;
}

template <typename IdxT>
__global__ void __launch_bounds__(256)
distinct_full_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                     const IdxT *__restrict__ perm, const RunEntry *__restrict__ q,
                     const unsigned long long *__restrict__ qcount, uint64_t cap, Instances inst, int prefix_len,
                     const unsigned long long *__restrict__ base, uint32_t *diff, RunEntry *__restrict__ q_out,
                     unsigned long long *qcount_out, uint64_t cap_out, DevFlags *flags, unsigned int *done) {
    if (stopped(inst)) return;
    const uint64_t count = umin64(*qcount, cap);
    const uint64_t total = base[count];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        // the last run whose range starts at or before i (empty ranges of
        // marked runs share their successor's start and come before it)
        uint64_t lo = 0, hi = count;
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (base[mid] <= i) lo = mid; else hi = mid;
        }
        const RunEntry e = q[lo];
        const uint64_t j = i - base[lo];
        if (j >= e.len) continue;  // cannot happen for a consistent scan
        if (!member_equals_first(bytes, offsets, perm, e, instance_base(inst, e.start), j, prefix_len))
            diff[lo] = 1u;
    }
    if (!last_cta(done)) return;
    for (uint64_t r = threadIdx.x; r < count; r += blockDim.x) {
        if (!((volatile uint32_t *)diff)[r]) continue;
        const unsigned long long k = atomicAdd(qcount_out, 1ull);
        if (k < cap_out) q_out[k] = q[r];
        else atomicOr(&flags->error, kErrInternal);
    }
}

// ---- copies filter for CTA-sized runs ----------------------------------------
//
// A run whose members are all copies of one string is final already (the
// stable code sort kept them in index order).  A CTA of 512 per run compares
// every member with the first: each thread's four members and the first have
// their index, offset and byte loads issued together (three round trips a
// run), and a run of copies gets length 0 so that the sorting
// kernel passes over it.  The sorting kernel keeps its own test for the runs
// that arrive later, from refinement.

constexpr int kCopiesThreads = 512;
constexpr int kCopiesPer = kMediumMax / kCopiesThreads;  // members a thread checks

template <typename IdxT>
__global__ void __launch_bounds__(kCopiesThreads)
copies_filter_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                     const IdxT *__restrict__ perm, RunEntry *__restrict__ q,
                     const unsigned long long *__restrict__ qcount, uint64_t cap, uint64_t perm_n, Instances inst,
                     int prefix_len) {
    if (stopped(inst)) return;
    static_assert(kCopiesPer * kCopiesThreads == kMediumMax, "a thread's members must cover the class");
    const int tid = threadIdx.x;
    const uint64_t count = umin64(*qcount, cap);
    for (uint64_t r = blockIdx.x; r < count; r += gridDim.x) {
        const RunEntry e = q[r];
        if (odd_run(e, perm_n) || e.len > (uint32_t)kMediumMax) continue;  // uniform over the CTA
        const uint64_t base = instance_base(inst, e.start);
        uint64_t g[kCopiesPer + 1];  // g[0]: the first member
        g[0] = base + perm[e.start];
#pragma unroll
        for (int u = 0; u < kCopiesPer; ++u) {
            const uint32_t j = (uint32_t)(u * kCopiesThreads + tid);
            g[u + 1] = j < e.len ? base + perm[e.start + j] : ~0ull;
        }
        uint64_t off[kCopiesPer + 1], len[kCopiesPer + 1];
#pragma unroll
        for (int u = 0; u <= kCopiesPer; ++u) {
            const uint64_t gg = g[u] == ~0ull ? g[0] : g[u];
            off[u] = offsets[gg];
            len[u] = offsets[gg + 1] - off[u];
        }
        const uint64_t l0 = len[0], from = min(window_offset(prefix_len, e.depth), l0);
        uint64_t w[kCopiesPer + 1];
#pragma unroll
        for (int u = 0; u <= kCopiesPer; ++u) w[u] = suffix_word(bytes + off[u], l0, from);
        bool eq = true;
#pragma unroll
        for (int u = 1; u <= kCopiesPer; ++u)
            eq &= len[u] == l0 && same_from(bytes + off[u], bytes + off[0], l0, from, w[u], w[0]);
        if (__syncthreads_and(eq) && tid == 0) q[r].len = 0;
    }
}

// ---- 33..2048: CTA per run ---------------------------------------------------

constexpr int kMedThreads = 512;

template <typename IdxT>
__device__ __forceinline__ bool elem_greater(uint32_t sa, uint64_t ka, IdxT ia,
                                             uint32_t sb, uint64_t kb, IdxT ib) {
    if (sa != sb) return sa > sb;
    if (ka != kb) return ka > kb;
    return ia > ib;
}

template <typename IdxT>
__global__ void __launch_bounds__(kMedThreads)
medium_runs_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                   IdxT *__restrict__ perm, const RunEntry *__restrict__ q,
                   const unsigned long long *__restrict__ qcount, uint64_t first, uint64_t cap, uint64_t perm_n,
                   Instances inst, int prefix_len, DevFlags *dirty) {
    if (stopped(inst)) return;
    constexpr int CAP = kMediumMax;
    __shared__ uint64_t s_key[CAP];
    __shared__ uint32_t s_seg[CAP];
    __shared__ IdxT s_idx[CAP];
    __shared__ uint8_t s_segact[CAP];
    __shared__ uint8_t s_newact[CAP];
    __shared__ uint32_t s_scan[kMedThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t count = umin64(*qcount, cap);
    const uint32_t cont_tag = (uint32_t)prefix_len + 8;

    for (uint64_t r = first + blockIdx.x; r < count; r += gridDim.x) {
        const RunEntry e = q[r];
        // length 0: copies of one string (marked by the copies filter)
        if (e.len < 2 || e.len > (uint32_t)CAP || e.start >= perm_n || e.len > perm_n - e.start) continue;
        const int len = (int)e.len;
        const uint64_t base = instance_base(inst, e.start);
        int P = 1;
        while (P < len) P <<= 1;
        __syncthreads();
        for (int j = tid; j < P; j += kMedThreads) {
            if (j < len) {
                s_idx[j] = perm[e.start + j];
                s_seg[j] = 0;
            } else {
                s_idx[j] = (IdxT)~(IdxT)0;
                s_seg[j] = 0xFFFFFFFFu;
                s_key[j] = ~0ull;
            }
            s_segact[j] = (j == 0);
        }
        {
            // copies of one string are already in index order: nothing to do
            __syncthreads();
            const uint64_t g0 = base + s_idx[0];
            const uint64_t o0 = offsets[g0], l0 = offsets[g0 + 1] - o0;
            const uint64_t from = min(window_offset(prefix_len, e.depth), l0);
            bool eq = true;
            for (int j = tid; j < len && eq; j += kMedThreads) {
                const uint64_t g = base + s_idx[j];
                const uint64_t off = offsets[g];
                eq = equal_from(bytes + off, offsets[g + 1] - off, bytes + o0, l0, from);
            }
            if (__syncthreads_and(eq)) continue;
        }
        uint32_t depth = e.depth;
        for (;;) {
            __syncthreads();
            const uint64_t o = window_offset(prefix_len, depth);
            for (int j = tid; j < len; j += kMedThreads) {
                if (s_segact[s_seg[j]]) {
                    const uint64_t g = base + s_idx[j];
                    const uint64_t off = offsets[g];
                    s_key[j] = window_key(bytes + off, offsets[g + 1] - off, o, prefix_len);
                } else {
                    s_key[j] = 0;
                }
            }
            __syncthreads();
            // Bitonic sort of P elements by (seg, key, idx), skipped when the
            // run is already in that order (e.g. copies of one string).
            bool unsorted = false;
            for (int j = tid; j + 1 < len; j += kMedThreads)
                unsorted |= elem_greater<IdxT>(s_seg[j], s_key[j], s_idx[j], s_seg[j + 1], s_key[j + 1], s_idx[j + 1]);
            const bool do_sort = __syncthreads_or(unsorted);
            for (int k = 2; do_sort && k <= P; k <<= 1) {
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    for (int i = tid; i < P; i += kMedThreads) {
                        const int ixj = i ^ jj;
                        if (ixj > i) {
                            const bool up = (i & k) == 0;
                            const bool gt = elem_greater<IdxT>(s_seg[i], s_key[i], s_idx[i],
                                                               s_seg[ixj], s_key[ixj], s_idx[ixj]);
                            if (gt == up) {
                                uint32_t ts = s_seg[i]; s_seg[i] = s_seg[ixj]; s_seg[ixj] = ts;
                                uint64_t tk = s_key[i]; s_key[i] = s_key[ixj]; s_key[ixj] = tk;
                                IdxT ti = s_idx[i]; s_idx[i] = s_idx[ixj]; s_idx[ixj] = ti;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            // New segments: heads where (seg, key) changes; a segment stays
            // active iff its members continue past the window and it has at
            // least two members.  Thread t owns items [t*4, t*4+4).
            constexpr int PER = CAP / kMedThreads;
            uint32_t hcount = 0;
            bool head[PER], act[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int j = tid * PER + u;
                head[u] = false;
                act[u] = false;
                if (j < len) {
                    const bool same_prev = j > 0 && s_seg[j - 1] == s_seg[j] && s_key[j - 1] == s_key[j];
                    const bool same_next = j + 1 < len && s_seg[j + 1] == s_seg[j] && s_key[j + 1] == s_key[j];
                    const bool was_active = s_segact[s_seg[j]] != 0;
                    head[u] = !same_prev;
                    act[u] = was_active && window_tag(s_key[j]) == cont_tag && (same_prev || same_next);
                    hcount += head[u];
                }
            }
            // exclusive scan of head counts
            uint32_t xs = hcount;
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                uint32_t y = __shfl_up_sync(kFull, xs, o2);
                if (lane >= o2) xs += y;
            }
            if (lane == 31) s_scan[warp] = xs;
            __syncthreads();
            uint32_t base = 0;
            for (int w = 0; w < warp; ++w) base += s_scan[w];
            base += xs - hcount;
            bool any = false;
            uint32_t segid = base;  // id of the segment the next head opens
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int j = tid * PER + u;
                if (j < len) {
                    if (head[u]) {
                        s_newact[segid] = act[u];
                        ++segid;
                    }
                    any |= act[u];
                }
            }
            __syncthreads();
            // relabel (segid - 1 is the segment of the last head at or before j)
            segid = base;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int j = tid * PER + u;
                if (j < len) {
                    if (head[u]) ++segid;
                    s_seg[j] = segid - 1;
                }
            }
            __syncthreads();
            for (int j = tid; j < len; j += kMedThreads) s_segact[j] = s_newact[j];
            if (!__syncthreads_or(any)) break;
            ++depth;
        }
        for (int j = tid; j < len; j += kMedThreads) perm[e.start + j] = s_idx[j];
        if (tid == 0) mark_dirty(dirty, e.start, (uint64_t)len);
    }
}

// ---- large-run helpers ---------------------------------------------------------

// run_base[r] = sum of lengths of runs before r; run_base[count] = total.
__global__ void run_scan_kernel(const RunEntry *__restrict__ runs, uint64_t count,
                                unsigned long long *__restrict__ run_base) {
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t b = 0; b < count; b += blockDim.x) {
        const uint64_t r = b + tid;
        const unsigned long long v = r < count ? runs[r].len : 0;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        unsigned long long wsum = 0;
        for (int w = 0; w < warp; ++w) wsum += s_warp[w];
        const unsigned long long carry = s_carry;
        if (r < count) run_base[r] = carry + wsum + x - v;
        __syncthreads();
        if (tid == blockDim.x - 1) s_carry = carry + wsum + x;
        __syncthreads();
    }
    if (tid == 0) run_base[count] = s_carry;
}

// The window keys of every string at one refinement depth, in string order.
// Offsets are read coalesced and the bytes nearly so (consecutive threads
// take consecutive strings); the refinement then gathers one word a member
// from here instead of a member's offsets and bytes from scattered sectors.
__global__ void window_dense_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                                    uint64_t n, int prefix_len, uint32_t depth, uint64_t *__restrict__ win) {
    const uint64_t o = window_offset(prefix_len, depth);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t off = offsets[i];
        win[i] = window_key(bytes + off, offsets[i + 1] - off, o, prefix_len);
    }
}

// win (nullable): window keys of all strings at depth win_depth; runs at
// that depth read their members' keys there.
template <typename IdxT>
__global__ void refine_keys_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                                   const IdxT *__restrict__ perm, const RunEntry *__restrict__ runs,
                                   uint64_t count, const unsigned long long *__restrict__ run_base,
                                   uint64_t total, Instances inst, int prefix_len,
                                   const uint64_t *__restrict__ win, uint32_t win_depth,
                                   uint64_t *__restrict__ keys, uint32_t *__restrict__ segs,
                                   uint32_t *__restrict__ vals, DevFlags *flags) {
    if (stopped(inst)) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool nonconst = false;
    for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < total; a += stride) {
        // run containing a: last r with run_base[r] <= a
        uint64_t lo = 0, hi = count;  // invariant run_base[lo] <= a < run_base[hi]
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (run_base[mid] <= a) lo = mid; else hi = mid;
        }
        const RunEntry r = runs[lo];
        const uint64_t pos = r.start + (a - run_base[lo]);
        const uint64_t base = instance_base(inst, r.start);
        const IdxT idx = perm[pos];
        const uint64_t g0 = base + perm[r.start];
        uint64_t k, k0;
        if (win != nullptr && r.depth == win_depth) {
            k = win[base + idx];
            k0 = win[g0];
        } else {
            const uint64_t o = window_offset(prefix_len, r.depth);
            const uint64_t off = offsets[base + idx];
            k = window_key(bytes + off, offsets[base + idx + 1] - off, o, prefix_len);
            const uint64_t off0 = offsets[g0];
            k0 = window_key(bytes + off0, offsets[g0 + 1] - off0, o, prefix_len);
        }
        nonconst |= k != k0;
        keys[a] = k;
        segs[a] = (uint32_t)lo;
        vals[a] = (uint32_t)idx;
    }
    if (__syncthreads_or(nonconst) && threadIdx.x == 0) atomicOr(&flags->nonconst, 1u);
}

__global__ void push_constant_runs_kernel(const RunEntry *__restrict__ runs, uint64_t count,
                                          const unsigned long long *__restrict__ run_base,
                                          const uint64_t *__restrict__ keys, TieArgs a) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t cont_tag = (uint32_t)a.prefix_len + 8;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < count; r += stride) {
        const RunEntry e = runs[r];
        const uint64_t k = keys[run_base[r]];
        if (window_tag(k) == cont_tag) push_run(a, e.start, e.len, e.depth + 1);
    }
}

}  // namespace

// Sorted-input test, second half: each queued adjacent pair (equal order
// keys, not both exact) compared in full; any pair out of order makes the
// input unsorted.
__global__ void pairs_ordered_kernel(const uint8_t *__restrict__ bytes, const uint64_t *__restrict__ offsets,
                                     const uint64_t *__restrict__ pairs, uint64_t count, DevFlags *flags) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const uint64_t p = pairs[i];
        const uint64_t a0 = offsets[p], a1 = offsets[p + 1], b1 = offsets[p + 2];
        bad |= compare_from(bytes + a0, a1 - a0, bytes + a1, b1 - a1, 0) > 0;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&flags->descent, 1u);
}

cudaError_t launch_pairs_ordered(const uint8_t *bytes, const uint64_t *offsets, const uint64_t *pairs,
                                 uint64_t count, DevFlags *flags, int num_sms, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64((count + 255) / 256, (uint64_t)num_sms * 8);
    pairs_ordered_kernel<<<grid, 256, 0, s>>>(bytes, offsets, pairs, count, flags);
    return cudaGetLastError();
}

cudaError_t launch_tie_detect(const TieArgs &a, TieMode mode, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const unsigned tiles = (unsigned)((a.n + kTieTile - 1) / kTieTile);
    switch (mode) {
        case kTieKeyFlag:
            if (a.segs == nullptr && a.runs == nullptr) {
                const uint64_t blocks = (a.n + kHeadThreads * kHeadItems - 1) / (kHeadThreads * kHeadItems);
                tie_heads_kernel<<<(unsigned)umin64(blocks, 152ull * 8), kHeadThreads, 0, s>>>(a);
            } else {
                tie_detect_kernel<kTieKeyFlag><<<tiles, kTieThreads, kTieSmem, s>>>(a);
            }
            break;
        case kTieValFlag: tie_detect_kernel<kTieValFlag><<<tiles, kTieThreads, kTieSmem, s>>>(a); break;
        case kTiePacked:
            if (a.bits == nullptr || a.pack_bits <= 0 || a.pack_bits > 63 || a.segs != nullptr)
                return cudaErrorInvalidValue;
            tie_detect_kernel<kTiePacked><<<tiles, kTieThreads, kTieSmem, s>>>(a);
            break;
        default: tie_detect_kernel<kTieRefine><<<tiles, kTieThreads, kTieSmem, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_small_runs(const uint8_t *bytes, const uint64_t *offsets, void *perm, int perm_u64,
                              const RunEntry *q, const unsigned long long *qcount, uint64_t first, uint64_t cap,
                              uint64_t perm_n, Instances inst, int prefix_len, int num_sms, cudaStream_t s,
                              DevFlags *dirty) {
    const unsigned grid = (unsigned)num_sms * 8;
    if (perm_u64) {
        pair_runs_kernel<uint64_t><<<grid, 256, 0, s>>>(bytes, offsets, static_cast<uint64_t *>(perm), q, qcount,
                                                        first, cap, perm_n, inst, prefix_len, dirty);
        small_runs_kernel<uint64_t><<<grid, 256, 0, s>>>(bytes, offsets, static_cast<uint64_t *>(perm), q,
                                                         qcount, first, cap, perm_n, inst, prefix_len, dirty);
    } else {
        pair_runs_kernel<uint32_t><<<grid, 256, 0, s>>>(bytes, offsets, static_cast<uint32_t *>(perm), q, qcount,
                                                        first, cap, perm_n, inst, prefix_len, dirty);
        small_runs_kernel<uint32_t><<<grid, 256, 0, s>>>(bytes, offsets, static_cast<uint32_t *>(perm), q,
                                                         qcount, first, cap, perm_n, inst, prefix_len, dirty);
    }
    return cudaGetLastError();
}

cudaError_t launch_distinct_large(const uint8_t *bytes, const uint64_t *offsets, const void *perm, int perm_u64,
                                  const RunEntry *q, const unsigned long long *qcount, uint64_t cap,
                                  uint64_t perm_n, Instances inst, int prefix_len, uint32_t *diff,
                                  unsigned long long *base, RunEntry *q_out, unsigned long long *qcount_out,
                                  uint64_t cap_out, DevFlags *flags, unsigned int *done2, int num_sms,
                                  cudaStream_t s) {
    const unsigned grid = (unsigned)num_sms * 2;
    if (perm_u64) {
        distinct_sample_kernel<uint64_t><<<grid, 256, 0, s>>>(bytes, offsets, static_cast<const uint64_t *>(perm), q,
                                                              qcount, cap, perm_n, inst, prefix_len, diff, base, done2);
        distinct_full_kernel<uint64_t><<<grid * 4, 256, 0, s>>>(bytes, offsets, static_cast<const uint64_t *>(perm),
                                                                q, qcount, cap, inst, prefix_len, base, diff, q_out,
                                                                qcount_out, cap_out, flags, done2 + 1);
    } else {
        distinct_sample_kernel<uint32_t><<<grid, 256, 0, s>>>(bytes, offsets, static_cast<const uint32_t *>(perm), q,
                                                              qcount, cap, perm_n, inst, prefix_len, diff, base, done2);
        distinct_full_kernel<uint32_t><<<grid * 4, 256, 0, s>>>(bytes, offsets, static_cast<const uint32_t *>(perm),
                                                                q, qcount, cap, inst, prefix_len, base, diff, q_out,
                                                                qcount_out, cap_out, flags, done2 + 1);
    }
    return cudaGetLastError();
}

cudaError_t launch_medium_runs(const uint8_t *bytes, const uint64_t *offsets, void *perm, int perm_u64,
                               const RunEntry *q, const unsigned long long *qcount, uint64_t first, uint64_t cap,
                               uint64_t perm_n, Instances inst, int prefix_len, int num_sms, cudaStream_t s,
                               DevFlags *dirty) {
    const unsigned grid = (unsigned)num_sms * 2;
    if (perm_u64)
        medium_runs_kernel<uint64_t><<<grid, kMedThreads, 0, s>>>(bytes, offsets, static_cast<uint64_t *>(perm),
                                                                  q, qcount, first, cap, perm_n, inst, prefix_len, dirty);
    else
        medium_runs_kernel<uint32_t><<<grid, kMedThreads, 0, s>>>(bytes, offsets, static_cast<uint32_t *>(perm),
                                                                  q, qcount, first, cap, perm_n, inst, prefix_len, dirty);
    return cudaGetLastError();
}

cudaError_t launch_copies_filter(const uint8_t *bytes, const uint64_t *offsets, const void *perm, int perm_u64,
                                 RunEntry *q, const unsigned long long *qcount, uint64_t cap, uint64_t perm_n,
                                 Instances inst, int prefix_len, int num_sms, cudaStream_t s) {
    const unsigned grid = (unsigned)num_sms * 8;
    if (perm_u64)
        copies_filter_kernel<uint64_t><<<grid, kCopiesThreads, 0, s>>>(bytes, offsets, static_cast<const uint64_t *>(perm),
                                                                       q, qcount, cap, perm_n, inst, prefix_len);
    else
        copies_filter_kernel<uint32_t><<<grid, kCopiesThreads, 0, s>>>(bytes, offsets, static_cast<const uint32_t *>(perm),
                                                                       q, qcount, cap, perm_n, inst, prefix_len);
    return cudaGetLastError();
}

cudaError_t launch_run_scan(const RunEntry *runs, uint64_t count, unsigned long long *run_base,
                            cudaStream_t s) {
    run_scan_kernel<<<1, 1024, 0, s>>>(runs, count, run_base);
    return cudaGetLastError();
}

cudaError_t launch_refine_keys_win(const uint8_t *bytes, const uint64_t *offsets, const void *perm, int perm_u64,
                                   const RunEntry *runs, uint64_t count, const unsigned long long *run_base,
                                   uint64_t total, Instances inst, int prefix_len, const uint64_t *win,
                                   uint32_t win_depth, uint64_t *keys, uint32_t *segs, uint32_t *vals,
                                   DevFlags *flags, cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64((total + 255) / 256, 152ull * 16);
    if (perm_u64)
        refine_keys_kernel<uint64_t><<<grid, 256, 0, s>>>(bytes, offsets, static_cast<const uint64_t *>(perm),
                                                          runs, count, run_base, total, inst, prefix_len, win,
                                                          win_depth, keys, segs, vals, flags);
    else
        refine_keys_kernel<uint32_t><<<grid, 256, 0, s>>>(bytes, offsets, static_cast<const uint32_t *>(perm),
                                                          runs, count, run_base, total, inst, prefix_len, win,
                                                          win_depth, keys, segs, vals, flags);
    return cudaGetLastError();
}

cudaError_t launch_refine_keys(const uint8_t *bytes, const uint64_t *offsets, const void *perm, int perm_u64,
                               const RunEntry *runs, uint64_t count, const unsigned long long *run_base,
                               uint64_t total, Instances inst, int prefix_len, uint64_t *keys, uint32_t *segs,
                               uint32_t *vals, DevFlags *flags, cudaStream_t s) {
    return launch_refine_keys_win(bytes, offsets, perm, perm_u64, runs, count, run_base, total, inst, prefix_len,
                                  nullptr, 0, keys, segs, vals, flags, s);
}

cudaError_t launch_window_dense(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, int prefix_len,
                                uint32_t depth, uint64_t *win, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64((n + 255) / 256, (uint64_t)num_sms * 8);
    window_dense_kernel<<<grid, 256, 0, s>>>(bytes, offsets, n, prefix_len, depth, win);
    return cudaGetLastError();
}

cudaError_t launch_push_constant_runs(const RunEntry *runs, uint64_t count, const unsigned long long *run_base,
                                      const uint64_t *keys, int prefix_len, RunEntry *q_small,
                                      RunEntry *q_medium, RunEntry *q_large, uint64_t cap_small,
                                      uint64_t cap_medium, uint64_t cap_large, int q_large_id,
                                      uint64_t perm_n, DevFlags *flags, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    TieArgs a{};
    a.prefix_len = prefix_len;
    a.q_small = q_small;
    a.q_medium = q_medium;
    a.q_large = q_large;
    a.cap_small = cap_small;
    a.cap_medium = cap_medium;
    a.cap_large = cap_large;
    a.q_large_id = q_large_id;
    a.perm_n = perm_n;
    a.flags = flags;
    const unsigned grid = (unsigned)umin64((count + 255) / 256, 1024);
    push_constant_runs_kernel<<<grid, 256, 0, s>>>(runs, count, run_base, keys, a);
    return cudaGetLastError();
}

}  // namespace hs
