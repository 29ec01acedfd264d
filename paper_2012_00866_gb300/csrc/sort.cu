// Step 2: stable LSD radix sort of (code, index) pairs -- the GPU replacement
// for the paper's introsort with "object swap" (Section 3.1 Step 2, Algorithm
// 1): moving the index with its code is the object swap; stability makes the
// result unique.
//
// Each pass is a single "onesweep" kernel (Adinets and Merrill, 2022): the
// global digit offsets come from histograms computed up front (fused into the
// encoder), each CTA ranks a tile of keys with warp-private digit counters
// (lanes with equal digits found by the warp match instruction, or by nine
// ballots where the warp holds many distinct digits), publishes its per-digit
// counts, scatters the tile into shared memory in digit order, resolves its
// global prefix by decoupled look-back over earlier tiles, and writes the
// tile out so that runs of equal digits leave as coalesced stores.  Digits
// are 9 bits wide (512 bins, one per thread in the per-digit phase); 512
// threads at <= 64 registers keep two CTAs (32 warps) resident per SM, with
// 12 keys a thread (8 when a segment id moves too).  The pairs are either a
// 64-bit key plus a 32-bit payload or, when the code and the string index
// fit one word together, that word alone.  Tile ids come from an atomic
// counter, so every tile a CTA waits on is already running; each wait is
// bounded and reports kErrTimeout.
#include <type_traits>

#include "hs_internal.h"

namespace hs {
namespace {

constexpr int kThreads = kSortThreads;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = kSortTile / kThreads;   // keys per thread
constexpr int kDpt = kBins / kThreads;         // digits per thread in the per-digit phases
constexpr int kMinBlocks = kSortMinBlocks;
constexpr int kLbBatch = 4;                    // look-back words per digit per round trip
// Per-item ranks among the warp's earlier items with the same digit are
// below 32 * items; they are packed 4 (8-bit) or 2 (16-bit) to a register.
static_assert(kDpt >= 1 && kDpt * kThreads == kBins, "digits must spread evenly over the threads");
static_assert(kItems * kThreads == kSortTile, "tile must be whole threads");
// Keys per thread by element layout.  Larger tiles mean fewer look-backs
// per key; (key, index) pairs and packed words take 12 (6144-key tiles, two
// CTAs per SM in shared memory); with a segment id as well a 6144-key tile
// would leave one CTA per SM, so segmented passes keep 8.  Look-back words
// are sized for kSortTile, the smallest tile.
constexpr int kWideItems = 12;
constexpr int items_for(bool has_seg) { return has_seg ? kItems : kWideItems; }
static_assert(kWideItems * kThreads >= kSortTile, "look-back words are sized for tiles of kSortTile keys");

// Bounded-wait test support (hs_test_bounded_waits): the look-back's poll
// budget, and the id of a tile whose look-back words are never published (a
// flag that nothing sets; -1: none).  Both are per device.
__device__ unsigned int g_spin_limit = kSpinLimit;
__device__ long long g_withhold_tile = -1;

// Exclusive scan of one u32 per thread over the block.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t wsum = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wsum += w < warp ? s_warp[w] : 0u;
    __syncthreads();
    return wsum + x - v;
}

// Shared-memory layout of one onesweep CTA (the dynamic part holds the tile).
struct OsShared {
    uint64_t *keys;
    uint32_t *vals;
    uint32_t *segs;
    uint32_t *whist;                 // kWarps x kBins warp counts, then warp offsets
    unsigned long long *gbase;       // per digit: global start minus tile-local start
    uint32_t *scan;                  // kWarps
    uint32_t *dstart;                // kBins tile-local digit starts
};

// One tile.  FULL: the tile holds TILE elements, so no element needs a
// bounds test and the write-out runs as ITEMS unrolled rounds; the last,
// partial tile takes the general form.  PACKED: each element is one word
// (key << pack_bits) | index; no payload is loaded, staged or stored.
template <bool FULL, bool HAS_SEG, bool DIGIT_SEG, bool SYNTH, int OUT, bool PACKED, int ITEMS>
__device__ __forceinline__ void onesweep_tile(const OnesweepArgs &a, const OsShared &s, const uint64_t tile) {
    constexpr int TILE = kThreads * ITEMS;
    constexpr int RBITS = (32 * ITEMS <= 256 && !SYNTH) ? 8 : 16;  // rank bits (ranks < 32 * ITEMS; SYNTH: + a flag)
    constexpr int RPR = 32 / RBITS;
    constexpr uint32_t RMASK = (1u << (SYNTH ? RBITS - 1 : RBITS)) - 1;  // SYNTH: top bit is the flag
    static_assert(ITEMS % 4 == 0, "tile must be whole groups of four items");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t n = a.n;
    const uint64_t tile_base = tile * TILE;
    const int shift = a.shift;
    const unsigned mask = a.mask;

    // Warp-striped load: warp w owns elements [w*32*ITEMS, (w+1)*32*ITEMS)
    // of the tile, item k of lane l is element w*32*ITEMS + k*32 + l, so
    // processing items in k order visits the warp's elements in input order
    // (stability).  Synthesised payloads (the element's own index) are made
    // at the scatter instead of being held; their not-exact bit waits in the
    // top bit of the item's 16-bit rank slot (ranks stay below 32 * ITEMS).
    static_assert(!SYNTH || (RBITS == 16 && 32 * ITEMS < (1 << 15)), "synthesised flags ride in 16-bit rank slots");
    const uint64_t wbase = tile_base + (uint64_t)warp * 32 * ITEMS;
    // elements of this warp inside the input (all of them in a full tile)
    const uint32_t wcount = FULL ? 32u * ITEMS : (uint32_t)(n > wbase ? umin64(n - wbase, 32u * ITEMS) : 0);
    uint64_t key[ITEMS];
    uint32_t val[ITEMS];
    uint32_t seg[ITEMS];
    uint32_t rankp[ITEMS / RPR] = {};
    {
        const uint64_t *kin = a.keys_in + wbase + lane;
        const uint32_t *vin = PACKED || SYNTH ? nullptr : a.vals_in + wbase + lane;
        const uint32_t *sin = HAS_SEG ? a.segs_in + wbase + lane : nullptr;
        const uint32_t *fin = SYNTH ? a.flag_bits + (wbase >> 5) : nullptr;  // one word per item, warp-uniform
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const bool valid = FULL || (uint32_t)(k * 32 + lane) < wcount;
            key[k] = valid ? kin[k * 32] : 0;
            val[k] = (PACKED || SYNTH || !valid) ? 0u : vin[k * 32];
            if (SYNTH && valid && a.flag_bits)
                rankp[k / RPR] |= ((fin[k] >> lane) & 1u) << (RBITS * (k % RPR) + RBITS - 1);
            seg[k] = (HAS_SEG && valid) ? sin[k * 32] : 0;
        }
    }
    auto digit_of = [&](int k) -> unsigned {
        return DIGIT_SEG ? ((seg[k] >> shift) & mask) : (unsigned)((key[k] >> shift) & mask);
    };

    // Ranking, four items at a time: the peer masks of the four (lanes
    // with the same digit) are independent and issue back to back; then for
    // each item the lowest lane of every equal-digit group (leader) advances
    // the warp's count by the group size with one shared atomic (the
    // __syncwarp orders the groups of consecutive items on the same
    // counter), and the counts before the adds are broadcast to the groups
    // last.  The masks come from the match instruction, or from ballots when
    // the warp's first item holds many distinct digits (prefer_ballots);
    // each form is unrolled on its own, with no branch between the groups.
    uint32_t *my_hist = s.whist + warp * kBins;
    unsigned peers0 = 0;
    auto rank_items = [&](auto by_ballots) {
        constexpr bool BALLOTS = decltype(by_ballots)::value;
#pragma unroll
        for (int g = 0; g < ITEMS; g += 4) {
            unsigned peers[4], before[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = g + q;
                if (FULL && k == 0) {
                    peers[q] = peers0;
                } else if (BALLOTS) {
                    peers[q] = match_by_ballots(digit_of(k));
                } else if (FULL) {
                    peers[q] = __match_any_sync(kFull, digit_of(k));
                } else {
                    const bool valid = (uint32_t)(k * 32 + lane) < wcount;
                    peers[q] = match_digit(digit_of(k), __ballot_sync(kFull, valid));
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = g + q;
                const bool valid = FULL || (uint32_t)(k * 32 + lane) < wcount;
                before[q] = 0;
                if (valid && lane == __ffs(peers[q]) - 1)
                    before[q] = atomicAdd(&my_hist[digit_of(k)], (unsigned)__popc(peers[q]));
                __syncwarp();
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = g + q;
                const bool valid = FULL || (uint32_t)(k * 32 + lane) < wcount;
                const int leader = valid ? __ffs(peers[q]) - 1 : lane;
                const unsigned b = __shfl_sync(kFull, before[q], leader);
                rankp[k / RPR] |= (b + __popc(peers[q] & lanemask_lt())) << (RBITS * (k % RPR));
            }
        }
    };
    if constexpr (FULL) {
        peers0 = __match_any_sync(kFull, digit_of(0));  // also item 0's mask
        if (prefer_ballots(peers0))
            rank_items(std::true_type{});
        else
            rank_items(std::false_type{});
    } else {
        rank_items(std::false_type{});  // the last, partial tile
    }
    __syncthreads();

    // Thread t owns digits t*kDpt .. t*kDpt + kDpt - 1: their tile counts
    // first, then (after the tile-local digit starts are known) each warp's
    // start for the digit inside the staged tile in place of its count.
    uint32_t total[kDpt];
#pragma unroll
    for (int j = 0; j < kDpt; ++j) total[j] = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
#pragma unroll
        for (int j = 0; j < kDpt; ++j) total[j] += s.whist[w * kBins + tid * kDpt + j];
    }
    uint64_t *lb = a.lookback + tile * kBins;
    const uint32_t epoch = a.epoch;
    const bool publish = (long long)tile != g_withhold_tile;
    // Publish this tile's counts as early as possible: later tiles can sum
    // past them before its global prefix is known.
#pragma unroll
    for (int j = 0; j < kDpt; ++j)
        if (publish)
            st_relaxed(&lb[tid * kDpt + j], lb_word(epoch, tile == 0 ? kLbInclusive : kLbAggregate, total[j]));

    // Tile-local digit starts and the shared-memory scatter need no global
    // prefix, so they run before the look-back, which then overlaps with
    // nothing but its own loads.
    uint32_t mine = 0;
#pragma unroll
    for (int j = 0; j < kDpt; ++j) mine += total[j];
    uint32_t dstart[kDpt];
    dstart[0] = block_exclusive_scan(mine, s.scan);
#pragma unroll
    for (int j = 1; j < kDpt; ++j) dstart[j] = dstart[j - 1] + total[j - 1];
    {
        uint32_t run[kDpt];
#pragma unroll
        for (int j = 0; j < kDpt; ++j) run[j] = dstart[j];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
#pragma unroll
            for (int j = 0; j < kDpt; ++j) {
                uint32_t *h = s.whist + w * kBins + tid * kDpt + j;
                const uint32_t c = *h;
                *h = run[j];
                run[j] += c;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        if (FULL || (uint32_t)(k * 32 + lane) < wcount) {
            const unsigned d = digit_of(k);
            const uint32_t r = (rankp[k / RPR] >> (RBITS * (k % RPR))) & RMASK;
            const uint32_t p = my_hist[d] + r;
            s.keys[p] = key[k];
            if (SYNTH) {
                const uint32_t bit = (rankp[k / RPR] >> (RBITS * (k % RPR) + RBITS - 1)) & 1u;
                s.vals[p] = ((uint32_t)wbase + (uint32_t)(k * 32 + lane)) | (bit << 31);
            } else if (!PACKED) {
                s.vals[p] = val[k];
            }
            if (HAS_SEG) s.segs[p] = seg[k];
        }
    }

    // Look-back for the thread's digits, walked together: per round trip
    // kLbBatch earlier tiles' words per digit; add aggregates until an
    // inclusive prefix; stop at the first word not yet written and poll it.
    uint64_t prefix[kDpt];
#pragma unroll
    for (int j = 0; j < kDpt; ++j) prefix[j] = 0;
    if (tile > 0) {
        int64_t t[kDpt];
        bool done[kDpt];
#pragma unroll
        for (int j = 0; j < kDpt; ++j) {
            t[j] = (int64_t)tile - 1;
            done[j] = false;
        }
        uint32_t spins = 0;
        const uint32_t spin_limit = g_spin_limit;
        while (true) {
            bool all_done = true;
#pragma unroll
            for (int j = 0; j < kDpt; ++j) all_done &= done[j];
            if (all_done) break;
            uint64_t v[kDpt][kLbBatch];
#pragma unroll
            for (int j = 0; j < kDpt; ++j)
#pragma unroll
                for (int i = 0; i < kLbBatch; ++i)
                    v[j][i] = (!done[j] && t[j] - i >= 0)
                                  ? ld_relaxed(&a.lookback[(uint64_t)(t[j] - i) * kBins + tid * kDpt + j])
                                  : 0;
            bool progress = false;
#pragma unroll
            for (int j = 0; j < kDpt; ++j) {
                if (done[j]) continue;
                bool stalled = false, incl = false;
                int used = 0;
#pragma unroll
                for (int i = 0; i < kLbBatch; ++i) {
                    if (incl || stalled || t[j] - i < 0) continue;
                    if ((uint32_t)(v[j][i] >> 58) != epoch) {
                        stalled = true;
                        continue;
                    }
                    prefix[j] += v[j][i] & kLbValueMask;
                    used = i + 1;
                    incl = (v[j][i] & (3ull << 56)) == kLbInclusive;
                }
                t[j] -= used;
                done[j] = incl || t[j] < 0;
                progress |= used > 0;
            }
            if (!progress) {
                if (++spins > spin_limit) {
                    atomicOr(&a.flags->error, kErrTimeout);
                    break;
                }
                if (spins > 8) __nanosleep(32);
            }
        }
#pragma unroll
        for (int j = 0; j < kDpt; ++j)
            if (publish) st_relaxed(&lb[tid * kDpt + j], lb_word(epoch, kLbInclusive, prefix[j] + total[j]));
    }
#pragma unroll
    for (int j = 0; j < kDpt; ++j)
        s.gbase[tid * kDpt + j] = a.bucket_base[tid * kDpt + j] + prefix[j] - dstart[j];
    __syncthreads();

    // Write-out in tile order: element i of the staged tile goes to its
    // digit's global start plus i, so equal digits leave as runs.
    // KEYS (compile time): the keys go out too (keys_out set).
    auto emit = [&](int i, uint64_t k, uint32_t sg, auto keys_tag) {
        constexpr bool KEYS = decltype(keys_tag)::value;
        const unsigned d = DIGIT_SEG ? ((sg >> shift) & mask) : (unsigned)((k >> shift) & mask);
        const uint64_t pos = s.gbase[d] + (uint64_t)i;
        if (pos >= n) {
            atomicOr(&a.flags->error, kErrInternal);
            return;
        }
        if (PACKED) {
            const uint64_t idx = k & ((1ull << a.pack_bits) - 1);
            if (OUT == kOutVals || KEYS) a.keys_out[pos] = k;
            if (OUT == kOutPerm32)
                static_cast<uint32_t *>(a.vals_out)[pos] = (uint32_t)idx;
            else if (OUT == kOutPerm64)
                static_cast<uint64_t *>(a.vals_out)[pos] = idx;
            return;
        }
        if (KEYS) a.keys_out[pos] = k;
        if (HAS_SEG) a.segs_out[pos] = sg;
        const uint32_t v = s.vals[i];
        if (OUT == kOutVals)
            static_cast<uint32_t *>(a.vals_out)[pos] = v;
        else if (OUT == kOutPerm32)
            static_cast<uint32_t *>(a.vals_out)[pos] = v & kIdxMask;
        else
            static_cast<uint64_t *>(a.vals_out)[pos] = (uint64_t)(v & kIdxMask);
    };
    if (FULL) {
        // every thread owns ITEMS elements: their shared loads issue together
        uint64_t k[ITEMS];
        uint32_t sg[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            k[j] = s.keys[j * kThreads + tid];
            sg[j] = HAS_SEG ? s.segs[j * kThreads + tid] : 0;
        }
        auto emit_all = [&](auto keys_tag) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) emit(j * kThreads + tid, k[j], sg[j], keys_tag);
        };
        if (a.keys_out)
            emit_all(std::true_type{});
        else
            emit_all(std::false_type{});
    } else {
        const int cnt = (int)umin64(TILE, n - tile_base);
        for (int i = tid; i < cnt; i += kThreads) {
            if (a.keys_out)
                emit(i, s.keys[i], HAS_SEG ? s.segs[i] : 0, std::true_type{});
            else
                emit(i, s.keys[i], HAS_SEG ? s.segs[i] : 0, std::false_type{});
        }
    }
}

template <bool HAS_SEG, bool DIGIT_SEG, bool SYNTH, int OUT, bool PACKED, int ITEMS>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
onesweep_kernel(const OnesweepArgs a) {
    constexpr int TILE = kThreads * ITEMS;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_scan[kWarps];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_dstart[kBins];
    OsShared s;
    s.keys = reinterpret_cast<uint64_t *>(smem);
    s.vals = reinterpret_cast<uint32_t *>(s.keys + TILE);
    s.segs = s.vals + (PACKED ? 0 : TILE);
    s.whist = s.segs + (HAS_SEG ? TILE : 0);
    s.gbase = reinterpret_cast<unsigned long long *>(s.whist + kWarps * kBins);
    s.scan = s_scan;
    s.dstart = s_dstart;

    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    for (int i = tid; i < kWarps * kBins; i += kThreads) s.whist[i] = 0;
    __syncthreads();
    const uint64_t tile = s_tile;
    if ((tile + 1) * TILE <= a.n)
        onesweep_tile<true, HAS_SEG, DIGIT_SEG, SYNTH, OUT, PACKED, ITEMS>(a, s, tile);
    else
        onesweep_tile<false, HAS_SEG, DIGIT_SEG, SYNTH, OUT, PACKED, ITEMS>(a, s, tile);
}

size_t onesweep_smem(bool has_seg, bool packed, int items) {
    const size_t tile = (size_t)kThreads * items;
    return tile * 8 + (packed ? 0 : tile * 4) + (has_seg ? tile * 4 : 0) + (size_t)kWarps * kBins * 4 +
           (size_t)kBins * 8;
}

template <bool HAS_SEG, bool DIGIT_SEG, bool SYNTH, int OUT, bool PACKED, int ITEMS>
cudaError_t launch_os_shape(const OnesweepArgs &a, cudaStream_t s) {
    constexpr int items = ITEMS;
    auto kern = onesweep_kernel<HAS_SEG, DIGIT_SEG, SYNTH, OUT, PACKED, items>;
    const size_t smem = onesweep_smem(HAS_SEG, PACKED, items);
    static bool configured = false;  // attribute is per function, idempotent
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const uint64_t tiles = (a.n + kThreads * items - 1) / (kThreads * items);
    kern<<<(unsigned)tiles, kThreads, smem, s>>>(a);  // one CTA per tile
    return cudaGetLastError();
}

// Keys per thread: segmented passes have one shape (8); the others run with
// 8 or 12 (items == 0: the default, 12), the choice of the tile-shape tuner.
template <bool HAS_SEG, bool DIGIT_SEG, bool SYNTH, int OUT, bool PACKED = false>
cudaError_t launch_os(const OnesweepArgs &a, cudaStream_t s, int items) {
    if constexpr (HAS_SEG) {
        return launch_os_shape<HAS_SEG, DIGIT_SEG, SYNTH, OUT, PACKED, kItems>(a, s);
    } else {
        if (items == kItems) return launch_os_shape<HAS_SEG, DIGIT_SEG, SYNTH, OUT, PACKED, kItems>(a, s);
        return launch_os_shape<HAS_SEG, DIGIT_SEG, SYNTH, OUT, PACKED, kWideItems>(a, s);
    }
}

// ---- up-front histograms -------------------------------------------------

constexpr int kHistThreads = 512;

template <bool HAS_SEG>
__global__ void __launch_bounds__(kHistThreads)
histogram_kernel(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ segs,
                 uint64_t n, unsigned long long *__restrict__ hist) {
    constexpr int P = HAS_SEG ? kHistPasses : kKeyPasses;
    extern __shared__ uint32_t s_hist[];
    for (int i = threadIdx.x; i < P * kBins; i += kHistThreads) s_hist[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * kHistThreads;
    const uint64_t n_round = (n + 31) & ~31ull;  // whole warps iterate together
    for (uint64_t i = (uint64_t)blockIdx.x * kHistThreads + threadIdx.x; i < n_round; i += stride) {
        const bool valid = i < n;
        const uint64_t k = valid ? keys[i] : 0;
#pragma unroll
        for (int p = 0; p < kKeyPasses; ++p)
            hist_add(s_hist + p * kBins, (unsigned)((k >> digit_shift(p)) & digit_mask(p)), valid);
        if (HAS_SEG) {
            const uint32_t sg = valid ? segs[i] : 0;
#pragma unroll
            for (int p = kKeyPasses; p < kHistPasses; ++p)
                hist_add(s_hist + p * kBins, (sg >> digit_shift(p)) & digit_mask(p), valid);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P * kBins; i += kHistThreads)
        if (s_hist[i]) atomicAdd(&hist[i], (unsigned long long)s_hist[i]);
}

// ---- pass plan -------------------------------------------------------------

// One CTA per pass: the histograms are independent.
__global__ void __launch_bounds__(kBins)
plan_kernel(const unsigned long long *__restrict__ hist, int npass, uint64_t n,
            unsigned long long *__restrict__ bucket_base, DevFlags *flags) {
    __shared__ unsigned long long s_warp[kBins / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int p = blockIdx.x; p < npass; p += gridDim.x) {
        const unsigned long long c = hist[p * kBins + tid];
        unsigned long long x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        unsigned long long wsum = 0;
        for (int w = 0; w < warp; ++w) wsum += s_warp[w];
        bucket_base[p * kBins + tid] = wsum + x - c;
        const int all_in_one = __syncthreads_or(c == n);
        if (tid == 0) flags->active[p] = (n > 1 && !all_in_one) ? 1u : 0u;
        __syncthreads();
    }
}

constexpr int kSegThreads = 512;

__global__ void __launch_bounds__(kSegThreads)
seg_fill_kernel(const uint64_t *__restrict__ seg_offsets, uint64_t num_segs, uint64_t n,
                const uint32_t *__restrict__ flag_bits, uint32_t *__restrict__ segs,
                uint32_t *__restrict__ vals, unsigned long long *__restrict__ hist, DevFlags *flags) {
    __shared__ uint32_t s_hist[kSegPasses * kBins];
    for (int i = threadIdx.x; i < kSegPasses * kBins; i += kSegThreads) s_hist[i] = 0;
    __syncthreads();
    bool bad = false;
    const uint64_t stride = (uint64_t)gridDim.x * kSegThreads;
    const uint64_t n_round = (n + 31) & ~31ull;  // whole warps iterate together
    for (uint64_t i = (uint64_t)blockIdx.x * kSegThreads + threadIdx.x; i < n_round; i += stride) {
        const bool valid = i < n;
        uint64_t lo = 0;
        if (valid) {
            uint64_t hi = num_segs;  // seg_offsets[lo] <= i < seg_offsets[hi]
            while (hi - lo > 1) {
                const uint64_t mid = (lo + hi) >> 1;
                if (seg_offsets[mid] <= i) lo = mid; else hi = mid;
            }
            const uint64_t local = i - seg_offsets[lo];
            bad |= local > kIdxMask;
            const uint32_t bit = flag_bits ? ((flag_bits[i >> 5] >> (i & 31)) & 1u) : 0u;
            segs[i] = (uint32_t)lo;
            vals[i] = ((uint32_t)local & kIdxMask) | (bit << 31);
        }
#pragma unroll
        for (int p = 0; p < kSegPasses; ++p)
            hist_add(s_hist + p * kBins, (uint32_t)(lo >> digit_shift(kKeyPasses + p)) & (kBins - 1), valid);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSegPasses * kBins; i += kSegThreads)
        if (s_hist[i]) atomicAdd(&hist[kKeyPasses * kBins + i], (unsigned long long)s_hist[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&flags->error, kErrInternal);
}

__global__ void identity_kernel(const uint32_t *__restrict__ flag_bits, uint64_t n, void *out, int mode) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t bit = flag_bits ? ((flag_bits[i >> 5] >> (i & 31)) & 1u) : 0u;
        if (mode == kOutVals)
            static_cast<uint32_t *>(out)[i] = (uint32_t)i | (bit << 31);
        else if (mode == kOutPerm32)
            static_cast<uint32_t *>(out)[i] = (uint32_t)i;
        else
            static_cast<uint64_t *>(out)[i] = i;
    }
}

}  // namespace

cudaError_t launch_onesweep(const OnesweepArgs &a, bool has_seg, bool digit_seg, bool synth,
                            OutMode out, cudaStream_t s, int items) {
    if (items != 0 && items != kItems && items != kWideItems) return cudaErrorInvalidValue;
    if (a.n == 0) return cudaSuccess;
    if (a.pack_bits > 0) {
        if (has_seg || digit_seg || synth || a.pack_bits > 63) return cudaErrorInvalidValue;
        if (out == kOutVals && a.keys_out == nullptr) return cudaErrorInvalidValue;
        switch (out) {
            case kOutVals: return launch_os<false, false, false, kOutVals, true>(a, s, items);
            case kOutPerm32: return launch_os<false, false, false, kOutPerm32, true>(a, s, items);
            default: return launch_os<false, false, false, kOutPerm64, true>(a, s, items);
        }
    }
    if (has_seg) {
        if (synth || out == kOutPerm64) return cudaErrorInvalidValue;
        if (out == kOutPerm32)
            return digit_seg ? launch_os<true, true, false, kOutPerm32>(a, s, items)
                             : launch_os<true, false, false, kOutPerm32>(a, s, items);
        return digit_seg ? launch_os<true, true, false, kOutVals>(a, s, items)
                         : launch_os<true, false, false, kOutVals>(a, s, items);
    }
    if (digit_seg) return cudaErrorInvalidValue;
    if (synth) {
        switch (out) {
            case kOutVals: return launch_os<false, false, true, kOutVals>(a, s, items);
            case kOutPerm32: return launch_os<false, false, true, kOutPerm32>(a, s, items);
            default: return launch_os<false, false, true, kOutPerm64>(a, s, items);
        }
    }
    switch (out) {
        case kOutVals: return launch_os<false, false, false, kOutVals>(a, s, items);
        case kOutPerm32: return launch_os<false, false, false, kOutPerm32>(a, s, items);
        default: return launch_os<false, false, false, kOutPerm64>(a, s, items);
    }
}

cudaError_t set_wait_test(uint32_t spin_limit, long long withhold_tile) {
    const uint32_t lim = spin_limit ? spin_limit : kSpinLimit;
    cudaError_t e = cudaMemcpyToSymbol(g_spin_limit, &lim, sizeof(lim));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_withhold_tile, &withhold_tile, sizeof(withhold_tile));
}

cudaError_t launch_histogram(const uint64_t *keys, const uint32_t *segs, uint64_t n,
                             unsigned long long *hist, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + kHistThreads * 16 - 1) / (kHistThreads * 16);
    const unsigned grid = (unsigned)umin64(blocks, (uint64_t)num_sms * 2);
    if (segs) {
        const size_t smem = (size_t)kHistPasses * kBins * 4;
        static bool configured = false;
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(histogram_kernel<true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            configured = true;
        }
        histogram_kernel<true><<<grid, kHistThreads, smem, s>>>(keys, segs, n, hist);
    } else {
        const size_t smem = (size_t)kKeyPasses * kBins * 4;
        histogram_kernel<false><<<grid, kHistThreads, smem, s>>>(keys, nullptr, n, hist);
    }
    return cudaGetLastError();
}

cudaError_t launch_plan(const unsigned long long *hist, int npass, uint64_t n,
                        unsigned long long *bucket_base, DevFlags *flags, cudaStream_t s) {
    if (npass <= 0) return cudaSuccess;
    plan_kernel<<<(unsigned)npass, kBins, 0, s>>>(hist, npass, n, bucket_base, flags);
    return cudaGetLastError();
}

__global__ void validate_segments_kernel(const uint64_t *__restrict__ seg_offsets, uint64_t num_segs, uint64_t n,
                                         DevFlags *flags) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < num_segs; i += stride) {
        bad |= seg_offsets[i] > seg_offsets[i + 1];
        bad |= seg_offsets[i + 1] - seg_offsets[i] > kIdxMask;  // local indices are 31-bit
        if (i == 0) bad |= seg_offsets[0] != 0;
        if (i == num_segs - 1) bad |= seg_offsets[num_segs] != n;
    }
    if (bad) atomicOr(&flags->error, kErrOffsets);
}

cudaError_t launch_validate_segments(const uint64_t *seg_offsets, uint64_t num_segs, uint64_t n, DevFlags *flags,
                                     cudaStream_t s) {
    if (num_segs == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64((num_segs + 255) / 256, 4096);
    validate_segments_kernel<<<grid, 256, 0, s>>>(seg_offsets, num_segs, n, flags);
    return cudaGetLastError();
}

cudaError_t launch_seg_fill(const uint64_t *seg_offsets, uint64_t num_segs, uint64_t n,
                            const uint32_t *flag_bits, uint32_t *segs, uint32_t *vals,
                            unsigned long long *hist, DevFlags *flags, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + kSegThreads * 8 - 1) / (kSegThreads * 8);
    const unsigned grid = (unsigned)umin64(blocks, (uint64_t)num_sms * 4);
    seg_fill_kernel<<<grid, kSegThreads, 0, s>>>(seg_offsets, num_segs, n, flag_bits, segs, vals, hist, flags);
    return cudaGetLastError();
}

cudaError_t launch_identity(const uint32_t *flag_bits, uint64_t n, void *out, OutMode mode,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)umin64((n + 255) / 256, 4096);
    identity_kernel<<<grid, 256, 0, s>>>(flag_bits, n, out, (int)mode);
    return cudaGetLastError();
}

}  // namespace hs
