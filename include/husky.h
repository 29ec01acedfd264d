/*
 * husky.h -- C ABI of the GB300 Huskysort string-argsort library (libhusky.so).
 *
 * The method (Hillyard, Liaozheng, K R, "Huskysort", arXiv 2012.00866):
 *   Step 1  encode every element into a 64-bit order-preserving "husky code"
 *           (Section 3.1 Step 1; Algorithm 4 stringToLong; Section 4.3
 *           asciiToLong and its constants);
 *   Step 2  sort the codes, moving the elements with them (Section 3.1
 *           Step 2, the "object swap");
 *   Step 3  if the coding was not perfect, fix the remaining inversions by
 *           comparing the elements themselves (Section 3.1 Step 3,
 *           Algorithm 1; skipped when perfect, Section 3.4).
 * Here Step 2 is a stable LSD radix sort of (code, index) pairs and Step 3
 * only touches runs of equal codes, the only places inversions can remain
 * when the coder is order preserving (Section 3.2 with p restricted to ties).
 *
 * Data model (all entry points)
 *   d_bytes    device pointer to the concatenated string bytes.
 *   d_offsets  device pointer to n + 1 uint64 offsets, non-decreasing; string i
 *              is d_bytes[d_offsets[i] .. d_offsets[i+1]).  Bytes compare as
 *              unsigned; a proper prefix is smaller.
 *   Every pointer argument named d_* is device memory owned by the caller;
 *   the library never frees or retains it past the call.  h_* pointers are
 *   host memory.
 *   d_ws/ws_bytes  caller-owned device scratch of at least the size reported
 *              by hs_workspace_size (or hs_batched_workspace_size); its
 *              contents on entry are irrelevant and undefined on return.
 *   stream     a cudaStream_t (passed as void*; NULL = legacy default stream).
 *              All device work is enqueued on it.  The calls synchronise this
 *              stream internally (to read small device-side counters) and
 *              return only after all their work has finished, so the status
 *              they return is final.
 *
 * Errors: every entry point returns an hs_status; HS_OK is 0, errors are
 * negative.  hs_last_error() returns a message for the calling host thread's
 * most recent failure.  Device-side waits are bounded: a wait that gives up
 * reports HS_ERR_TIMEOUT; the library never traps or asserts on the device.
 */
#ifndef HUSKY_H
#define HUSKY_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HS_API __attribute__((visibility("default")))
#else
#define HS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HS_OK = 0,
    HS_ERR_INVALID_ARG = -1,  /* bad pointer, size, enum, or offsets       */
    HS_ERR_CODER_DOMAIN = -2, /* ASCII7 coder given a byte >= 0x80 in the
                                 first 9 bytes of a string, or the ALPHA
                                 coder an alphabet of more than 63 bytes    */
    HS_ERR_OOM = -3,          /* host allocation failed                     */
    HS_ERR_CUDA = -4,         /* a CUDA runtime call failed                 */
    HS_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up         */
    HS_ERR_INTERNAL = -6,     /* an internal consistency check failed       */
    HS_ERR_WORKSPACE = -7     /* ws_bytes smaller than required             */
} hs_status;

/* Coders (Algorithm 4 parameters).
 *   HS_CODER_ASCII7  bitWidth 7, maxLength 64/7 = 9, mask 0x7F (asciiToLong,
 *                    Section 4.3).  Order preserving only on bytes < 0x80.
 *   HS_CODER_BYTE8   bitWidth 8, maxLength 8, no mask: order preserving on
 *                    all bytes (this library's coder for arbitrary bytes).
 *                    UTF-16 text passed as big-endian bytes sorts in
 *                    code-unit order (a Java String's order), and this coder
 *                    is then the Unicode coder of Section 4.3 (unicodeToLong:
 *                    4 units x 16 bits) without its final >>> 1, which only
 *                    served Java's signed long compare.
 *   HS_CODER_ALPHA   byte-range coder, generalising the 5-bit and 6-bit
 *                    letter codings of Section 3.2: with lo / hi the smallest
 *                    / largest byte of bytes[offsets[0] .. offsets[n]), byte
 *                    c codes as c - lo + 1 (0 is the padding) in
 *                    w = ceil(log2(hi - lo + 2)) bits ('a'..'z': 5 bits,
 *                    'A'..'z': 6), for maxLength 8: a sort key of 8w + 1
 *                    bits.  Lowercase text: a 41-bit key, five 9-bit radix
 *                    passes where ASCII7 needs seven (and, for up to
 *                    2^(64 - 8w) strings, the code and the string's index
 *                    share one 64-bit word through the sort).  Order
 *                    preserving on all bytes; exact iff length <= 8.  Applies when the
 *                    range has at most 63 values (w <= 6), else
 *                    HS_ERR_CODER_DOMAIN.
 *   HS_CODER_AUTO    ALPHA when the range has at most 31 values (w <= 5, where
 *                    it saves radix passes), else ASCII7, re-encoding with
 *                    BYTE8 when any string has a byte >= 0x80 among its first
 *                    9 bytes. */
typedef enum { HS_CODER_AUTO = 0, HS_CODER_ASCII7 = 1, HS_CODER_BYTE8 = 2, HS_CODER_ALPHA = 3 } hs_coder;

/* Sort strategies for Step 2; both give the identical permutation.
 *   HS_MODE_PLAIN    LSD radix sort of the 64-bit sort keys (9-bit digits,
 *                    digits constant over all keys skipped).
 *   HS_MODE_LEARNED  a learned CDF model (RMI: FP32 1->32->32->1 root,
 *                    4096 linear leaves) trained on a 1% sample of the codes
 *                    picks a monotone bucket per code; the pairs are
 *                    partitioned by bucket and each bucket sorted by code;
 *                    buckets over 4096 keys that hold different codes go
 *                    through a segmented radix sort.  Runs as PLAIN when
 *                    n < 65536 or when the strings need the BYTE8 coder.
 *   HS_MODE_AUTO     the library's choice; currently HS_MODE_PLAIN: on every
 *                    measured workload the plain path is faster (2-3x on
 *                    zipf words and skewed strings) or within 1% (strings
 *                    with long shared prefixes).  Its workspace is the plain
 *                    mode's.
 */
typedef enum { HS_MODE_PLAIN = 0, HS_MODE_LEARNED = 1, HS_MODE_AUTO = 2 } hs_mode;

/* Index type of the output permutation. */
typedef enum { HS_U32 = 0, HS_U64 = 1 } hs_index_t;

/* Largest n accepted by hs_argsort (the internal payload keeps one flag bit
 * beside a 31-bit index). */
#define HS_MAX_N ((uint64_t)0x7FFFFFFF)

/* hs_encode -- Step 1 alone (Algorithms 2, 3 and 4).
 *   d_codes      out, device, n uint64: code of string i.
 *   h_all_exact  out, host, nullable: 1 if every string is exactly
 *                represented (length <= maxLength and, when non-empty, last
 *                byte != 0: "a" and "a\0" share a code), else 0 -- the
 *                paper's "perfect" flag (Algorithm 3).
 *   coder        hs_coder; with HS_CODER_AUTO the coder actually used is
 *                written to *h_coder_used when that pointer is non-NULL.
 * Returns HS_ERR_CODER_DOMAIN for HS_CODER_ASCII7 on bytes >= 0x80. */
HS_API hs_status hs_encode(const uint8_t *d_bytes, const uint64_t *d_offsets,
                    uint64_t n, int coder, uint64_t *d_codes,
                    int *h_all_exact, int *h_coder_used, void *d_ws,
                    size_t ws_bytes, void *stream);

/* hs_argsort -- Steps 1-3: the stable argsort of n strings.
 *   d_perm   out, device, n entries of uint32 (out_t = HS_U32) or uint64
 *            (HS_U64): d_perm[k] is the index of the k-th smallest string;
 *            equal strings appear in increasing index order.  This is the
 *            unique stable ascending argsort under unsigned-byte
 *            lexicographic order.
 *   mode     hs_mode; coder hs_coder.
 *   n        0 <= n <= HS_MAX_N; n = 0 is a no-op.
 * Plain mode also recognises an input already in order: right after Step 1
 * each string's code is compared with its predecessor's; without a descent
 * (and with the pairs of equal codes compared in full) the call writes the
 * identity permutation and skips Steps 2 and 3.  An unsorted input pays one
 * early-exit kernel for the test. */
HS_API hs_status hs_argsort(const uint8_t *d_bytes, const uint64_t *d_offsets,
                     uint64_t n, int mode, int coder, int out_t, void *d_perm,
                     void *d_ws, size_t ws_bytes, void *stream);

/* hs_argsort_batched -- many independent sorts in one call.
 *   d_seg_offsets  device, num_segs + 1 uint64 string-index boundaries:
 *                  instance s owns strings seg_offsets[s] ..
 *                  seg_offsets[s+1] - 1 (non-decreasing, last = n).
 *   d_perm         out, device, n uint32: for instance s, entries
 *                  d_perm[seg_offsets[s] .. seg_offsets[s+1]) hold the stable
 *                  argsort of that instance as LOCAL indices (0-based within
 *                  the instance).
 *   Each instance must hold fewer than 2^31 strings (HS_ERR_INVALID_ARG
 *   otherwise: at once when n > num_segs * (2^31 - 1), else from the device
 *   check of seg_offsets); n may exceed 2^32. */
HS_API hs_status hs_argsort_batched(const uint8_t *d_bytes, const uint64_t *d_offsets,
                             const uint64_t *d_seg_offsets, uint64_t num_segs,
                             uint64_t n, int coder, uint32_t *d_perm,
                             void *d_ws, size_t ws_bytes, void *stream);

/* hs_argsort_host -- hs_argsort on strings and a permutation in HOST memory
 * (the paper's setting: an array in the host's memory, sorted and returned
 * there).  The paper has no GPU transfer step; this entry point owns it.
 *   h_bytes, h_offsets  host (pinned for full speed; pageable works but the
 *              copies then block the calling thread): the data model above,
 *              with h_offsets[n] = total byte count.
 *   h_perm     out, host, n entries of uint32 / uint64 as in hs_argsort.
 *   d_ws       device workspace of hs_host_workspace_size(n, h_offsets[n],
 *              mode, out_t) bytes: the hs_argsort workspace followed by
 *              device copies of the bytes, the offsets and the permutation.
 * The offsets and bytes are copied in chunks of whole 1024-string tiles on a
 * second stream owned by the library; each chunk is encoded (Step 1) as soon
 * as it has arrived, so the encoder runs under the transfer.  Steps 2-3 run
 * on the device copies and the permutation is copied back into h_perm before
 * the call returns.  Chunk boundaries with decreasing offsets are rejected
 * (HS_ERR_INVALID_ARG) before any copy; the rest of the offsets are checked
 * on the device as in hs_argsort.  h_bytes, h_offsets and h_perm must not be
 * device memory (HS_ERR_INVALID_ARG). */
HS_API hs_status hs_argsort_host(const uint8_t *h_bytes, const uint64_t *h_offsets,
                                 uint64_t n, int mode, int coder, int out_t,
                                 void *h_perm, void *d_ws, size_t ws_bytes,
                                 void *stream);
/* Workspace needed by hs_argsort_host for n strings of total_bytes bytes. */
HS_API hs_status hs_host_workspace_size(uint64_t n, uint64_t total_bytes,
                                        int mode, int out_t, size_t *out);

/* hs_argsort_noalloc -- hs_argsort for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a deployment convenience.
 *
 * Who needs it: code that runs inside a host application which owns the
 * GPU's memory through its own pool and forbids side allocations (an engine
 * plug-in or user-defined function, for instance), code on a latency-critical
 * path where cudaMalloc's implicit device-wide synchronisation would stall
 * other streams, and code whose memory budget is fixed when it is loaded.
 * Such a caller can still pass its own inputs and output, but not a
 * workspace.
 *
 * Scratch comes from one static device array of HS_NOALLOC_SCRATCH_BYTES
 * (16 MiB) inside the library; every GPU on which the library is loaded holds
 * it until the process exits.  No cudaMalloc, cudaFree or other allocating
 * routine is called.  The first call in each CUDA context looks up the
 * array's device address with cudaGetSymbolAddress while that context's
 * device is current, and later calls in the context reuse it; make that first
 * call before any stream capture begins on the device.  After a device reset
 * the next call runs in a new context and looks the address up again (again
 * before any capture).
 *
 * All calls share the one array and it keeps the previous call's contents
 * (the call clears what must start at zero itself).  Calls whose GPU work
 * overlaps -- on different streams or host threads -- race on the array and
 * must be serialised by the caller.
 *
 * Arguments are those of hs_argsort with mode HS_MODE_PLAIN and no
 * workspace; n must not exceed HS_NOALLOC_MAX_N (HS_ERR_INVALID_ARG
 * otherwise, before any device work).  The permutation is identical to
 * hs_argsort's. */
#define HS_NOALLOC_MAX_N ((uint64_t)262144)
#define HS_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

HS_API hs_status hs_argsort_noalloc(const uint8_t *d_bytes,
                                    const uint64_t *d_offsets, uint64_t n,
                                    int coder, int out_t, void *d_perm,
                                    void *stream);

/* Workspace needed by hs_encode / hs_argsort for n strings (mode, out_t as
 * in hs_argsort).  total_bytes (the byte-buffer size) is accepted for
 * forward compatibility and currently unused.  Writes *out; HS_OK. */
HS_API hs_status hs_workspace_size(uint64_t n, uint64_t total_bytes, int mode,
                            int out_t, size_t *out);

/* Workspace needed by hs_argsort_batched for n strings in num_segs
 * instances. */
HS_API hs_status hs_batched_workspace_size(uint64_t n, uint64_t num_segs,
                                    size_t *out);

/* Per-kernel timing (no counterpart in the paper: measurement support).
 * While enabled, every kernel the library launches is bracketed by CUDA
 * events recorded on the caller's stream; after each call the elapsed times
 * are added to a process-wide table, one row per kernel kind, with the
 * launch count and the algorithmic bytes the launches had to move (inputs
 * read once plus outputs written once).  Enabling resets the table. */
typedef struct {
    char name[32];
    uint64_t launches;
    double total_ms;
    double algo_bytes;
} hs_kernel_stat;

HS_API hs_status hs_stats_enable(int on);

/* Copies up to max rows into out (host) and writes the number of rows that
 * exist to *count. */
HS_API hs_status hs_stats_read(hs_kernel_stat *out, int max, int *count);

/* hs_shutdown -- release what the library keeps between calls: the copy
 * streams of hs_argsort_host (one per device it ran on), the pooled CUDA
 * events of the host hand-offs and of the per-kernel timing, the pooled
 * pinned host buffers that receive the device-side control block, and the
 * timing table (timing is switched off).  Call it with no library call in flight;
 * later calls recreate what they need.  The allocation-free entry point's
 * static scratch is part of the loaded image and is not released.
 * Safe to call without a GPU or twice; returns HS_OK (HS_ERR_CUDA if a
 * destroy call failed; the rest is still released). */
HS_API hs_status hs_shutdown(void);
/* Tile-shape tuner (no counterpart in the paper: a tuning aid for the
 * radix passes).  The first sort of each layout -- packed (code, index)
 * words (layout 0) or (key, payload) pairs (layout 1) -- in each size class
 * floor(log2 n), for n >= 2^20, runs two of its radix passes with 12 and with
 * 8 keys per thread, times them with CUDA events and keeps the faster shape
 * for later sorts of that class in the process.  The shape never changes a
 * result.  mode 1: tune (the default); 0: use the default shape (12) for
 * classes not tuned yet; 2: forget every choice and tune again.
 * hs_autotune_choice writes the keys per thread chosen for (layout, n), or 0
 * when that class is not tuned. */
HS_API hs_status hs_autotune(int mode);
HS_API hs_status hs_autotune_choice(int layout, uint64_t n, int *items);

/* Numeric coders.  Section 6.1 and Table 4 benchmark Huskysort on Integer, Long and
 * Double arrays and Section 3.2 names a perfect coding for date-times (one
 * nanosecond over 128 years fits 64 bits); the paper gives no bit layout for
 * them.  Each value is coded here as an unsigned 64-bit key whose order is the
 * values' order (Java's compareTo for each type), distinct values getting
 * distinct keys: a perfect coding, so Step 3 never runs.
 *   HS_NUM_U64       uint64: the value itself.
 *   HS_NUM_I64       int64 (two's complement): value XOR 2^63.
 *   HS_NUM_I32       int32: (value XOR 2^31) in the low 32 bits.
 *   HS_NUM_F64       IEEE 754 binary64, as Double.compare orders it: every
 *                    NaN is first replaced by the canonical quiet NaN
 *                    0x7FF8000000000000 (all NaNs equal, above +infinity),
 *                    then a value with the sign bit set is complemented and
 *                    any other gets the sign bit set (so -0.0 < 0.0).
 *   HS_NUM_F32       IEEE 754 binary32 the same way (canonical NaN
 *                    0x7FC00000), in the low 32 bits.
 *   HS_NUM_DATETIME  int64 nanoseconds from the epoch (a date-time as
 *                    epoch second * 10^9 + nanosecond; about +-292 years
 *                    around 1970), coded as HS_NUM_I64.
 * 32-bit types leave the top 32 key bits zero, so their sort needs four
 * radix passes instead of eight. */
typedef enum {
    HS_NUM_U64 = 0,
    HS_NUM_I64 = 1,
    HS_NUM_I32 = 2,
    HS_NUM_F64 = 3,
    HS_NUM_F32 = 4,
    HS_NUM_DATETIME = 5
} hs_numeric;

/* Codes of n values (device, 8 bytes each, 4 for HS_NUM_I32 / HS_NUM_F32)
 * into d_codes (device, n uint64).  No workspace; asynchronous on stream.
 * HS_ERR_INVALID_ARG for a bad type or a NULL pointer with n > 0. */
HS_API hs_status hs_encode_numeric(const void *d_values, uint64_t n, int type,
                                   uint64_t *d_codes, void *stream);

/* Workspace needed by hs_argsort_numeric for n values. */
HS_API hs_status hs_numeric_workspace_size(uint64_t n, int out_t, size_t *out);

/* Stable argsort of n numeric values (device) by the order above: d_perm[k]
 * (device, uint32 or uint64 by out_t) is the index of the k-th smallest
 * value, equal values in index order.  The codes are sorted by the same
 * radix passes as the string codes; the last pass writes the permutation.
 * 0 <= n <= HS_MAX_N; workspace and stream as in hs_argsort. */
HS_API hs_status hs_argsort_numeric(const void *d_values, uint64_t n, int type,
                                    int out_t, void *d_perm, void *d_ws,
                                    size_t ws_bytes, void *stream);

/* BigInteger coder.  Section 6.1 and Table 4 sort BigInteger arrays; the paper gives no
 * coder.  Value i is its minimal two's complement bytes, big-endian (Java's
 * BigInteger.toByteArray), at d_bytes[d_offsets[i] .. d_offsets[i+1]), at
 * most 32767 bytes.  Each is turned into the byte string header || value,
 * header the big-endian u16 0x8000 + L (value >= 0) or 0x7FFF - L (value < 0)
 * for a value of L bytes, whose unsigned-byte order is numeric order; the
 * strings then go through hs_argsort's path with the byte coder.  d_perm
 * (device, uint32 or uint64 by out_t) receives the stable argsort by numeric
 * value.  total_bytes: the size of the byte buffer (d_offsets[n] - d_offsets[0]
 * must not exceed it).  Returns HS_ERR_INVALID_ARG if a value is empty, not
 * minimal (a redundant leading 0x00 or 0xFF) or too long. */
HS_API hs_status hs_bigint_workspace_size(uint64_t n, uint64_t total_bytes,
                                          int out_t, size_t *out);
HS_API hs_status hs_argsort_bigint(const uint8_t *d_bytes,
                                   const uint64_t *d_offsets, uint64_t n,
                                   uint64_t total_bytes, int out_t,
                                   void *d_perm, void *d_ws, size_t ws_bytes,
                                   void *stream);

/* BigDecimal coder.  Section 6.1 and Table 4 sort BigDecimal arrays; the
 * paper gives no coder.  Value i is its decimal text at
 * d_bytes[d_offsets[i] .. d_offsets[i+1]), in the form Java's
 * BigDecimal(String) accepts: an optional '+' or '-', digits with at most
 * one '.' and at least one digit, then optionally 'e' or 'E', an optional
 * sign and the exponent's digits (its value below 10^9); at most 32767 bytes.
 * With the value written as 0.d1 d2 .. dk x 10^X (d1 and dk nonzero) each
 * text becomes a byte string: a class byte (zero; or the sign and whether
 * |X| < 2^23), the exponent in 3 bytes (|X| < 2^23) or 5, complemented for
 * negatives, then the digits two to a byte (99 minus the pair for negatives,
 * which end with 0xFF).  Unsigned-byte order of these strings is numeric
 * order, and values equal under compareTo (1.0 and 1.00) give equal strings;
 * hs_argsort's path sorts them with the byte coder, whose 8-byte prefix
 * holds up to 8 digits.  d_perm (device, uint32 or uint64 by out_t) receives the stable
 * argsort by value.  total_bytes: the size of the byte buffer.  Returns
 * HS_ERR_INVALID_ARG if a text is outside that form or too long, or its
 * offsets decrease or pass total_bytes. */
HS_API hs_status hs_bigdecimal_workspace_size(uint64_t n, uint64_t total_bytes,
                                              int out_t, size_t *out);
HS_API hs_status hs_argsort_bigdecimal(const uint8_t *d_bytes,
                                       const uint64_t *d_offsets, uint64_t n,
                                       uint64_t total_bytes, int out_t,
                                       void *d_perm, void *d_ws,
                                       size_t ws_bytes, void *stream);

/* Test support for the bounded device-side waits.  A radix pass's tiles wait
 * on the counts that earlier tiles publish (decoupled look-back); each wait
 * gives up after a poll budget, records HS_ERR_TIMEOUT and lets its kernel
 * finish, and the fix-up kernels then do nothing.  This call sets, on the
 * current device, the budget in polls (0 restores the default of 2^22) and
 * the id of one tile per pass whose counts are never published
 * (withhold_tile; -1, the default, publishes all), so that a test can make a
 * wait run out and check that the status reaches the caller and the next call
 * succeeds.  Results are wrong while a tile is withheld.  Not for use while
 * other library calls run.  HS_ERR_INVALID_ARG for withhold_tile < -1. */
HS_API hs_status hs_test_bounded_waits(uint32_t spin_limit, int64_t withhold_tile);

/* Message describing the calling thread's last failure ("" if none).  The
 * pointer stays valid until the next library call on this thread. */
HS_API const char *hs_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
HS_API int hs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HUSKY_H */
