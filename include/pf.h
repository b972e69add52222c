/*
 * pf.h - pre-alignment filtering of read / reference-segment pairs on one
 * GB300 GPU (sm_103a).
 *
 * The method is the thesis of M. Alser, "Accelerating the Understanding of
 * Life's Code through Better Algorithms and Hardware Design" (ETH Zurich,
 * 2018, rev. 2019):
 *   - the (2E+1)-diagonal neighbourhood map of pairwise mismatches
 *     (Ch. 6, Eq. 6.1; vacant cells are mismatches, Ch. 6 Discussion),
 *   - the SneakySnake decider on the unweighted neighbourhood maze
 *     (Ch. 8, Eq. 8.2, §8.4.2),
 *   - the GateKeeper decider: Hamming fast path, amending of short zero
 *     streaks, AND of the 2E+1 masks and popcount (Ch. 5, §5.2.1-§5.2.3),
 *   - verification of accepted pairs by banded Levenshtein distance
 *     (Ch. 2 "Accelerating Read Alignment": Ukkonen's band of 2E+1
 *     diagonals), here a bit-vector (Myers/Hyyrö style) kernel.
 *
 * Conventions shared by every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller unless a
 *     parameter says "host".  Calls are asynchronous on the context's
 *     stream; pf_sync() joins them.  The library owns only its context,
 *     its scratch memory and its tuning table.
 *   - The grid column is the reference position i; the diagonal offset
 *     d in [-E, E] indexes the read: cell (i, d) compares ref[i] with
 *     read[i+d].  Cells with i+d outside the read are mismatches.
 *   - 'N' (either case) never matches, not even another 'N'.
 *   - A read and its reference segment have the same length len >= 0.
 *     len = 0 gives accept = 1, count = 0, dist = 0.
 *   - 0 <= E <= PF_MAX_E.  Counts saturate at E + 1; accept = (count <= E).
 *   - Errors a host check can see (null pointers, negative sizes, E_max
 *     out of range) return PF_EINVAL at once and launch nothing.  Errors
 *     found on the device (a per-pair E above E_max or a negative length; a
 *     byte that is not A/C/G/T/N) mark that pair's outputs (count = -1,
 *     accept = 0, dist = -1) or pack the byte as N, and are reported by the
 *     next pf_sync() as PF_EINVAL (PF_EDATA for bytes).  Errors are sticky
 *     per context until pf_last_error() is read.  No exception crosses
 *     this interface.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PF_MAX_E 31

#if defined(__GNUC__)
#define PF_API __attribute__((visibility("default")))
#else
#define PF_API
#endif

typedef struct pf_ctx pf_ctx;

typedef enum {
    PF_OK = 0,
    PF_EINVAL = 1,      /* bad argument */
    PF_ENOMEM = 2,      /* device or pinned allocation failed */
    PF_ECUDA = 3,       /* a CUDA runtime call failed */
    PF_ETIMEOUT = 4,    /* a bounded wait ran out */
    PF_EBUSY = 5,       /* serving loop not in the needed state */
    PF_ECANCELLED = 6,  /* request cancelled */
    PF_EDATA = 7        /* input bytes outside A/C/G/T/N (packed as N) */
} pf_status;

/* Decider mask.  With both bits set the two deciders share one pass over
 * the map; their outputs occupy two slots: [0, n) SneakySnake and
 * [n, 2n) GateKeeper. */
enum { PF_SNEAKYSNAKE = 1u, PF_GATEKEEPER = 2u };

typedef struct {
    int device;         /* CUDA device ordinal */
    void *stream;       /* cudaStream_t the context launches on; NULL = the
                           per-thread default stream */
    size_t hbm_budget;  /* bytes the serving loop may hold for admitted
                           requests; 0 = a quarter of free device memory */
    unsigned flags;     /* reserved, must be 0 */
} pf_config;

/* Packed sequences: three bit-planes of 32-bit words.  Base b of a
 * sequence sets bit (b % 32) of word (b / 32) counted from the sequence's
 * first word, in `lo` (low code bit), `hi` (high code bit) and `nmask`
 * (1 for N).  Codes: A = 00, C = 01, G = 10, T = 11 (§5.2.3 prints A = 00
 * and T = 11).  The unused tail of a sequence's last word is N.
 * Sequence s starts at word word_off[s] (int64, device) or, when word_off
 * is NULL, at word s * stride_words. */
typedef struct {
    const uint32_t *lo;
    const uint32_t *hi;
    const uint32_t *nmask;
    const int64_t *word_off;
    int64_t stride_words;
} pf_seqs;

/* Pair p is read sequence p of `read` against reference segment p of
 * `ref` (the problem statement of §8.1: reference A, read B, both of
 * length m). */
typedef struct {
    pf_seqs read;
    pf_seqs ref;
} pf_pairs;

/* ---- context ----------------------------------------------------------- */

/* Create a context on cfg->device.  *out receives an opaque handle owned by
 * the library; release it with pf_destroy.  PF_EINVAL on a bad config,
 * PF_ECUDA if the device cannot be used. */
PF_API pf_status pf_create(pf_ctx **out, const pf_config *cfg);

/* Wait for outstanding work, free everything the context owns. */
PF_API pf_status pf_destroy(pf_ctx *ctx);

/* Change the stream later calls are enqueued on (cudaStream_t). */
PF_API pf_status pf_set_stream(pf_ctx *ctx, void *stream);

/* Block until every call enqueued so far has finished; return the first
 * error recorded since the last pf_last_error (device-side errors
 * included). */
PF_API pf_status pf_sync(pf_ctx *ctx);

/* Message of the first recorded error (static or context-owned storage,
 * valid until the next call on ctx); clears the sticky error. */
PF_API const char *pf_last_error(pf_ctx *ctx);

/* Name of a status code. */
PF_API const char *pf_status_string(pf_status s);

/* ---- a1: packing (§5.2.3 two-bit encoding, host Read Encoder of Ch. 4) --- */

/* Host helper: word offsets for sequences with byte ranges
 * [byte_off_host[s], byte_off_host[s+1]).  Writes nseq + 1 exclusive
 * prefix sums of ceil(len/32) into word_off_host (host, may be NULL) and
 * the total into *total_words. */
PF_API pf_status pf_pack_layout(const int64_t *byte_off_host, int64_t nseq,
                         int64_t *word_off_host, int64_t *total_words);

/* Pack nseq ASCII sequences.  ascii: device bytes; byte_off, word_off:
 * device int64[nseq+1] (sequence s occupies bytes [byte_off[s],
 * byte_off[s+1]) and words [word_off[s], word_off[s+1]) of each plane);
 * lo/hi/nmask: caller-allocated device planes of word_off[nseq] words.
 * Bits past a sequence's end in its last word, and any words a word_off
 * leaves beyond ceil(len/32), are N.  Bytes other than A/C/G/T/N (either
 * case) inside a sequence pack as N and raise PF_EDATA at the next
 * pf_sync; bytes outside every sequence never change a plane or raise it. */
PF_API pf_status pf_pack(pf_ctx *ctx, const uint8_t *ascii, const int64_t *byte_off,
                  const int64_t *word_off, int64_t nseq,
                  uint32_t *lo, uint32_t *hi, uint32_t *nmask);

/* A ragged layout grouped by threshold and length, for batches whose
 * pairs carry their own E.  The scheduler runs the pairs of one threshold
 * together (in pair order); laid out in pair order, they are scattered over
 * the planes and each one's words cost whole DRAM sectors of their own.
 * Here sequence s gets its ceil(len/32) words (len from byte_off_host) in
 * the order of (E_host[s], min(ceil(len/32), 64), s): the pairs of one
 * threshold and length lie back to back, in pair order.  E_host: host
 * int16[nseq] (pair p's read and reference are sequence p of two
 * buffers packed with the same layout), or NULL to group by length alone.
 * Writes each sequence's first word into word_start_host (host int64[nseq],
 * may be NULL) and the planes' size into *total_words.  PF_EINVAL if an
 * offset falls or an E_host[s] is outside [0, PF_MAX_E]. */
PF_API pf_status pf_pack_layout_grouped(const int64_t *byte_off_host, const int16_t *E_host,
                                        int64_t nseq, int64_t *word_start_host,
                                        int64_t *total_words);

/* Pack nseq ASCII sequences into words given per sequence: word_start is
 * device int64[nseq], and sequence s (bytes [byte_off[s], byte_off[s+1]))
 * occupies words [word_start[s], word_start[s] + ceil(len/32)) of each
 * plane, in any order; the ranges must not overlap and must lie inside
 * the caller's planes (pf_pack_layout_grouped's do, for planes of
 * *total_words words).  Otherwise as pf_pack.  The sequences are then
 * addressed with word_off = word_start in pf_seqs. */
PF_API pf_status pf_pack_starts(pf_ctx *ctx, const uint8_t *ascii, const int64_t *byte_off,
                                const int64_t *word_start, int64_t nseq, uint32_t *lo,
                                uint32_t *hi, uint32_t *nmask);

/* Same for nseq sequences of one length len stored back to back:
 * sequence s is ascii[s*len, (s+1)*len) and occupies words
 * [s*W, (s+1)*W) with W = ceil(len/32). */
PF_API pf_status pf_pack_fixed(pf_ctx *ctx, const uint8_t *ascii, int64_t nseq, int len,
                        uint32_t *lo, uint32_t *hi, uint32_t *nmask);

/* ---- a2-a4, a7: filtering ----------------------------------------------- */

/* Neighbourhood map + deciders for n pairs through the batch scheduler:
 * pairs are grouped by the configuration their threshold is tuned to and,
 * inside a group, by length class (ceil(len/32) words); each group runs the
 * tuned mapping (threads per pair, work chunk) in one persistent launch.
 * Batches below pf_set_small_batch's size take one plain launch (with one
 * threshold for the batch, E NULL and E_max <= 15, the plain kernel with
 * that threshold fixed at compile time).
 *   deciders  PF_SNEAKYSNAKE, PF_GATEKEEPER or both (two output slots)
 *   lens      device int32[n], pair lengths
 *   E         device int16[n] per-pair thresholds, or NULL for E_max for
 *             every pair
 *   E_max     host int, 0..PF_MAX_E, upper bound of every E[p]
 *   accept    device uint8[slots*n]
 *   count     device int16[slots*n], saturated obstacle / edit counts */
PF_API pf_status pf_filter(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                    const int32_t *lens, const int16_t *E, int E_max,
                    uint8_t *accept, int16_t *count, int64_t n);

/* The plain kernel: one thread per pair, one launch over all pairs, no
 * scheduler.  Same arguments and results as pf_filter. */
PF_API pf_status pf_filter_plain(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                          const int32_t *lens, const int16_t *E, int E_max,
                          uint8_t *accept, int16_t *count, int64_t n);

/* The plain kernel with one threshold E (0..15) fixed at compile time: one
 * thread per pair, one launch, every pair filtered at E.  It separates what
 * specialising the threshold gains from what the scheduler's batching and
 * two-phase kernels gain.  Outputs as pf_filter; PF_EINVAL for E > 15. */
PF_API pf_status pf_filter_plain_exact(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                                       const int32_t *lens, int E, uint8_t *accept,
                                       int16_t *count, int64_t n);

/* ---- a7: scheduler tuning --------------------------------------------------- */

/* Kernel configurations of the batch scheduler.  Writes up to cap entries
 * (lanes per pair, diagonal slots per lane, largest E served, the one E an
 * exact-threshold configuration serves or -1, and for the two-phase form
 * the pair length in 32-column words up to which its mask words stay in
 * shared memory, else 0) into the host arrays (any may be NULL) and the
 * number of configurations into *count.  The two-phase form builds every
 * word's mask words (and runs GateKeeper) first, then runs SneakySnake as a
 * per-thread loop of steps over them; longer pairs, and GateKeeper alone,
 * take the fused word loop. */
PF_API pf_status pf_kernel_configs(int *tpp, int *dpt, int *ecap, int *exact_e, int *words,
                                   int cap, int *count);

/* Autotune on a batch as it is: its pairs are grouped by threshold (E,
 * device int16[n], required) and length class, as the scheduler groups
 * them, and for every threshold with at least 1,024 pairs each
 * configuration serving it (and work items of 64, 256 and 1,024 pairs) is
 * timed on up to `sample` of that threshold's own pairs (0 = 2^20; the
 * same share of each of its length classes, each share a run of the class
 * in the scheduler's order), reps timed runs each after one warm-up; the
 * fastest becomes the scheduler's choice for (deciders, E).  Thresholds with fewer pairs keep
 * their choice.  Synchronises the context stream; allocates its output
 * buffers (freed on return).  PF_EINVAL as pf_filter, or for n <= 0,
 * reps <= 0, sample < 0 or a NULL E. */
PF_API pf_status pf_tune_batch(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                               const int32_t *lens, const int16_t *E, int E_max, int64_t n,
                               int64_t sample, int reps);

/* Batches of fewer than `pairs` pairs skip the scheduler: one launch of the
 * plain one-thread-per-pair kernel serving E_max, no binning and no
 * per-threshold launches, whose fixed costs dominate small batches.
 * Default 2^20; 0 sends every batch of pf_filter / pf_filter_verify /
 * pf_run_host through the batched scheduler (unless pf_tune chose the
 * plain kernel).  PF_EINVAL for pairs < 0. */
PF_API pf_status pf_set_small_batch(pf_ctx *ctx, int64_t pairs);

/* enable != 0 (the default): pf_filter_verify and pf_run_host with
 * SneakySnake selected leave out of verification the accepted pairs whose SneakySnake
 * count equals their Hamming distance, whose distance is then known (see
 * pf_filter_verify); 0 verifies every accepted pair.  Results are the same
 * either way.  PF_EINVAL only for a NULL context. */
PF_API pf_status pf_set_resolve_by_bounds(pf_ctx *ctx, int enable);

/* Use configuration cfg and a work chunk of `chunk` pairs (1..65536) for
 * threshold E under decider set `deciders` in later pf_filter calls; cfg =
 * -1 selects the plain kernel.  PF_EINVAL if cfg cannot serve E. */
PF_API pf_status pf_tune_set(pf_ctx *ctx, unsigned deciders, int E, int cfg, int chunk);

/* The configuration and chunk currently used for (deciders, E); cfg = -1
 * when pf_tune chose the plain kernel. */
PF_API pf_status pf_tune_get(pf_ctx *ctx, unsigned deciders, int E, int *cfg, int *chunk);

/* Autotuner: time every configuration that serves E, with work chunks of
 * 64, 256 and 1024 pairs, and the plain one-thread-per-pair kernel, on the
 * n given pairs evaluated at threshold E (CUDA events on the context's
 * stream, best of `reps` runs each), keep the fastest for (deciders, E) and
 * report it (host outputs, may be NULL; *best_cfg = -1 for the plain
 * kernel, which later batches take whenever every threshold they can hold
 * chose it).  The plain kernel is the default at E = 0 (one diagonal, bound
 * by memory); a measurement replaces a default only by a 10% margin.  Synchronises the stream.  Allocates and frees its own
 * output buffers. */
PF_API pf_status pf_tune(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                         const int32_t *lens, int E, int64_t n, int reps,
                         int *best_cfg, int *best_chunk, float *best_ms);

/* ---- measurement: the integer-pipe peak ------------------------------------ */

/* Microbenchmark of the integer pipes the filter runs on (no counterpart in
 * the thesis; it measures the roofline's denominator on the GPU at hand).
 * Every thread of a full-occupancy grid runs many independent dependency
 * chains of one instruction mix, `launches` launches back to back on the
 * context stream, timed with CUDA events after one warm-up launch (each
 * launch takes tens of milliseconds):
 *   kind 0  32-bit LOP3 and funnel-shift (SHF) instructions in equal
 *           numbers: the map's and GateKeeper's mix
 *   kind 1  POPC, each feeding a LOP3
 * *ops_per_s (host) receives the instructions of the mix executed per
 * second over all threads (one instruction of one thread = one op),
 * *ms_per_launch (host, may be NULL) the mean launch time.  Synchronises
 * the context stream.  PF_EINVAL for kind outside 0..1, launches outside
 * 1..1000 or a NULL ops_per_s. */
PF_API pf_status pf_peak_int(pf_ctx *ctx, int kind, int launches, double *ops_per_s,
                             double *ms_per_launch);

/* ---- a5: compaction ------------------------------------------------------ */

/* Indices p (ascending) with flags[p] != 0, p < n, into idx (device
 * int64[n]); their number into *n_out (device int64). */
PF_API pf_status pf_compact(pf_ctx *ctx, const uint8_t *flags, int64_t n,
                     int64_t *idx, int64_t *n_out);

/* Compaction that allocates nothing, for callers that cannot allocate
 * device memory: a framework whose own allocator owns every byte of device
 * memory, or a latency path that cannot take cudaMalloc's implicit device
 * synchronisation.  The thesis has no counterpart: this is an interface
 * convenience.  Same result as pf_compact, but no context is needed and the
 * per-tile counters live in a fixed 256 KiB device array of the library
 * instead of context scratch:
 *   flags, idx, n_out  as in pf_compact (device pointers)
 *   stream             cudaStream_t to launch on (NULL = legacy default)
 * The current device must own flags, idx, n_out and the stream.
 * n must be <= 134,217,728; larger n returns PF_EINVAL and launches nothing.
 * PF_ECUDA if a launch fails.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the life
 * of the process, so make that call before any stream capture, and do not
 * call this function again after a cudaDeviceReset (or any other teardown of
 * the device's primary context) in the same process: the kept address would
 * be stale.  Every call shares the array: calls whose kernels overlap on the
 * GPU (other streams, other threads) race and must be serialised by the
 * caller.  Every GPU that loads the library holds the array until the
 * process exits. */
PF_API pf_status pf_compact_noalloc(const uint8_t *flags, int64_t n, int64_t *idx,
                                    int64_t *n_out, void *stream);

/* ---- The thesis's other deciders on the same neighbourhood map ---------- */

/* The three calls below take the arguments of pf_filter (one decider, one
 * output slot: accept[n] and count[n], count = min(edits, E+1), accept =
 * count <= E; a pair with len < 0 or E outside [0, E_max] gets count -1,
 * accept 0 and makes pf_sync report PF_EINVAL).  Asynchronous on the
 * context stream; caller-owned device buffers.  Per pair one thread builds
 * the map a word at a time. */

/* SneakySnake on sub-matrices (§8.5): the map is cut into non-overlapping
 * sub-matrices of t columns (1 <= t <= 32; the last one holds what is
 * left), each solved as its own Sneaky Snake Problem: the snake enters its
 * first column free to pick any row, a pipe that reaches its last column
 * leaves it, and at most y >= 1 replications (searches) run in it, so it
 * contributes min(y, its obstacles).  The count is the sum over the
 * sub-matrices; never above SneakySnake's, so no pair within E is
 * rejected.  PF_EINVAL for t or y out of range. */
PF_API pf_status pf_filter_partitioned(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens,
                                       const int16_t *E, int E_max, int t, int y,
                                       uint8_t *accept, int16_t *count, int64_t n);

/* Shouji (Ch. 6): for each of the m windows of 4 columns, the diagonal
 * 4-bit vector with the most zeros (ties: the first, in diagonal order
 * d = -E..E, whose first bit is 0, else the first) replaces the Shouji
 * bit-vector's four bits there when it holds more zeros than they do; the
 * bit-vector starts all ones, window cells past the end read as 1, and the
 * count is the ones left in the bit-vector. */
PF_API pf_status pf_filter_shouji(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens,
                                  const int16_t *E, int E_max, uint8_t *accept, int16_t *count,
                                  int64_t n);

/* GateKeeper with SHD's conventions (Ch. 3), for accuracy comparisons:
 *   PF_SHD_VACANT_ZERO  out-of-range cells of the shifted masks are 0 (as
 *                       SHD's arithmetic shifts fill them) instead of 1;
 *   PF_SHD_STREAK       each maximal run of L ones of the final bit-vector
 *                       counts ceil(L/3) edits (SHD's conservative counting
 *                       charges three consecutive ones as one edit).
 * flags = 0 gives GateKeeper's count; other bits are PF_EINVAL. */
#define PF_SHD_VACANT_ZERO 1u
#define PF_SHD_STREAK 2u
PF_API pf_status pf_filter_shd(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens,
                               const int16_t *E, int E_max, unsigned flags, uint8_t *accept,
                               int16_t *count, int64_t n);

/* ---- a6: verification ---------------------------------------------------- */

/* dist = min(Levenshtein(read, ref), E + 1) for the selected pairs, exact.
 *   idx == NULL : pairs 0..n-1, dist[p] written for each.
 *   idx != NULL : pairs idx[t] for t < *n_idx (device int64, <= n);
 *                 dist[idx[t]] written, other entries untouched. */
PF_API pf_status pf_verify(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens,
                    const int16_t *E, int E_max, const int64_t *idx,
                    const int64_t *n_idx, int64_t n, int32_t *dist);

/* Whole path for n pairs: filter (deciders as in pf_filter), compact the
 * pairs the first selected decider accepts, verify them; dist[p] =
 * min(ED, E+1) for those and E + 1 for every rejected pair.  With
 * SneakySnake selected, an accepted pair whose obstacle count equals its Hamming
 * distance (a lower and an upper bound on its banded edit distance) gets
 * that count as dist from the filter and is not verified (the same value
 * the verifier would write); pf_set_resolve_by_bounds turns this off. */
PF_API pf_status pf_filter_verify(pf_ctx *ctx, unsigned deciders, const pf_pairs *pairs,
                           const int32_t *lens, const int16_t *E, int E_max,
                           uint8_t *accept, int16_t *count, int32_t *dist, int64_t n);

/* The number of pairs the most recent pf_filter_verify on this context sent
 * to verification (its accepted pairs less those resolved by equal bounds).
 * Synchronises the context stream.  PF_EINVAL if there is no such call, or
 * if a later call on the context reallocated its scratch memory. */
PF_API pf_status pf_last_verified_count(pf_ctx *ctx, int64_t *n_verified);

/* ---- host memory for the host-buffer calls ------------------------------- */

/* Page-locked host memory backed by 2 MB pages where the system has them.
 * Blocks are carved out of a few large regions (at least 1 GB each; Linux:
 * an anonymous mapping advised for transparent huge pages, registered with
 * cudaHostRegister once) that live for the rest of the process; a freed
 * block's space is reused.  Meant for the buffers pf_run_host and serving
 * requests upload from and write to: fewer, larger pages leave the device
 * fewer address translations to make (uploads from page-locked memory
 * allocated buffer by buffer were measured to stall for milliseconds at
 * times; from such regions less often).  *ptr receives a 256-byte-aligned
 * block of at least `bytes` bytes (host, owned by the caller until
 * pf_host_free).  PF_EINVAL for bytes == 0 or a null ptr, PF_ENOMEM if a
 * region cannot be mapped, PF_ECUDA if registering it fails.  Needs no
 * context; thread-safe. */
PF_API pf_status pf_host_alloc(size_t bytes, void **ptr);

/* Release a block of pf_host_alloc (NULL is a no-op); PF_EINVAL for any
 * other pointer.  No GPU work may still use it. */
PF_API pf_status pf_host_free(void *ptr);

/* ---- a7: the whole path on host buffers, chunked and graph-replayed ------ */

/* Pack, filter, compact and verify n pairs held in HOST memory, chunk by
 * chunk: two slots with their own device buffers and streams alternate,
 * so one chunk's upload overlaps the other's device work; each slot's
 * device work (offsets, pack, filter, compaction, verification) is captured
 * once as a CUDA graph and replayed for every chunk of that size.  Returns
 * when every result is in host memory.
 *   reads, refs  host ASCII; pair p is bytes [byte_off[p], byte_off[p+1])
 *                of both (host int64[n+1]) or, when byte_off is NULL,
 *                bytes [p*len, (p+1)*len)
 *   E            host int16[n], or NULL for E_max for every pair
 *   accept, count, dist  host outputs as in pf_filter_verify
 *   chunk_pairs  pairs per chunk (>= 1; 0 = 2^20)
 * Page-locked host buffers (pf_host_alloc's, or any registered memory)
 * are copied asynchronously; pageable ones work but serialise the copies.
 * Allocates its slot buffers (freed on return). */
PF_API pf_status pf_run_host(pf_ctx *ctx, unsigned deciders, const uint8_t *reads,
                             const uint8_t *refs, const int64_t *byte_off, int len,
                             const int16_t *E, int E_max, uint8_t *accept, int16_t *count,
                             int32_t *dist, int64_t n, int64_t chunk_pairs);

/* ---- a8: serving (continuous batching) ------------------------------------ */

/* The accelerator of Ch. 4 streams pairs through its filtering units and
 * returns each decision as soon as it is made.  Here a host scheduler
 * thread admits requests as they arrive, by slots and device memory, and
 * feeds them to the GPU while earlier ones run; results go back to each
 * request's host buffers as soon as its last pair is done.  Two modes:
 *
 * PF_SERVE_BATCHED (the default): continuous batching into device batches.
 *   Admitted requests are placed, in arrival order, into the open batch;
 *   their bytes are uploaded by the copy engine at once (a request larger
 *   than the room left is split, the rest going to the next batch).  A batch
 *   is launched as soon as fewer than two batches are on the GPU, so
 *   requests that arrive while one runs gather in the next and batches grow
 *   with the load.  Each batch runs the tuned path of pf_filter_verify
 *   (pack, the scheduler's binned and tuned filter kernels, compaction,
 *   verification) on its pairs, with the serving context's tuning table;
 *   an epilogue kernel writes each pair's results into its request's
 *   buffers (directly when they are page-locked).  hbm_budget sizes the
 *   batch buffers; a request of any size streams through them.
 * PF_SERVE_DEVICE_LOOP: a persistent device loop takes work items (chunks
 *   of admitted requests) from a ring in mapped host memory and packs,
 *   filters (a generic runtime-threshold kernel, 8 lanes per pair) and
 *   verifies each chunk inside one block.  No launch per batch; a request
 *   must fit the budget whole.  Every device wait is bounded: the loop
 *   exits after idle_exit_us without work (the scheduler relaunches it on
 *   demand) or when stopped. */
#define PF_SERVE_BATCHED 0
#define PF_SERVE_DEVICE_LOOP 1

typedef struct {
    size_t hbm_budget;   /* device bytes for admitted requests (device loop)
                            or batch buffers (batched); 0 = the context's
                            hbm_budget, else a quarter of free device memory */
    int max_requests;    /* requests admitted at once, 1..4096 (0 = 256) */
    int chunk_pairs;     /* device loop: pairs per work item, 32..1024
                            (0 = 1024) */
    int workers;         /* device loop: blocks of the loop (0 = 2 per SM) */
    int idle_exit_us;    /* device loop: the loop ends after this long
                            without work, 50..10^6 (0 = 500) */
    int start_paused;    /* nonzero: admit and stage, but run nothing until
                            pf_serve_resume */
    int mode;            /* PF_SERVE_BATCHED or PF_SERVE_DEVICE_LOOP */
    int batch_pairs;     /* batched: most pairs in one device batch, 0 = up
                            to 2^20 as the budget allows; >= 0 */
    int overlap_pairs;   /* batched: while a batch runs, the next one is
                            launched beside it only once it holds this many
                            pairs (else it keeps growing until the GPU has
                            no batch); 0 = 2^18 */
} pf_serve_config;

/* One request: n pairs in HOST memory.  Pair p is reads[byte_off[p] ..
 * byte_off[p+1]) against refs[byte_off[p] .. byte_off[p+1]).  All buffers
 * belong to the caller and must stay valid until pf_wait/pf_poll reports
 * the request done.  Page-locked buffers are fastest: their bytes are
 * uploaded asynchronously and, in the batched mode, the GPU reads offsets
 * and thresholds and writes results in place; pageable ones are copied
 * through pinned staging memory.  Outputs as in pf_filter_verify: accept and count
 * [slots*n], dist [n] = min(ED, E+1) for pairs the first selected decider
 * accepts, E+1 for the others. */
typedef struct {
    unsigned deciders;
    int64_t n;
    const uint8_t *reads;
    const uint8_t *refs;
    const int64_t *byte_off;   /* host int64[n+1], non-decreasing */
    const int16_t *E;          /* host int16[n], each 0..PF_MAX_E */
    uint8_t *accept;
    int16_t *count;
    int32_t *dist;
} pf_request;

typedef struct {
    uint64_t submitted, completed, failed, pairs_completed;
    uint64_t loop_launches;    /* device loop: times it was (re)started;
                                  batched: device batches launched */
    /* seconds summed over completed requests: waiting for admission,
     * uploading, on the device (published to complete), results back */
    double queue_s, stage_s, device_s, drain_s;
    /* the longest single request in each of those phases, seconds */
    double queue_max_s, stage_max_s, device_max_s, drain_max_s;
    /* batched mode: pairs over all batches, the largest batch, GPU time of
     * the batches (from the end of their uploads to their last kernel), and
     * the scheduler thread's time placing requests and enqueuing batches */
    uint64_t batch_pairs, batch_pairs_max;
    double batch_gpu_s, place_host_s, launch_host_s;
} pf_serve_stats;

/* Start serving on ctx (PF_EBUSY if already serving).  Allocates the
 * device buffers of the mode, pinned staging memory and the scheduler
 * thread.  The batched mode copies ctx's tuning table (pf_tune,
 * pf_tune_batch, pf_tune_set, pf_set_small_batch, pf_set_resolve_by_bounds
 * made before this call) into a private context of the serving thread, so
 * calls on ctx may run beside it. */
PF_API pf_status pf_serve_start(pf_ctx *ctx, const pf_serve_config *cfg);

/* Queue a request; *ticket identifies it.  Malformed requests (null
 * pointers, decreasing offsets, E outside [0, PF_MAX_E]) return PF_EINVAL,
 * requests that could never fit the budget PF_ENOMEM (device loop: the
 * request whole; batched: one pair, or the pinned staging a pageable
 * request needs); neither is queued. */
PF_API pf_status pf_submit(pf_ctx *ctx, const pf_request *req, uint64_t *ticket);

/* *done = 1 once the request's results are in its host buffers. */
PF_API pf_status pf_poll(pf_ctx *ctx, uint64_t ticket, int *done);

/* Wait up to timeout_ms (< 0: no limit) for the request.  Returns its
 * status (PF_OK, PF_EINVAL for pairs the device found invalid,
 * PF_ECANCELLED if serving stopped first) or PF_ETIMEOUT if it is still in
 * flight; *latency_ms (may be NULL) = submit to results in host memory.  A
 * finished ticket is released by the first pf_wait that reports it. */
PF_API pf_status pf_wait(pf_ctx *ctx, uint64_t ticket, int timeout_ms, double *latency_ms);

/* Run a loop started with start_paused. */
PF_API pf_status pf_serve_resume(pf_ctx *ctx);

PF_API pf_status pf_serve_stats_get(pf_ctx *ctx, pf_serve_stats *out);

/* Open-loop load replay, for offered-load measurements: from the calling
 * thread, submit request pool[i % npool] at arrival_s[i] seconds after the
 * call (i < count, arrival_s non-decreasing), then wait for all of them.
 * latency_ms[i] (host, count entries) receives each request's submit-to-
 * results latency, *elapsed_s the time from the call to the last result.
 * Requests of the pool may be in flight more than once at a time; their
 * outputs are then written more than once with the same values.  Returns
 * the first non-OK request status, PF_OK otherwise. */
PF_API pf_status pf_serve_replay(pf_ctx *ctx, const pf_request *pool, int npool,
                                 const double *arrival_s, int count, double *latency_ms,
                                 double *elapsed_s);

/* Batched mode: the most recent device batches (up to the last 65,536),
 * oldest first, PF_SERVE_TRACE_FIELDS doubles each, into records (host,
 * cap records; *count receives how many were written):
 *   [0] launch time and [1] completion time (seconds since pf_serve_start,
 *       on the scheduler thread's clock: when it enqueued the batch and
 *       when it saw the batch finish),
 *   [2] pairs, [3] request parts,
 *   [4] ms the batch's GPU work waited for its uploads and for the batch
 *       before it (from its enqueue on the compute stream to its start),
 *   [5] ms of GPU work (start of its first kernel to end of its last),
 *   [6] ms the scheduler spent enqueuing it, [7] its decider set,
 *   [8..12] ms of GPU work in its phases: offsets, packing, filter,
 *       compaction and verification, epilogue.
 * PF_EBUSY when not serving in the batched mode. */
#define PF_SERVE_TRACE_FIELDS 13
PF_API pf_status pf_serve_trace(pf_ctx *ctx, double *records, int cap, int *count);

/* Stop the device loop and the scheduler; requests not finished end with
 * PF_ECANCELLED. */
PF_API pf_status pf_serve_stop(pf_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
