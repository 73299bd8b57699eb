/*
 * gbsieve.h -- C ABI of the GB300 segmented sieve of Eratosthenes.
 *
 * The operation (paper, Section 3.1, "Algorithm Design"): the sieve of
 * Eratosthenes marks as composite the multiples of each prime, starting with
 * the multiples of 2; what stays unmarked is prime.  Section 1 gives the bound
 * that makes a range sieve possible: n is prime iff no prime <= sqrt(n)
 * divides it, so [lo, hi) is decided by the "base primes" <= sqrt(hi - 1).
 * Eq. 3 splits the integers into blocks; here a block is a shared-memory
 * segment and the last one may be short.
 *
 * Conventions shared by every call:
 *  - Ranges are half-open [lo, hi) of unsigned 64-bit integers, lo <= hi.
 *    lo == hi is an empty range (0 primes, success).  hi may not exceed the
 *    context's hi_max (SIEVE_ERANGE), and hi_max is at most 2^62.
 *  - count(lo, hi) = #{p prime : lo <= p < hi}; 0 and 1 are not prime.
 *  - Odd-only bitmap: let o0 = lo | 1 (the first odd integer >= lo).  Bit i
 *    (32-bit word i >> 5, bit i & 31, least significant first, words in
 *    little-endian order) is 1 iff o0 + 2 i is prime, for
 *    0 <= i < nbits = ceil((hi - o0) / 2) (0 when o0 >= hi).  The bitmap has
 *    ceil(nbits / 32) words; bits past nbits in the last word are written 0.
 *    2 has no bit (it is even); it is counted by count and listed by list.
 *  - List: the primes of [lo, hi) in ascending order, 2 included.
 *  - Pointers named *_dev are CUDA device pointers on the context's device,
 *    owned by the caller (e.g. torch.Tensor.data_ptr()); the library never
 *    frees them.  All other pointers are host pointers owned by the caller.
 *  - Every call is synchronous (it returns after the GPU work it started has
 *    finished) unless its comment says otherwise.  Work runs on the
 *    context's stream.  A context is not thread-safe; separate contexts are
 *    independent.
 *  - Return value: 0 (SIEVE_OK) or a negative SIEVE_E* code; output
 *    arguments are unspecified on error except where stated.
 *    sieve_strerror() names a code; sieve_last_error() gives the context's
 *    last message (e.g. the CUDA error string).
 */
#ifndef GBSIEVE_H
#define GBSIEVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIEVE_OK        0
#define SIEVE_EINVAL   -1  /* bad argument: lo > hi, NULL pointer, bad size */
#define SIEVE_ERANGE   -2  /* hi > hi_max, or hi > 2^32 for a uint32 list */
#define SIEVE_ETRUNC   -3  /* output capacity < result size; *n = size needed */
#define SIEVE_ENOMEM   -4  /* device or host allocation failed */
#define SIEVE_ECUDA    -5  /* a CUDA runtime call failed */
#define SIEVE_ETIMEOUT -6  /* a bounded wait ran out */
#define SIEVE_EBUSY    -7  /* server: no free slot or memory for the request */
#define SIEVE_ENOENT   -8  /* server: unknown ticket */
#define SIEVE_EDEVICE  -9  /* a kernel reported an internal limit was hit */

typedef struct sieve_ctx sieve_ctx;

/*
 * Create a context for ranges with hi <= hi_max (2 <= hi_max <= 2^62) on CUDA
 * device `device`.  cuda_stream is a cudaStream_t to run on (NULL: the
 * context creates and owns its own non-blocking stream).  Creation generates
 * the base primes <= floor(sqrt(hi_max - 1)) on the device (Section 1's bound)
 * and the pre-sieved pattern tile; both stay resident until sieve_destroy.
 * On success *out receives the context.
 */
int sieve_create(sieve_ctx **out, uint64_t hi_max, int device, void *cuda_stream);

/* Release every device and host resource of the context (NULL is a no-op). */
void sieve_destroy(sieve_ctx *ctx);

/*
 * Number of primes in [lo, hi) (Section 3.1 sieve, counted), written to the
 * host integer *count.
 */
int sieve_count(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *count);

/*
 * As sieve_count, but the count is written to the device integer
 * *count_dev and the call is ASYNCHRONOUS: it returns after enqueueing the
 * work on the context's stream.  *count_dev is overwritten (UINT64_MAX if a
 * bucket list overflowed or a device-side wait gave up).  Calls may follow
 * one another without a synchronisation.
 */
int sieve_count_dev(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *count_dev);

/*
 * Odd-only prime bitmap of [lo, hi) (layout above) into out_dev[0 .. words),
 * words = ceil(nbits / 32).  out_words is the capacity of out_dev in 32-bit
 * words: fewer than needed gives SIEVE_ETRUNC and writes nothing.  Words
 * past the needed ones are not touched.  If count is not NULL the number of
 * primes in [lo, hi) is also written to the host integer *count.
 */
int sieve_bitmap(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t *out_dev,
                 size_t out_words, uint64_t *count);

/* Number of 32-bit words of the odd-only bitmap of [lo, hi). */
uint64_t sieve_bitmap_words(uint64_t lo, uint64_t hi);

/*
 * Ascending list of the primes in [lo, hi) as uint32 values into
 * out_dev[0 .. *n).  Requires hi <= 2^32 (SIEVE_ERANGE otherwise).  *n
 * receives the number of primes in the range even when it exceeds cap; then
 * the call returns SIEVE_ETRUNC and writes nothing, so out_dev = NULL with
 * cap = 0 is the size query.  Uses a context-owned scratch bitmap that grows
 * to the largest range listed so far.
 */
int sieve_list(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t *out_dev,
               size_t cap, uint64_t *n);

/* As sieve_list with uint64 values; any hi <= hi_max. */
int sieve_list64(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *out_dev,
                 size_t cap, uint64_t *n);

/*
 * Compaction only: the ascending uint32 prime list of [lo, hi) read from an
 * odd-only bitmap of [lo, hi) that is already on the device (bitmap_dev,
 * layout above, e.g. written by sieve_bitmap).  Same *n / cap / ETRUNC
 * contract as sieve_list; requires hi <= 2^32.  For this call and the list
 * calls, out_dev = NULL with cap > 0 is SIEVE_EINVAL, before any GPU work.
 */
int sieve_compact(sieve_ctx *ctx, const uint32_t *bitmap_dev, uint64_t lo,
                  uint64_t hi, uint32_t *out_dev, size_t cap, uint64_t *n);

/*
 * Asynchronous forms of sieve_bitmap and sieve_compact for stream pipelines
 * (bitmap, then list, then whatever consumes it, with no host round trip).
 * Arguments, layouts and argument errors are those of the synchronous calls,
 * except that the count goes to a device integer and the call returns after
 * enqueueing its work on the context's stream.  Buffers must stay valid until
 * the stream has run the work.  Calls may follow one another without a
 * synchronisation (a call first waits, on the host, until the previous call's
 * launch parameters have been copied to the device).
 *
 * sieve_bitmap_dev: *count_dev (required) = the number of primes in [lo, hi),
 *   or UINT64_MAX if a bucket list overflowed or a device-side wait gave up;
 *   the bitmap is then not valid (the synchronous call retries instead).
 * sieve_compact_dev: *n_dev = the number of primes in [lo, hi), or UINT64_MAX
 *   if the compaction's bounded wait for another tile's offset gave up (then
 *   the list is not valid; not seen in normal runs).  The list is written in one
 *   pass (each tile's offset found by decoupled look-back, no separate counting
 *   pass), so it is not known to fit before it is written: the first
 *   min(*n_dev, cap) primes are written, and *n_dev > cap after synchronising
 *   means the list was truncated.  cap = 0 with out_dev = NULL is the size query.
 *   Requires hi <= 2^32.
 */
int sieve_bitmap_dev(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t *out_dev,
                     size_t out_words, uint64_t *count_dev);
int sieve_compact_dev(sieve_ctx *ctx, const uint32_t *bitmap_dev, uint64_t lo,
                      uint64_t hi, uint32_t *out_dev, size_t cap, uint64_t *n_dev);

/*
 * Batched counting: m ranges [lo[i], hi[i]) (host arrays) sieved by one
 * persistent kernel launch (replayed from a CUDA graph captured per batch
 * capacity).  counts[i] (host) receives each range's prime count.  If
 * bitmaps_dev is not NULL, bitmaps_dev[i] (a host array of device pointers,
 * any of which may be NULL) receives range i's odd-only bitmap; its capacity
 * must be at least sieve_bitmap_words(lo[i], hi[i]) words.  m = 0 is a no-op.
 */
int sieve_batch_count(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi,
                      size_t m, uint64_t *counts, uint32_t *const *bitmaps_dev);

/*
 * Launch parameters of one range of a batch (sieve_batch_count_params), so
 * that ranges of different size classes are each sieved with their own
 * choice inside the same launch -- the GPU form of the paper's Algorithm 1,
 * which picks the work split of a block by its size.  A field left 0 takes the
 * context's value (sieve_set_param).  Results never depend on these.
 */
typedef struct {
    uint32_t seg_bytes;     /* segment bytes: a multiple of 32 in 1024 .. 229376 */
    uint32_t wheel;         /* 30 or 210 (the mod-210 wheel serves count-only batches) */
    uint64_t bucket_limit;  /* mod 30: base primes >= this go through bucket lists;
                               1 << 62 for none */
    uint32_t mid_limit;     /* base primes below this use the per-phase (mod 30) or
                               per-class (mod 210) tier, larger ones the wheel walk */
    uint32_t mr_percent;    /* as SIEVE_PARAM_MR_PERCENT; UINT32_MAX: never */
} sieve_range_params;

/*
 * As sieve_batch_count, with params[i] (a host array of m, or NULL for the
 * context's parameters everywhere) the launch parameters of range i.  The
 * ranges on the mod-30 wheel are sieved by one persistent kernel launch and
 * those on the mod-210 wheel by a second one; both are captured together in one
 * CUDA graph (per batch shape) and replayed as one graph launch.  Ranges whose
 * parameters call for bucket lists make the batch launch directly instead.
 * SIEVE_EINVAL for an out-of-range field, or wheel 210 with bitmaps_dev set.
 */
int sieve_batch_count_params(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi,
                             size_t m, const sieve_range_params *params, uint64_t *counts,
                             uint32_t *const *bitmaps_dev);

/*
 * Compaction that allocates no device memory, for callers that cannot call
 * cudaMalloc (code running inside a fixed memory arena, a real-time loop that
 * must not take the allocator's locks, or a plug-in whose host owns all
 * device memory).  The paper has no counterpart: this is a deployment aid.
 *
 * Same result and *n / cap / SIEVE_ETRUNC contract as sieve_compact, without
 * a context: it runs on cuda_stream (a cudaStream_t; NULL = the legacy
 * default stream) of the current device.  Its scratch (per-tile popcounts,
 * their prefix sums, the total) is a fixed __device__ array of about 384 KiB
 * inside the library, held by every GPU that loads the library until the
 * process exits.  Limit: the bitmap may have at most SIEVE_STATIC_MAX_WORDS
 * words (the whole of [0, 2^32)); larger ranges, or hi > 2^32, return
 * SIEVE_ERANGE before any GPU work.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  The address is kept for the life of the process: do
 * not call this function on a device after cudaDeviceReset of that device.
 * out_dev = NULL with cap = 0 is the size query; NULL with cap > 0 is
 * SIEVE_EINVAL, before any GPU work.  All calls on a device share the one array: calls that
 * overlap on the GPU (other streams or host threads) race, so serialise them.
 * The array keeps the last call's contents; every entry is written before it
 * is read, so nothing needs clearing.  Synchronous, like sieve_compact.
 */
#define SIEVE_STATIC_MAX_WORDS (1ull << 26)
int sieve_compact_static(const uint32_t *bitmap_dev, uint64_t lo, uint64_t hi,
                         uint32_t *out_dev, size_t cap, uint64_t *n,
                         void *cuda_stream);

/*
 * ---------------------------------------------------------------- serving
 * A request server on a context: sieve requests of mixed sizes arrive at any
 * time from any host thread and are sieved by continuous batching.  A host
 * scheduler thread splits every admitted request into runs of consecutive
 * segments; each scheduling tick launches ONE persistent sieve kernel over
 * runs taken from all requests that still have work (at most tick_segments
 * segments in all), and up to two ticks are in flight on the GPU.  A request
 * that arrives while others run joins the next tick, so short requests are
 * not stuck behind long ones, and a long request advances a few segments per
 * tick.  Base primes and the pattern tile are the context's, shared
 * read-only; the server has its own streams and buffers, so the context stays
 * usable from other threads.  A request's result does not depend on what else
 * is in flight: every run is sieved the same way as by sieve_count, and the
 * runs of a request partition its range.
 *
 * Admission: a request is rejected with SIEVE_EBUSY when max_requests are in
 * flight or, for a list request, when its device memory -- the odd-only bitmap
 * plus room for at most 2 w / ln w + 64 primes, w = hi - lo (the
 * Montgomery-Vaughan form of the Brun-Titchmarsh bound on primes in an
 * interval) -- does not fit in what is left of max_device_bytes.
 */
typedef struct sieve_server sieve_server;

#define SIEVE_REQ_COUNT 0 /* result: the count */
#define SIEVE_REQ_LIST  1 /* result: the count and the ascending primes (uint64, host) */
#define SIEVE_REQ_LIST_OFFSETS 2 /* result: the count and the ascending offsets p - lo of
                                    the primes (uint32, host): half the bytes of a list,
                                    for ranges with hi - lo <= 2^32 (else SIEVE_ERANGE at
                                    submit).  Results cross to the host over a link of
                                    about 193 GB/s, which bounds a stream of list requests */

typedef struct {
    uint32_t max_requests;     /* requests admitted and not yet released (0: 1024) */
    uint32_t tick_segments;    /* segments per scheduling tick (0: 4 x SMs) */
    uint64_t max_device_bytes; /* device memory for list requests (0: 4 GiB) */
    uint32_t serial_ticks;     /* 1: both tick slots on one stream, so a tick's kernels start only
                                  when the previous tick's have ended; 0 (default): one stream per
                                  slot, so the next tick's CTAs fill the SMs the previous tick's
                                  last segments leave idle */
    uint32_t reserved;
    uint64_t host_arena_bytes; /* pinned host memory that list results are copied into by DMA
                                  (0: 1 GiB); results that do not fit go through a bounce buffer */
} sieve_server_cfg;

typedef struct {
    uint64_t lo, hi; /* the range [lo, hi), hi <= the context's hi_max */
    int32_t kind;    /* SIEVE_REQ_COUNT, SIEVE_REQ_LIST or SIEVE_REQ_LIST_OFFSETS */
    int32_t reserved;
} sieve_req;

typedef struct {
    int32_t status;         /* SIEVE_OK, or the error this request failed with */
    int32_t kind;
    uint64_t count;         /* primes in [lo, hi) */
    const uint64_t *primes; /* SIEVE_REQ_LIST: `count` primes, host memory owned by the
                               server, valid until sieve_server_release; else NULL.  It is
                               pinned memory (a 1 GiB arena the results are copied into by
                               DMA) unless the arena was full, then ordinary heap memory */
    double latency_us;      /* from submit to the result being ready on the host */
    const uint32_t *offsets; /* SIEVE_REQ_LIST_OFFSETS: `count` offsets p - lo, memory as for
                               primes; else NULL */
} sieve_result;

typedef struct {
    uint64_t submitted, completed, rejected, ticks;
    uint64_t integers;      /* sum of hi - lo over completed requests */
    uint32_t in_flight;     /* admitted, not yet completed */
    uint32_t reserved;
    uint64_t device_bytes_reserved;
    uint64_t segments;      /* segments sieved by the ticks so far */
    double tick_gpu_ms;     /* sum over ticks of the GPU time from a tick's first launch to its
                               last copy (CUDA events); ticks on two streams may overlap */
} sieve_server_counters;

/* Start a server on ctx (cfg may be NULL for defaults).  ctx must outlive it. */
int sieve_server_create(sieve_ctx *ctx, const sieve_server_cfg *cfg, sieve_server **out);

/* Admit a request; *ticket identifies it.  SIEVE_EBUSY if it does not fit now,
 * SIEVE_EINVAL / SIEVE_ERANGE for a bad range or kind.  Never blocks on GPU work. */
int sieve_server_submit(sieve_server *srv, const sieve_req *req, uint64_t *ticket);

/* Wait up to timeout_us microseconds (< 0: no limit) for a request's result.
 * SIEVE_ETIMEOUT if it is not ready by then, SIEVE_ENOENT for an unknown or
 * released ticket.  May be called again after a timeout or a success. */
int sieve_server_poll(sieve_server *srv, uint64_t ticket, sieve_result *res, int64_t timeout_us);

/* Completion queue: wait up to timeout_us microseconds (< 0: no limit) until at
 * least one request has completed and not yet been reported here, then write up
 * to cap such tickets, in completion order, to tickets[0 .. *n).  Each completed
 * request is reported once (whether or not it was also polled), so a caller can
 * collect and release results without polling every ticket.  SIEVE_ETIMEOUT
 * (*n = 0) if none completed in time. */
int sieve_server_wait_any(sieve_server *srv, uint64_t *tickets, size_t cap, size_t *n, int64_t timeout_us);

/* Forget a completed request and free its result (SIEVE_EBUSY if not done). */
int sieve_server_release(sieve_server *srv, uint64_t ticket);

/* Counters since creation. */
int sieve_server_stats(sieve_server *srv, sieve_server_counters *st);

/* Finish the work in flight, stop the scheduler and free the server. */
void sieve_server_destroy(sieve_server *srv);

/* Tunable launch parameters (see sieve_set_param / sieve_get_param). */
#define SIEVE_PARAM_SEGMENT_BYTES 1 /* shared-memory segment, bytes; multiple of 32 */
#define SIEVE_PARAM_THREADS       2 /* threads per CTA: 256, 512 or 1024 */
#define SIEVE_PARAM_SMALL_LIMIT   3 /* primes below this are crossed warp-cooperatively (default 304) */
#define SIEVE_PARAM_CTAS_PER_SM   4 /* persistent CTAs per SM */
#define SIEVE_PARAM_CHUNK_SEGMENTS 5 /* consecutive segments per work item (1..64; default 32) */
#define SIEVE_PARAM_BUCKET_LIMIT  6 /* primes >= this go through bucket lists; 0 = segment bytes;
                                       default 2^62 (off: direct crossing measured faster) */
#define SIEVE_PARAM_MR_PERCENT    8 /* a range of width w < this % of the base primes above 2^16
                                       it would need is sieved with the primes below 2^16 only and
                                       its survivors tested by deterministic Miller-Rabin (the first
                                       twelve primes as bases, exact for n < 3.18e23); 0 = never;
                                       default 0 (off: measured slower on the 4096-interval
                                       batch at every threshold tried) */
#define SIEVE_PARAM_MID_LIMIT     9 /* primes from the small limit up to this are crossed one lane
                                       per prime with per-byte-phase sub-progressions, larger ones
                                       by walking the wheel; 0 = segment bytes / 3 (default) */
#define SIEVE_PARAM_WHEEL         10 /* count-only calls (sieve_count, sieve_count_dev,
                                        sieve_batch_count without bitmaps) sieve on the mod-30 wheel
                                        (30, default) or the mod-210 wheel (210: 48 bits per 210
                                        integers, multiples of 7 not crossed); results are the same */
#define SIEVE_PARAM_SMALL_LIMIT_210 11 /* mod-210 wheel: primes below this are crossed one warp per
                                          (prime, class) with conflict-free lanes (default 128) */
#define SIEVE_PARAM_MID_LIMIT_210 12 /* mod-210 wheel: primes from the small limit up to this are
                                        crossed one lane per prime with per-class sub-progressions,
                                        larger ones by the wheel walk (0 = segment words / 6) */
#define SIEVE_PARAM_BATCH_ORDER   13 /* sieve_batch_count launches the ranges in the given order
                                        (0, default), heaviest first by estimated work (1), or
                                        heaviest and lightest alternating (2); results are the same */
#define SIEVE_PARAM_FAULT_WAIT    14 /* test hook: 1 = synchronous calls report the failure of a
                                        device-side wait (SIEVE_EDEVICE) after their launch, as the
                                        sieve does when a bounded wait in a kernel runs out */
#define SIEVE_PARAM_PRESIEVE      15 /* mod-30 kernels: largest prime whose multiples come from
                                        pre-sieved patterns ANDed into each segment instead of being
                                        crossed: 19 (one pattern, 7..19), 59 (default: three further
                                        patterns, 23..31, 37..43 and 47..59) or 71 (a fourth, 61..71);
                                        results are the same */
#define SIEVE_PARAM_CURSOR_MB     7 /* device memory (MiB) for per-CTA wheel cursors of the large
                                       primes, carried across the segments of a work item; used
                                       when they fit and enough segments resume one (half of a
                                       single range's, three quarters of a batch's) (default
                                       1024; 0 = recompute per segment) */

/* Set a launch parameter for later calls on ctx (SIEVE_EINVAL if out of range). */
int sieve_set_param(sieve_ctx *ctx, int param, int64_t value);
/* Read a launch parameter into *value. */
int sieve_get_param(sieve_ctx *ctx, int param, int64_t *value);

/* Facts about the context: base prime count and limit, SM count. */
typedef struct {
    uint64_t hi_max;
    uint64_t prime_limit;   /* floor(sqrt(hi_max - 1)) */
    uint64_t n_base_primes; /* primes <= prime_limit, 2 included */
    int32_t device;
    int32_t num_sms;
    uint64_t device_bytes;  /* device memory the context holds */
} sieve_info;

int sieve_get_info(sieve_ctx *ctx, sieve_info *info);

/*
 * Copy the context's resident base primes (ascending uint32, 2 first) to the
 * host array out[0 .. min(cap, n)); *n receives their number.
 */
int sieve_base_primes(sieve_ctx *ctx, uint32_t *out, size_t cap, uint64_t *n);

/*
 * Self-test of the bounded device-side wait the sieve uses for its bulk
 * shared-memory copies: one CTA waits on an mbarrier for at most `limit` polls.
 * With arm != 0 a 4 KB bulk copy completes the barrier (*timed_out = 0); with
 * arm == 0 nothing does, the wait runs out and *timed_out = 1 -- the kernel
 * returns normally and the context stays usable.  SIEVE_EINVAL for limit 0.
 */
int sieve_selftest_wait(sieve_ctx *ctx, int arm, uint32_t limit, int *timed_out);

/*
 * Exact number of bit-clears the crossing-off loop performs for [lo, hi):
 * the multiples p*m in [lo, hi) with p a base prime >= 23, m >= p and m
 * coprime to 30 (the mod-30 wheel after the pre-sieve of 7..19), or coprime
 * to 210 when SIEVE_PARAM_WHEEL is 210 (the count path's wheel).  Host-only
 * arithmetic; this is the algorithmic work used as a roofline numerator.
 */
int sieve_crossing_work(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *clears);

/*
 * As sieve_crossing_work, counting only the base primes p >= pmin (pmin <= 23
 * gives sieve_crossing_work).  With pmin = 61 on the mod-30 wheel it is the
 * clears left to the crossing loop's atomics after the further pre-sieved
 * patterns of 23..59 (SIEVE_PARAM_PRESIEVE = 59) have made the others.
 */
int sieve_crossing_work_ge(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t pmin, uint64_t *clears);

/*
 * Roofline probes: what this GPU sustains for the operations the sieve's
 * kernels are bound by, so that their rates can be set against a measured
 * ceiling.  The paper has no counterpart (it reports no hardware rates).
 * Runs on the context's stream and returns when done; *value receives:
 *  - SIEVE_PROBE_SMEM_AND_CONFLICT_FREE: shared-memory atomicAnd, lane l of
 *    every warp always on bank l, in lane-operations per SM clock (one CTA
 *    of 1024 threads per SM, timed with clock64, so clock-independent);
 *  - SIEVE_PROBE_SMEM_AND_RANDOM: the same on pseudo-random words (bank
 *    conflicts as they fall), lane-operations per SM clock;
 *  - SIEVE_PROBE_SMEM_STORE_CONFLICT_FREE: plain 32-bit stores, lane l on
 *    bank l, lane-operations per SM clock;
 *  - SIEVE_PROBE_HBM_WRITE: write-only HBM bandwidth in GB/s (10^9 B/s),
 *    16-byte stores over buf_dev[0 .. bytes) (device memory of the caller,
 *    16-byte aligned, at least 1 MiB; use more than the 129 MB L2), best of
 *    five timed passes after a warm-up.
 * buf_dev and bytes are ignored by the shared-memory probes.  The probes
 * allocate a few bytes of device memory for their results.
 */
#define SIEVE_PROBE_SMEM_AND_CONFLICT_FREE   1
#define SIEVE_PROBE_SMEM_AND_RANDOM          2
#define SIEVE_PROBE_SMEM_STORE_CONFLICT_FREE 3
#define SIEVE_PROBE_HBM_WRITE                4
int sieve_probe(sieve_ctx *ctx, int kind, void *buf_dev, uint64_t bytes, double *value);

/* The context's CUDA stream (a cudaStream_t) -- for event timing by callers. */
void *sieve_stream(sieve_ctx *ctx);

/* Static name of an error code. */
const char *sieve_strerror(int code);

/* The context's last error message ("" if none), copied under the context's
 * lock into a buffer of the calling thread, valid until that thread's next
 * call of this function (safe while a server runs on the context). */
const char *sieve_last_error(sieve_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* GBSIEVE_H */
