// sieve_api.cu -- host side of gbsieve: the context (resident base primes,
// pattern tile, scratch), range planning, launches and the C ABI of
// include/gbsieve.h.
//
// Base primes (Section 1's sqrt bound) are made on the device in three
// stages, each using the sieve itself: primes < 256 by trial division, then
// primes <= min(limit, 65535) by sieving with those, then primes <= limit
// (limit = floor(sqrt(hi_max - 1)) <= 2^31) by sieving with the primes below
// 65536.  Every stage's output is a list made by the compaction kernels.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "host.h"

using namespace gbs;

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
    } while (0)

namespace gbs {

namespace {
const char *kNames[] = {"ok", "invalid argument", "range exceeds limit", "output truncated",
                        "out of memory", "CUDA error", "timed out", "busy", "unknown ticket",
                        "device-side limit hit"};
}  // namespace

int fail(sieve_ctx *c, int code, const std::string &msg) {
    if (c) {
        std::lock_guard<std::mutex> lk(c->err_mu);
        std::snprintf(c->last_error, sizeof c->last_error, "%s", msg.c_str());
    }
    return code;
}

int cuda_fail(sieve_ctx *c, cudaError_t e, const char *where) {
    cudaGetLastError();  // clear a non-sticky launch error
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(c, SIEVE_ENOMEM, m);
    return fail(c, SIEVE_ECUDA, m);
}

// floor(sqrt(n)) for n < 2^64: the double square root is within one of it,
// then exact integer corrections (r < 2^32, so (r + 1)^2 does not overflow
// below 2^64 - 2^33).
uint64_t isqrt64(uint64_t n) {
    uint64_t r = (uint64_t)std::sqrt((double)n);
    if (r > 0xffffffffull) r = 0xffffffffull;
    while (r * r > n) --r;
    while (r < 0xffffffffull && (r + 1) * (r + 1) <= n) ++r;
    return r;
}

uint64_t bitmap_words_of(uint64_t lo, uint64_t hi) {
    uint64_t o0 = lo | 1;
    if (o0 >= hi) return 0;
    uint64_t nbits = (hi - o0 + 1) / 2;
    return (nbits + 31) / 32;
}

namespace {

// Number of base primes p with p * p < hi, i.e. p <= floor(sqrt(hi - 1)).
// Base primes p <= sqrt(hi - 1): a binary search inside the bucket of 1024
// integers that holds the bound (ctx->h_prime_bucket[b] = index of the first
// base prime >= 1024 b).
uint32_t primes_needed(const sieve_ctx *ctx, uint64_t hi) {
    if (hi < 2) return 0;
    const std::vector<uint32_t> &primes = ctx->h_primes;
    const std::vector<uint32_t> &bucket = ctx->h_prime_bucket;
    const uint64_t lim = isqrt64(hi - 1);
    auto first = primes.begin(), last = primes.end();
    if (!bucket.empty()) {
        const uint64_t b = lim / 1024;
        if (b + 1 < bucket.size()) {
            first = primes.begin() + bucket[b];
            last = primes.begin() + bucket[b + 1];
        } else {
            first = primes.begin() + bucket.back();
        }
    }
    return (uint32_t)(std::upper_bound(first, last, lim, [](uint64_t v, uint32_t p) { return v < p; }) -
                      primes.begin());
}

// Index of the first prime >= limit, at least the first crossing prime.
uint32_t first_at_least(const std::vector<uint32_t> &primes, uint64_t limit) {
    if (limit > 0xffffffffull) return (uint32_t)primes.size();
    uint32_t e = (uint32_t)(std::lower_bound(primes.begin(), primes.end(), (uint32_t)limit) - primes.begin());
    return std::max<uint32_t>(e, kFirstCrossingPrime);
}

template <typename T>
int dev_alloc(sieve_ctx *ctx, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    *p = static_cast<T *>(q);
    ctx->device_bytes += std::max<size_t>(count, 1) * sizeof(T);
    return SIEVE_OK;
}

template <typename T>
void dev_free(sieve_ctx *ctx, T *&p, size_t count) {
    if (p) {
        cudaFree(p);
        ctx->device_bytes -= std::max<size_t>(count, 1) * sizeof(T);
    }
    p = nullptr;
}

void drop_graphs(sieve_ctx *ctx) {
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second);
    ctx->graphs.clear();
}

}  // namespace

int alloc_launch_buffers(sieve_ctx *ctx, LaunchBuffers &lb, size_t m) {
    if (m <= lb.cap) return SIEVE_OK;
    free_launch_buffers(ctx, lb);
    const size_t cap = std::max<size_t>(m, 64);
    const size_t block = LaunchBuffers::block_bytes(cap);
    int rc = dev_alloc(ctx, &lb.d_block, block);
    if (rc) return rc;
    rc = dev_alloc(ctx, &lb.d_acc, cap + 2);
    if (rc) return rc;
    CK(cudaMallocHost(&lb.h_block, block));
    CK(cudaMallocHost(&lb.h_acc, (cap + 2) * sizeof(unsigned long long)));
    CK(cudaEventCreateWithFlags(&lb.consumed, cudaEventDisableTiming));
    lb.cap = cap;
    return SIEVE_OK;
}

void free_launch_buffers(sieve_ctx *ctx, LaunchBuffers &lb) {
    const size_t block = LaunchBuffers::block_bytes(lb.cap);
    if (lb.d_block) dev_free(ctx, lb.d_block, block);
    if (lb.d_acc) dev_free(ctx, lb.d_acc, lb.cap + 2);
    if (lb.h_block) cudaFreeHost(lb.h_block);
    if (lb.h_acc) cudaFreeHost(lb.h_acc);
    if (lb.consumed) cudaEventDestroy(lb.consumed);
    lb = LaunchBuffers();
}

int block_wait(sieve_ctx *ctx, LaunchBuffers &lb) {
    if (lb.consumed) CK(cudaEventSynchronize(lb.consumed));
    return SIEVE_OK;
}

// The first bytes of lb's pinned block to the device and its accumulators
// [0, acc_n) zeroed.  Outside a graph capture a block of at most kUploadMaxBytes
// goes as a kernel parameter (one launch instead of a copy and a memset; the
// host block is free again at once).  Otherwise it is copied, and an event marks
// when the copy has run (not inside a capture, whose copies run at replay, after
// which the caller synchronises).  extra: the Miller-Rabin lists (n_list
// entries) are copied too.
static int upload_block(sieve_ctx *ctx, LaunchBuffers &lb, size_t bytes, size_t acc_n, size_t n_list,
                        cudaStream_t stream) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(stream, &st));
    const bool capturing = st != cudaStreamCaptureStatusNone;
    if (!capturing && !n_list && bytes <= kUploadMaxBytes) {
        CK(launch_upload(lb.d_block, lb.h_block, bytes, lb.d_acc, acc_n, stream));
        return SIEVE_OK;
    }
    CK(cudaMemcpyAsync(lb.d_block, lb.h_block, bytes, cudaMemcpyHostToDevice, stream));
    if (n_list) {
        CK(cudaMemcpyAsync(lb.d_mr(), lb.h_mr(), n_list * sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
        CK(cudaMemcpyAsync(lb.d_mrw(), lb.h_mrw(), (n_list + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
    }
    if (!capturing && lb.consumed) CK(cudaEventRecord(lb.consumed, stream));
    CK(cudaMemsetAsync(lb.d_acc, 0, acc_n * sizeof(unsigned long long), stream));
    return SIEVE_OK;
}

int alloc_compact_scratch(sieve_ctx *ctx, CompactScratch &cs, size_t tiles) {
    if (!cs.d_total) {
        int rc = dev_alloc(ctx, &cs.d_total, 1);
        if (rc) return rc;
        CK(cudaMallocHost(&cs.h_total, sizeof(unsigned long long)));
    }
    if (tiles <= cs.cap) return SIEVE_OK;
    dev_free(ctx, cs.counts, cs.cap);
    dev_free(ctx, cs.offsets, cs.cap);
    dev_free(ctx, cs.status, cs.cap + 1);
    cs.cap = 0;
    int rc = dev_alloc(ctx, &cs.counts, tiles);
    if (rc) return rc;
    rc = dev_alloc(ctx, &cs.offsets, tiles);
    if (rc) return rc;
    rc = dev_alloc(ctx, &cs.status, tiles + 1);
    if (rc) return rc;
    cs.cap = tiles;
    return SIEVE_OK;
}

void free_compact_scratch(sieve_ctx *ctx, CompactScratch &cs) {
    dev_free(ctx, cs.counts, cs.cap);
    dev_free(ctx, cs.offsets, cs.cap);
    dev_free(ctx, cs.status, cs.cap + 1);
    dev_free(ctx, cs.d_total, 1);
    if (cs.h_total) cudaFreeHost(cs.h_total);
    cs = CompactScratch();
}

// Fill one RangeDesc (item_first is set at launch).  Segments start at a wheel
// byte Bbase with 30 Bbase <= lo and 30 Bbase + 1 = (lo | 1) (mod 64).
// Whether per-CTA cursors pay for themselves with chunks of C segments: they
// save the start computation of every large prime in every segment of a chunk
// but its first, and cost their stores and coarser work items.  Measured: a
// single range gains from half its segments resuming (at 10^14: 18 % with half,
// 35 % with 94 %); a batch of mostly one-segment ranges loses (9 % with 49 %),
// so batches need three quarters.
bool cursors_pay(const RangeDesc *rd, size_t m, uint32_t C, uint64_t segs) {
    if (C < 2 || segs == 0) return false;
    uint64_t resumes = 0;
    for (size_t i = 0; i < m; ++i) resumes += rd[i].nseg - (rd[i].nseg + C - 1) / C;
    return m == 1 ? 2 * resumes >= segs : 4 * resumes >= 3 * segs;
}

RangeDesc plan_range(const sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t seg_bytes, int mode,
                     uint32_t *bitmap) {
    RangeDesc r;
    std::memset(&r, 0, sizeof r);
    r.lo = lo;
    r.hi = hi;
    r.bitmap = bitmap;
    r.bitmap_words = bitmap_words_of(lo, hi);
    if (lo >= hi) return r;
    const uint64_t o0 = lo | 1;
    // t0 = 0 (mod 30) and t0 = o0 - 1 (mod 64): t0 = 30 x with 15 x = (o0 - 1) / 2 (mod 32),
    // and 15 is its own inverse mod 32.
    const uint64_t a = ((o0 - 1) & 63) / 2;
    const int64_t t0_res = 30 * (int64_t)((15 * a) & 31);  // residue of t0 mod 960
    int64_t diff = ((int64_t)(lo % 960) - t0_res) % 960;
    if (diff < 0) diff += 960;
    const int64_t t0 = (int64_t)lo - diff;  // >= -930
    r.Bbase = t0 / 30;
    r.bucket_first = 0xffffffffu;
    const uint64_t span = 30ull * seg_bytes;
    r.nseg = (uint64_t)(((int64_t)hi - t0 + (int64_t)span - 1) / (int64_t)span);
    r.n_use = primes_needed(ctx, hi);
    r.seg_bytes = seg_bytes;
    uint64_t corr = (lo <= 2 && 2 < hi) ? 1 : 0;
    if (mode == kModeCount) corr += (lo <= 3 && 3 < hi ? 1 : 0) + (lo <= 5 && 5 < hi ? 1 : 0);
    r.corr = corr;
    return r;
}

int prepare_launch(sieve_ctx *ctx, const Params &prm, int mode, LaunchBuffers &lb, size_t m, BucketStore *bs,
                   CursorStore *cs, uint64_t *items_out, const RangeOverride *ro) {
    const std::vector<uint32_t> &h = ctx->h_primes;
    RangeDesc *rd = lb.h_ranges();
    uint64_t segs = 0;
    uint32_t nmax = 0, smax = 0;
    for (size_t i = 0; i < m; ++i) {
        segs += rd[i].nseg;
        if (rd[i].nseg) nmax = std::max(nmax, rd[i].n_use);
        smax = std::max(smax, rd[i].seg_bytes);
    }
    if (!smax) smax = prm.seg_bytes;
    const uint64_t grid = (uint64_t)ctx->num_sms * prm.ctas_per_sm;
    const uint32_t small_end = first_at_least(h, prm.small_limit);
    // Per range: per-phase sub-progressions for primes below S / 3 (about three hits
    // per progression in a full segment; measured best on pi(10^12) among S / 8 ..
    // S / 2.8), and bucket lists from the bucket limit on (never below the walk tier).
    // A range of one segment shorter than S takes a third of its own length: above
    // it a prime has few hits there, and the walk visits only those, while the
    // per-phase tier sets up every class of every prime for each segment.
    uint32_t mid_lo = 0xffffffffu, mid_hi = small_end, bfirst = 0xffffffffu;
    for (size_t i = 0; i < m; ++i) {
        const uint32_t ml = ro && ro[i].mid_limit ? ro[i].mid_limit : prm.mid_limit;
        uint32_t len = rd[i].seg_bytes;
        if (rd[i].nseg == 1) {  // wheel bytes from the grid origin to hi
            const int64_t ints = (int64_t)rd[i].hi - 30 * rd[i].Bbase;
            len = (uint32_t)std::min<int64_t>(len, std::max<int64_t>((ints + 29) / 30, 1));
        }
        const uint32_t mid_lim = ml ? ml : std::max<uint32_t>(len / 3, 23);
        rd[i].mid_end = std::max(small_end, first_at_least(h, mid_lim));
        const uint64_t bl = ro && ro[i].bucket_limit ? ro[i].bucket_limit : prm.bucket_limit;
        const uint32_t bf = std::max(first_at_least(h, bl ? bl : rd[i].seg_bytes), rd[i].mid_end);
        rd[i].bucket_first = bs && rd[i].nseg && bf < rd[i].n_use ? bf : 0xffffffffu;
        if (!rd[i].nseg) continue;
        mid_lo = std::min(mid_lo, rd[i].mid_end);
        mid_hi = std::max(mid_hi, rd[i].mid_end);
        bfirst = std::min(bfirst, rd[i].bucket_first);
    }
    if (mid_lo == 0xffffffffu) mid_lo = mid_hi;
    const bool buckets = bfirst != 0xffffffffu;
    // Per-CTA cursors for the large primes (4 B each) when they fit the budget
    // and every offset fits 29 bits (p < 2^27); not with bucket lists.  A range's
    // cursors are indexed from its own walk tier start, never below mid_lo.
    const uint32_t n_large = nmax > mid_lo ? nmax - mid_lo : 0;
    bool cursors = cs && !buckets && n_large && h[nmax - 1] < (1u << 27) &&
                   (uint64_t)grid * n_large * 4 <= (uint64_t)prm.cursor_mb << 20;
    // Chunks (several segments per work item) pay off with bucket lists and
    // cursors; keep at least 4 items per CTA so the last wave stays short.
    uint32_t C = prm.chunk_segs;
    while (C > 1 && segs / C < 4 * grid) C /= 2;
    if (cursors && !cursors_pay(rd, m, C, segs)) cursors = false;
    if (!buckets && !cursors) C = 1;
    uint64_t items = 0;
    for (size_t i = 0; i < m; ++i) {
        rd[i].item_first = items;
        items += (rd[i].nseg + C - 1) / C;
    }
    // Miller-Rabin path for narrow ranges high up: sieving with the primes below
    // 2^16 and testing the survivors (about 5 % of the integers, each some 10^4
    // instructions when prime) beats visiting every base prime (about 100
    // instructions each) when the width is below mr_percent % of the primes
    // that would be skipped.
    // Such a range is one segment long; a count-mode one keeps its raw wheel
    // words (and a bitmap-mode one without an output its odd-only words) in
    // scratch for k_mr_filter.
    const uint32_t mr_end = first_at_least(h, 65536);
    const uint64_t mr_square = mr_end < h.size() ? (uint64_t)h[mr_end] * h[mr_end] : ~0ull;
    uint32_t n_mr = 0;
    size_t scratch_words = 0;
    std::vector<size_t> scratch_at;
    for (size_t i = 0; i < m; ++i) {
        rd[i].mr = 0;
        const uint32_t mrp = !ro || !ro[i].mr_percent ? prm.mr_percent
                             : ro[i].mr_percent == 0xffffffffu ? 0u : ro[i].mr_percent;
        if (mrp && rd[i].nseg == 1 && rd[i].n_use > mr_end && rd[i].hi > mr_square &&
            (rd[i].hi - rd[i].lo) * 100 < (uint64_t)mrp * (rd[i].n_use - mr_end)) {
            rd[i].mr = 1;
            lb.h_mr()[n_mr++] = (uint32_t)i;
            if (mode == kModeCount) {  // raw wheel words of the one segment
                const int64_t need = (((int64_t)rd[i].hi - 30 * rd[i].Bbase + 29) / 30 + 31) & ~31ll;
                scratch_at.push_back(scratch_words);
                scratch_words += (size_t)need / 4;
            } else if (!rd[i].bitmap) {
                scratch_at.push_back(scratch_words);
                scratch_words += rd[i].bitmap_words;
            } else {
                scratch_at.push_back(~(size_t)0);
            }
        }
    }
    if (scratch_words > ctx->mr.words) {
        dev_free(ctx, ctx->mr.d, ctx->mr.words);
        ctx->mr.words = 0;
        int rc = dev_alloc(ctx, &ctx->mr.d, std::max<size_t>(scratch_words, 1 << 16));
        if (rc) return rc;
        ctx->mr.words = std::max<size_t>(scratch_words, 1 << 16);
    }
    for (uint32_t q = 0; q < n_mr; ++q)
        if (scratch_at[q] != ~(size_t)0) rd[lb.h_mr()[q]].bitmap = ctx->mr.d + scratch_at[q];
    // prefix sums of the words the Miller-Rabin filter scans (raw wheel words in count
    // mode, odd-only words in bitmap mode), one thread per word
    {
        uint32_t *pw = lb.h_mrw();
        uint64_t acc = 0;
        for (uint32_t q = 0; q < n_mr; ++q) {
            pw[q] = (uint32_t)acc;
            const RangeDesc &r = rd[lb.h_mr()[q]];
            acc += mode == kModeCount ? (uint64_t)((((int64_t)r.hi - 30 * r.Bbase + 29) / 30 + 31) & ~31ll) / 4
                                      : r.bitmap_words;
        }
        pw[n_mr] = (uint32_t)acc;
    }
    SieveLaunch &L = *reinterpret_cast<SieveLaunch *>(lb.h_block);
    std::memset(&L, 0, sizeof L);
    L.ranges = lb.d_ranges();
    L.n_ranges = (uint32_t)m;
    L.n_items = items;
    L.item_counter = lb.d_acc;
    L.counts = lb.d_acc + 1;
    L.overflow = reinterpret_cast<unsigned *>(lb.d_acc + m + 1);
    L.primes = ctx->d_primes;
    L.magic = ctx->d_magic;
    L.tile = ctx->d_tile;
    L.tile_stride = ctx->tile_stride;
    if (prm.presieve >= 59) {
        L.xtile0 = ctx->d_tile + ctx->tile_stride * kTileCopies;
        L.xtile1 = L.xtile0 + kXTileStride0 * kTileCopies;
        L.xtile2 = L.xtile1 + kXTileStride1 * kTileCopies;
        L.small_first = kFirstCrossingPrimeX;
        if (prm.presieve == 71) {
            L.xtile3 = L.xtile2 + kXTileStride2 * kTileCopies;
            L.small_first = kFirstCrossingPrimeX4;
        }
    } else {
        L.small_first = kFirstCrossingPrime;
    }
    L.seg_bytes = smax;
    L.chunk_segs = C;
    L.small_end = small_end;
    L.mid_end = mid_hi;
    L.mr_end = mr_end;
    L.mr_square = mr_square;
    L.mr_list = lb.d_mr();
    L.mr_words = lb.d_mrw();
    L.n_mr = n_mr;
    L.bucket_first = bfirst;
    if (buckets) {
        // expected hits per full segment: 8 S / p per bucket prime (one per wheel
        // class with probability S / p); the list capacity is that with a margin,
        // for the largest segment and the earliest bucket start of the launch
        double e = 0;
        for (uint32_t i = bfirst; i < nmax; ++i) e += 8.0 * smax / h[i];
        uint64_t cap = (uint64_t)(bs->slack * e) + 4096;
        cap = (cap + 31) & ~31ull;
        const size_t need = (size_t)grid * C * cap;
        if (need > bs->entries) {
            dev_free(ctx, bs->d, bs->entries);
            bs->entries = 0;
            int rc = dev_alloc(ctx, &bs->d, need);
            if (rc) return rc;
            bs->entries = need;
        }
        L.buckets = bs->d;
        L.bucket_cap = (uint32_t)cap;
    }
    if (cursors && C > 1) {
        const size_t need = (size_t)grid * n_large;
        if (need > cs->entries) {
            dev_free(ctx, cs->d, cs->entries);
            cs->entries = 0;
            int rc = dev_alloc(ctx, &cs->d, need);
            if (rc) return rc;
            cs->entries = need;
        }
        L.cursors = cs->d;
        L.cursor_stride = n_large;
    }
    *items_out = items;
    return SIEVE_OK;
}

// grid: sieve CTAs (0: no sieve launch); mr_grid: Miller-Rabin CTAs (0: none);
// n_list: entries of the Miller-Rabin list to copy.
int enqueue_launch(sieve_ctx *ctx, cudaStream_t stream, const Params &prm, int mode, LaunchBuffers &lb, size_t m,
                   int grid, int mr_grid, size_t n_list) {
    int rc = upload_block(ctx, lb, kLaunchHeader + m * sizeof(RangeDesc), m + 2, n_list, stream);
    if (rc) return rc;
    const SieveLaunch *d = reinterpret_cast<const SieveLaunch *>(lb.d_block);
    const uint32_t smem = reinterpret_cast<const SieveLaunch *>(lb.h_block)->seg_bytes;  // the largest segment
    if (grid > 0) CK(launch_sieve(mode, d, grid, prm.threads, smem, stream));
    if (mr_grid > 0) CK(launch_mr_filter(mode, d, mr_grid, stream));
    return SIEVE_OK;
}

int launch_ranges(sieve_ctx *ctx, cudaStream_t stream, const Params &prm, int mode, LaunchBuffers &lb, size_t m,
                  BucketStore *bs, CursorStore *cs, const RangeOverride *ro) {
    uint64_t items = 0;
    int rc = prepare_launch(ctx, prm, mode, lb, m, bs, cs, &items, ro);
    if (rc) return rc;
    const uint64_t grid = (uint64_t)ctx->num_sms * prm.ctas_per_sm;
    const uint32_t n_mr = reinterpret_cast<const SieveLaunch *>(lb.h_block)->n_mr;
    return enqueue_launch(ctx, stream, prm, mode, lb, m, (int)std::min<uint64_t>(grid, items),
                          n_mr ? 8 * ctx->num_sms : 0, n_mr);
}

// Segment size of the mod-210 count path: the configured segment rounded down
// to a multiple of 3 words (2 whole groups per 3 words).
uint32_t w210_segment_words(const Params &prm) {
    const uint32_t w = std::min(prm.seg_bytes, kW210MaxSegmentBytes) / 4;
    return std::max<uint32_t>(w / 3 * 3, 3);
}

// One range on the mod-210 wheel: segments start at group lo / 210.
RangeDesc plan_range210(const sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t seg_words) {
    RangeDesc r;
    std::memset(&r, 0, sizeof r);
    r.lo = lo;
    r.hi = hi;
    if (lo >= hi) return r;
    r.Bbase = (int64_t)(lo / 210);
    const uint64_t span = 210ull * (seg_words / 3 * 2);
    r.nseg = (hi - 210ull * (uint64_t)r.Bbase + span - 1) / span;
    r.n_use = primes_needed(ctx, hi);
    r.seg_bytes = 4 * seg_words;
    r.bucket_first = 0xffffffffu;
    for (uint64_t q : {2, 3, 5, 7}) r.corr += lo <= q && q < hi;
    return r;
}

// Plan a count-only launch of the m ranges in lb on the mod-210 wheel (no
// bucket lists, no Miller-Rabin path): fills the launch header; *items_out is
// the number of work items.
int prepare_launch210(sieve_ctx *ctx, const Params &prm, LaunchBuffers &lb, size_t m, CursorStore *cs,
                      uint64_t *items_out, const RangeOverride *ro) {
    const std::vector<uint32_t> &h = ctx->h_primes;
    RangeDesc *rd = lb.h_ranges();
    uint64_t segs = 0;
    uint32_t nmax = 0, smax = 0;
    for (size_t i = 0; i < m; ++i) {
        segs += rd[i].nseg;
        if (rd[i].nseg) nmax = std::max(nmax, rd[i].n_use);
        smax = std::max(smax, rd[i].seg_bytes);
    }
    if (!smax) smax = 4 * w210_segment_words(prm);
    const uint64_t grid = (uint64_t)ctx->num_sms * prm.ctas_per_sm;
    const uint32_t small_end = std::max(kFirstCrossingPrime, first_at_least(h, prm.small_limit210));
    // per range: primes below words / 6 have at least two hits per sub-progression in
    // a full segment
    uint32_t mid_lo = 0xffffffffu, mid_hi = small_end;
    for (size_t i = 0; i < m; ++i) {
        const uint32_t ml = ro && ro[i].mid_limit ? ro[i].mid_limit : prm.mid_limit210;
        const uint32_t mid_lim = ml ? ml : std::max<uint32_t>(rd[i].seg_bytes / 4 / 6, 23);
        rd[i].mid_end = std::max(small_end, first_at_least(h, mid_lim));
        rd[i].bucket_first = 0xffffffffu;
        if (!rd[i].nseg) continue;
        mid_lo = std::min(mid_lo, rd[i].mid_end);
        mid_hi = std::max(mid_hi, rd[i].mid_end);
    }
    if (mid_lo == 0xffffffffu) mid_lo = mid_hi;
    const uint32_t n_large = nmax > mid_lo ? nmax - mid_lo : 0;
    bool cursors = cs && n_large && h[nmax - 1] < (1u << 27) &&
                   (uint64_t)grid * n_large * 4 <= (uint64_t)prm.cursor_mb << 20;
    uint32_t C = prm.chunk_segs;
    while (C > 1 && segs / C < 4 * grid) C /= 2;
    if (cursors && !cursors_pay(rd, m, C, segs)) cursors = false;
    if (!cursors) C = 1;
    uint64_t items = 0;
    for (size_t i = 0; i < m; ++i) {
        rd[i].item_first = items;
        items += (rd[i].nseg + C - 1) / C;
    }
    SieveLaunch &L = *reinterpret_cast<SieveLaunch *>(lb.h_block);
    std::memset(&L, 0, sizeof L);
    L.ranges = lb.d_ranges();
    L.n_ranges = (uint32_t)m;
    L.n_items = items;
    L.item_counter = lb.d_acc;
    L.counts = lb.d_acc + 1;
    L.overflow = reinterpret_cast<unsigned *>(lb.d_acc + m + 1);
    L.primes = ctx->d_primes;
    L.magic = ctx->d_magic;
    L.seg_bytes = smax;
    L.small_first = kFirstCrossingPrime;
    L.chunk_segs = C;
    L.small_end = small_end;
    L.mid_end = mid_hi;
    L.bucket_first = 0xffffffffu;
    if (cursors && C > 1) {
        const size_t need = (size_t)grid * n_large;
        if (need > cs->entries) {
            dev_free(ctx, cs->d, cs->entries);
            cs->entries = 0;
            int rc = dev_alloc(ctx, &cs->d, need);
            if (rc) return rc;
            cs->entries = need;
        }
        L.cursors = cs->d;
        L.cursor_stride = n_large;
    }
    *items_out = items;
    return SIEVE_OK;
}

// Block copy, accumulator clear and the mod-210 sieve over `grid` CTAs.
int enqueue_launch210(sieve_ctx *ctx, cudaStream_t stream, const Params &prm, LaunchBuffers &lb, size_t m, int grid) {
    int rc = upload_block(ctx, lb, kLaunchHeader + m * sizeof(RangeDesc), m + 2, 0, stream);
    if (rc) return rc;
    const uint32_t smem = (reinterpret_cast<const SieveLaunch *>(lb.h_block)->seg_bytes + 15) & ~15u;
    if (grid > 0)
        CK(launch_sieve210(reinterpret_cast<const SieveLaunch *>(lb.d_block), ctx->d_tab210, ctx->d_tile210,
                           ctx->tile210_stride, grid, prm.threads, smem, stream));
    return SIEVE_OK;
}

int launch_ranges210(sieve_ctx *ctx, cudaStream_t stream, const Params &prm, LaunchBuffers &lb, size_t m,
                     CursorStore *cs, const RangeOverride *ro) {
    uint64_t items = 0;
    int rc = prepare_launch210(ctx, prm, lb, m, cs, &items, ro);
    if (rc) return rc;
    const uint64_t grid = (uint64_t)ctx->num_sms * prm.ctas_per_sm;
    return enqueue_launch210(ctx, stream, prm, lb, m, (int)std::min<uint64_t>(grid, items));
}

// Compaction without the host read of the total: the count goes to the device
// integer *n_dev and nothing waits for the stream.  A list is written in one pass
// (tile offsets by decoupled look-back), truncated at cap; a size query (no
// output) takes the popcount and scan kernels.
int compact_async(sieve_ctx *ctx, cudaStream_t stream, CompactScratch &cs, const uint32_t *bitmap_dev, uint64_t lo,
                  uint64_t hi, void *out_dev, size_t cap, uint64_t *n_dev, int out64) {
    const uint64_t nwords = bitmap_words_of(lo, hi);
    const uint32_t two = (lo <= 2 && 2 < hi) ? 1 : 0;
    const uint64_t ntiles = (nwords + kCompactTileWords - 1) / kCompactTileWords;
    int rc = alloc_compact_scratch(ctx, cs, ntiles);
    if (rc) return rc;
    if (ntiles) {
        if (out_dev) {  // also the prime 2 and the count
            CK(cudaMemsetAsync(cs.status, 0, (ntiles + 1) * sizeof(unsigned long long), stream));
            CK(launch_emit_onepass(bitmap_dev, nwords, ntiles, lo | 1, two, out_dev, out64, ctx->num_sms, stream, cap,
                                   2, cs.status, n_dev));
        } else {
            CK(launch_tile_popc(bitmap_dev, nwords, cs.counts, ntiles, ctx->num_sms * 8, stream));
            CK(launch_tile_scan(cs.counts, cs.offsets, ntiles, cs.d_total, stream));
            CK(launch_store_count(cs.d_total, two, n_dev, stream));
        }
        return SIEVE_OK;
    }
    // no odd integer in the range: the list is [2] or empty
    if (two && cap) CK(launch_put_two(out_dev, out64, stream));
    CK(launch_store_count(nullptr, two, n_dev, stream));
    return SIEVE_OK;
}

int compact_with(sieve_ctx *ctx, cudaStream_t stream, CompactScratch &cs, const uint32_t *bitmap_dev, uint64_t lo,
                 uint64_t hi, void *out_dev, size_t cap, uint64_t *n, int out64, uint64_t sub) {
    if (!out_dev && cap) return fail(ctx, SIEVE_EINVAL, "null output with a nonzero capacity");
    const uint64_t nwords = bitmap_words_of(lo, hi);
    const uint32_t two = (lo <= 2 && 2 < hi) ? 1 : 0;
    const uint64_t ntiles = (nwords + kCompactTileWords - 1) / kCompactTileWords;
    int rc = alloc_compact_scratch(ctx, cs, ntiles);
    if (rc) return rc;
    uint64_t total = 0;
    const int grid = ctx->num_sms * 8;
    if (ntiles) {
        // popcounts, scan, then the list itself, all enqueued at once: the emitting
        // kernels read the total on the device and write only if the list fits in cap
        CK(launch_tile_popc(bitmap_dev, nwords, cs.counts, ntiles, grid, stream));
        CK(launch_tile_scan(cs.counts, cs.offsets, ntiles, cs.d_total, stream));
        if (out_dev) {
            CK(launch_emit(bitmap_dev, nwords, cs.offsets, ntiles, (lo | 1) - sub, two, out_dev, out64,
                           ctx->num_sms, stream, cs.d_total, cap, 2 - sub));
        }
        CK(cudaMemcpyAsync(cs.h_total, cs.d_total, sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        total = *cs.h_total;
    }
    *n = total + two;
    if (*n > cap) return fail(ctx, SIEVE_ETRUNC, "output capacity below the prime count");  // nothing written
    if (*n == 0 || ntiles) return SIEVE_OK;
    // no odd integer in the range: the list is [2]
    CK(launch_put_two(out_dev, out64, stream, sub));
    CK(cudaStreamSynchronize(stream));
    return SIEVE_OK;
}

}  // namespace gbs

namespace {

// Copy the m counts and the flag word to lb.h_acc and wait; *overflowed = 1 if
// a bucket list overflowed (bit 0: the results are then invalid, a retry with
// larger lists helps); bit 1 is a wait that hit its limit in the kernel.
int finish(sieve_ctx *ctx, LaunchBuffers &lb, size_t m, int *overflowed) {
    CK(cudaMemcpyAsync(lb.h_acc, lb.d_acc + 1, (m + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if ((lb.h_acc[m] & 2ull) || ctx->params.fault_wait)
        return fail(ctx, SIEVE_EDEVICE, "a device-side wait hit its limit");
    *overflowed = (lb.h_acc[m] & 1ull) != 0;
    return SIEVE_OK;
}

// Launch parameters for one range [lo, hi).  When the range has at most 8 waves
// of full segments over the grid, the segment is shortened (in 32-byte steps,
// not below 4 KB) so that the segments fill whole waves: otherwise the last
// wave runs a few segments while the other CTAs wait.
Params single_range_params(const sieve_ctx *ctx, uint64_t lo, uint64_t hi) {
    Params p = ctx->params;
    if (hi <= lo) return p;
    const uint64_t grid = (uint64_t)ctx->num_sms * p.ctas_per_sm;
    const uint64_t bytes = (hi - lo) / 30 + 64;  // wheel bytes, plus the grid origin's slack
    const uint64_t n0 = (bytes + p.seg_bytes - 1) / p.seg_bytes;
    if (n0 > 8 * grid) return p;
    const uint64_t waves = (n0 + grid - 1) / grid;
    uint64_t sb = (bytes + waves * grid - 1) / (waves * grid);
    sb = std::max<uint64_t>((sb + 31) & ~31ull, 4096);
    if (sb < p.seg_bytes) p.seg_bytes = (uint32_t)sb;
    return p;
}

// launch + finish on the context's stream, re-running with larger bucket lists
// if one overflowed (never expected: the margin is far above the spread of the
// hit counts).  Counts are left in ctx->lb.h_acc[0..m).
int run_sync(sieve_ctx *ctx, const Params &prm, int mode, size_t m) {
    for (int attempt = 0; attempt < 4; ++attempt) {
        int rc = launch_ranges(ctx, ctx->stream, prm, mode, ctx->lb, m, &ctx->buckets, &ctx->cursors);
        if (rc) return rc;
        int of = 0;
        rc = finish(ctx, ctx->lb, m, &of);
        if (rc) return rc;
        if (!of) return SIEVE_OK;
        ctx->buckets.slack *= 2;
    }
    return fail(ctx, SIEVE_EDEVICE, "bucket lists overflowed repeatedly");
}

int ensure_bitmap(sieve_ctx *ctx, size_t words) {
    if (words <= ctx->bitmap_cap) return SIEVE_OK;
    dev_free(ctx, ctx->d_bitmap, ctx->bitmap_cap);
    ctx->bitmap_cap = 0;
    int rc = dev_alloc(ctx, &ctx->d_bitmap, words);
    if (rc) return rc;
    ctx->bitmap_cap = words;
    return SIEVE_OK;
}

// Every single-range and batched call writes the context's pinned launch block
// after this: it first waits until the block's last copy has run.
int ensure_launch(sieve_ctx *ctx, size_t m) {
    int rc = block_wait(ctx, ctx->lb);
    if (rc) return rc;
    if (m <= ctx->lb.cap) return SIEVE_OK;
    drop_graphs(ctx);  // they reference the old buffers
    return alloc_launch_buffers(ctx, ctx->lb, m);
}

// Sieve [0, limit + 1) into the scratch bitmap with the current base primes
// (they cover sqrt(limit)) and compact it into a fresh device array.
int primes_upto(sieve_ctx *ctx, uint64_t limit, uint32_t **out_dev, std::vector<uint32_t> &out_h) {
    const uint64_t hi = limit + 1;
    int rc = ensure_launch(ctx, 1);
    if (rc) return rc;
    rc = ensure_bitmap(ctx, bitmap_words_of(0, hi));
    if (rc) return rc;
    ctx->lb.h_ranges()[0] = plan_range(ctx, 0, hi, ctx->params.seg_bytes, kModeBitmap, ctx->d_bitmap);
    rc = run_sync(ctx, ctx->params, kModeBitmap, 1);
    if (rc) return rc;
    uint64_t n = 0;
    rc = compact_with(ctx, ctx->stream, ctx->cs, ctx->d_bitmap, 0, hi, nullptr, 0, &n, 0);
    if (rc != SIEVE_ETRUNC && rc != SIEVE_OK) return rc;
    uint32_t *d = nullptr;
    rc = dev_alloc(ctx, &d, n);
    if (rc) return rc;
    uint64_t n2 = 0;
    rc = compact_with(ctx, ctx->stream, ctx->cs, ctx->d_bitmap, 0, hi, d, n, &n2, 0);
    if (rc) {
        dev_free(ctx, d, n);
        return rc;
    }
    out_h.resize(n);
    CK(cudaMemcpy(out_h.data(), d, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    *out_dev = d;
    return SIEVE_OK;
}

int make_base_primes(sieve_ctx *ctx) {
    // stage 1: primes < 256 by trial division
    uint32_t *d_tiny = nullptr, *d_ntiny = nullptr;
    int rc = dev_alloc(ctx, &d_tiny, 64);
    if (rc) return rc;
    rc = dev_alloc(ctx, &d_ntiny, 1);
    if (rc) return rc;
    CK(launch_tiny_primes(d_tiny, d_ntiny, ctx->stream));
    uint32_t ntiny = 0;
    CK(cudaMemcpyAsync(&ntiny, d_ntiny, sizeof ntiny, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, d_ntiny, 1);
    ctx->h_primes.resize(ntiny);
    CK(cudaMemcpy(ctx->h_primes.data(), d_tiny, ntiny * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    ctx->d_primes = d_tiny;
    size_t cur_n = 64;
    rc = dev_alloc(ctx, &ctx->d_magic, cur_n);
    if (rc) return rc;
    CK(launch_magic(ctx->d_primes, ctx->d_magic, ctx->h_primes.size(), ctx->stream));

    // stages 2 and 3
    const uint64_t stages[2] = {std::min<uint64_t>(ctx->prime_limit, 65535), ctx->prime_limit};
    for (int st = 0; st < 2; ++st) {
        const uint64_t lim = stages[st];
        if (!ctx->h_primes.empty() && ctx->h_primes.back() >= lim) break;
        if (st == 1 && lim <= 65535) break;
        uint32_t *d_next = nullptr;
        std::vector<uint32_t> h_next;
        rc = primes_upto(ctx, lim, &d_next, h_next);
        if (rc) return rc;
        dev_free(ctx, ctx->d_primes, cur_n);
        dev_free(ctx, ctx->d_magic, cur_n);
        ctx->d_primes = d_next;
        cur_n = h_next.size();
        ctx->h_primes.swap(h_next);
        rc = dev_alloc(ctx, &ctx->d_magic, cur_n);
        if (rc) return rc;
        CK(launch_magic(ctx->d_primes, ctx->d_magic, ctx->h_primes.size(), ctx->stream));
    }
    // keep primes <= prime_limit
    std::vector<uint32_t> &h = ctx->h_primes;
    h.resize(std::upper_bound(h.begin(), h.end(), (uint32_t)std::min<uint64_t>(ctx->prime_limit, 0xffffffffu)) -
             h.begin());
    std::vector<uint32_t> &bucket = ctx->h_prime_bucket;
    bucket.assign(ctx->prime_limit / 1024 + 2, 0);
    for (size_t b = 0, i = 0; b < bucket.size(); ++b) {
        while (i < h.size() && h[i] < 1024ull * b) ++i;
        bucket[b] = (uint32_t)i;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return SIEVE_OK;
}

int check_range(sieve_ctx *ctx, uint64_t lo, uint64_t hi) {
    if (!ctx) return SIEVE_EINVAL;
    if (lo > hi) return fail(ctx, SIEVE_EINVAL, "lo > hi");
    if (hi > ctx->hi_max) return fail(ctx, SIEVE_ERANGE, "hi exceeds the context's hi_max");
    return SIEVE_OK;
}

int set_device(sieve_ctx *ctx) {
    CK(cudaSetDevice(ctx->device));
    return SIEVE_OK;
}

int bitmap_into(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t *out_dev, uint64_t *count) {
    int rc = ensure_launch(ctx, 1);
    if (rc) return rc;
    const Params prm = single_range_params(ctx, lo, hi);
    ctx->lb.h_ranges()[0] = plan_range(ctx, lo, hi, prm.seg_bytes, kModeBitmap, out_dev);
    rc = run_sync(ctx, prm, kModeBitmap, 1);
    if (rc) return rc;
    if (count) *count = ctx->lb.h_acc[0];
    return SIEVE_OK;
}

// A batched launch replayed from a CUDA graph captured once per GraphKey: for
// the mod-30 ranges (ctx->lb, m of them) the block copy, accumulator clear and
// persistent sieve kernel over the full grid (CTAs without work exit at once),
// the same for the mod-210 ranges (ctx->lb210, m210 of them), and the copy-back
// of both sets of counts.  The launch parameters and range descriptors live in
// the pinned blocks that the graph's first copies read, so a replay only needs
// the blocks refreshed.  Batches that need bucket lists are not captured
// (*used = false).  ro / ro210: per-range overrides (or null).
int batch_graph(sieve_ctx *ctx, int mode, size_t m, size_t m210, const RangeOverride *ro,
                const RangeOverride *ro210, bool *used) {
    *used = false;
    const Params &prm = ctx->params;
    uint64_t items = 0;
    int rc = SIEVE_OK;
    if (m) {
        rc = prepare_launch(ctx, prm, mode, ctx->lb, m, &ctx->buckets, &ctx->cursors, &items, ro);
        if (rc) return rc;
        if (reinterpret_cast<const SieveLaunch *>(ctx->lb.h_block)->bucket_first != 0xffffffffu) return SIEVE_OK;
    }
    // mod-210 cursors only when the mod-30 launch does not use the same store
    CursorStore *cs210 = m && reinterpret_cast<const SieveLaunch *>(ctx->lb.h_block)->cursors ? nullptr
                                                                                               : &ctx->cursors;
    if (m210) {
        rc = prepare_launch210(ctx, prm, ctx->lb210, m210, cs210, &items, ro210);
        if (rc) return rc;
    }
    if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    const uint32_t smem = m ? reinterpret_cast<const SieveLaunch *>(ctx->lb.h_block)->seg_bytes : 0;
    const uint32_t smem210 = m210 ? reinterpret_cast<const SieveLaunch *>(ctx->lb210.h_block)->seg_bytes : 0;
    const GraphKey key{m, m210, mode, smem, smem210};
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        const int grid = ctx->num_sms * prm.ctas_per_sm;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        if (m) rc = enqueue_launch(ctx, ctx->capture_stream, prm, mode, ctx->lb, m, grid, 8 * ctx->num_sms, m);
        if (!rc && m210) rc = enqueue_launch210(ctx, ctx->capture_stream, prm, ctx->lb210, m210, grid);
        cudaError_t e1 = cudaSuccess;
        if (m)
            e1 = cudaMemcpyAsync(ctx->lb.h_acc, ctx->lb.d_acc + 1, (m + 1) * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, ctx->capture_stream);
        if (e1 == cudaSuccess && m210)
            e1 = cudaMemcpyAsync(ctx->lb210.h_acc, ctx->lb210.d_acc + 1, (m210 + 1) * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, ctx->capture_stream);
        cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &g);
        if (rc || e1 != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : cuda_fail(ctx, e1 != cudaSuccess ? e1 : e2, "graph capture");
        }
        cudaGraphExec_t ex = nullptr;
        cudaError_t e3 = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) return cuda_fail(ctx, e3, "cudaGraphInstantiate");
        it = ctx->graphs.emplace(key, ex).first;
    }
    CK(cudaGraphLaunch(it->second, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if ((m && (ctx->lb.h_acc[m] & 2ull)) || (m210 && (ctx->lb210.h_acc[m210] & 2ull)) || ctx->params.fault_wait)
        return fail(ctx, SIEVE_EDEVICE, "a device-side wait hit its limit");
    *used = true;
    return SIEVE_OK;
}

int ensure_launch210(sieve_ctx *ctx, size_t m) {
    int rc = block_wait(ctx, ctx->lb210);
    if (rc) return rc;
    if (m <= ctx->lb210.cap) return SIEVE_OK;
    drop_graphs(ctx);  // they reference the old buffers
    return alloc_launch_buffers(ctx, ctx->lb210, m);
}

// Count m ranges (and write their bitmaps if bitmaps_dev is set) with per-range
// parameters rp (or the context's for all, rp = null): the ranges on each wheel
// are sieved by one persistent launch, both captured in one CUDA graph.
int batch_impl(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi, size_t m, const sieve_range_params *rp,
               uint64_t *counts, uint32_t *const *bitmaps_dev) {
    const Params &prm = ctx->params;
    const int mode = bitmaps_dev ? kModeBitmap : kModeCount;
    // resolve each range's wheel and segment size
    std::vector<uint8_t> w210(m, 0);
    std::vector<uint32_t> seg(m, prm.seg_bytes);
    size_t n210 = 0;
    for (size_t i = 0; i < m; ++i) {
        const uint32_t wheel = rp && rp[i].wheel ? rp[i].wheel : (uint32_t)prm.wheel;
        if (bitmaps_dev && wheel == 210 && rp && rp[i].wheel == 210)
            return fail(ctx, SIEVE_EINVAL, "the mod-210 wheel has no bitmap output");
        w210[i] = !bitmaps_dev && wheel == 210;
        n210 += w210[i];
        if (rp && rp[i].seg_bytes) seg[i] = rp[i].seg_bytes;
    }
    const size_t n30 = m - n210;
    int rc = ensure_launch(ctx, std::max<size_t>(n30, 1));
    if (rc) return rc;
    if (n210) {
        rc = ensure_launch210(ctx, n210);
        if (rc) return rc;
    }
    auto plan = [&](size_t i) {
        return w210[i] ? plan_range210(ctx, lo[i], hi[i], std::max<uint32_t>(std::min(seg[i], kW210MaxSegmentBytes) / 4 / 3 * 3, 3))
                       : plan_range(ctx, lo[i], hi[i], seg[i], mode, bitmaps_dev ? bitmaps_dev[i] : nullptr);
    };
    // Launch order (SIEVE_PARAM_BATCH_ORDER): as given, heaviest first, or heaviest
    // and lightest alternating -- GPU forms of sieving the last blocks from both
    // ends, since persistent CTAs take work items in launch order.  Estimated work
    // of a range: every segment visits its n_use base primes (about 3 warp
    // instructions each) and crosses 0.16 warp instructions per integer.
    std::vector<uint32_t> &order = ctx->batch_order;
    order.resize(m);
    for (size_t i = 0; i < m; ++i) order[i] = (uint32_t)i;
    if (prm.batch_order) {
        std::vector<double> cost(m);
        for (size_t i = 0; i < m; ++i) {
            const RangeDesc r = plan(i);
            cost[i] = 3.0 * (double)r.nseg * r.n_use + 0.16 * (double)(hi[i] - lo[i]);
        }
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
        if (prm.batch_order == 2) {  // heaviest, lightest, second heaviest, ...
            std::vector<uint32_t> mixed;
            mixed.reserve(m);
            for (size_t a = 0, b = m; a < b;) {
                mixed.push_back(order[a++]);
                if (a < b) mixed.push_back(order[--b]);
            }
            order.swap(mixed);
        }
    }
    // launch position of each range on its wheel
    std::vector<uint32_t> pos30, pos210;
    std::vector<RangeOverride> ro30, ro210;
    pos30.reserve(n30);
    pos210.reserve(n210);
    for (size_t k = 0; k < m; ++k) {
        const uint32_t i = order[k];
        RangeOverride o;
        if (rp) {
            o.mid_limit = rp[i].mid_limit;
            o.bucket_limit = rp[i].bucket_limit;
            o.mr_percent = rp[i].mr_percent;
        }
        if (w210[i]) {
            ctx->lb210.h_ranges()[pos210.size()] = plan(i);
            pos210.push_back(i);
            ro210.push_back(o);
        } else {
            ctx->lb.h_ranges()[pos30.size()] = plan(i);
            pos30.push_back(i);
            ro30.push_back(o);
        }
    }
    bool used = false;
    rc = batch_graph(ctx, mode, n30, n210, rp ? ro30.data() : nullptr, rp ? ro210.data() : nullptr, &used);
    if (rc) return rc;
    if (!used) {  // bucket lists: direct launches, re-run with larger lists if one overflowed
        for (int attempt = 0;; ++attempt) {
            if (attempt == 4) return fail(ctx, SIEVE_EDEVICE, "bucket lists overflowed repeatedly");
            rc = launch_ranges(ctx, ctx->stream, prm, mode, ctx->lb, n30, &ctx->buckets, &ctx->cursors,
                               rp ? ro30.data() : nullptr);
            if (rc) return rc;
            int of = 0;
            rc = finish(ctx, ctx->lb, n30, &of);
            if (rc) return rc;
            if (!of) break;
            ctx->buckets.slack *= 2;
        }
        if (n210) {
            rc = launch_ranges210(ctx, ctx->stream, prm, ctx->lb210, n210, nullptr, rp ? ro210.data() : nullptr);
            int of = 0;
            if (!rc) rc = finish(ctx, ctx->lb210, n210, &of);
            if (rc) return rc;
        }
    }
    for (size_t k = 0; k < pos30.size(); ++k) counts[pos30[k]] = ctx->lb.h_acc[k];
    for (size_t k = 0; k < pos210.size(); ++k) counts[pos210[k]] = ctx->lb210.h_acc[k];
    return SIEVE_OK;
}

}  // namespace

extern "C" {

const char *sieve_strerror(int code) {
    int i = -code;
    if (i < 0 || i >= (int)(sizeof kNames / sizeof kNames[0])) return "unknown error";
    return kNames[i];
}

const char *sieve_last_error(sieve_ctx *ctx) {
    // the context's buffer may be rewritten by a server thread at any time: hand out a
    // copy taken under the lock, in a buffer of the calling thread
    static thread_local char copy[sizeof(sieve_ctx::last_error)];
    if (!ctx) return "";
    std::lock_guard<std::mutex> lk(ctx->err_mu);
    std::memcpy(copy, ctx->last_error, sizeof copy);
    copy[sizeof copy - 1] = 0;
    return copy;
}

uint64_t sieve_bitmap_words(uint64_t lo, uint64_t hi) { return lo > hi ? 0 : bitmap_words_of(lo, hi); }

void *sieve_stream(sieve_ctx *ctx) { return ctx ? (void *)ctx->stream : nullptr; }

int sieve_create(sieve_ctx **out, uint64_t hi_max, int device, void *cuda_stream) {
    if (!out) return SIEVE_EINVAL;
    *out = nullptr;
    if (hi_max < 2 || hi_max > (1ull << 62)) return SIEVE_ERANGE;
    sieve_ctx *ctx = new (std::nothrow) sieve_ctx;
    if (!ctx) return SIEVE_ENOMEM;
    ctx->device = device;
    ctx->hi_max = hi_max;
    ctx->prime_limit = isqrt64(hi_max - 1);
    auto bail = [&](int code) {
        sieve_destroy(ctx);
        return code;
    };
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "cudaSetDevice"));
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "cudaDeviceGetAttribute"));
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "cudaStreamCreate"));
        ctx->own_stream = true;
    }
    e = set_sieve_smem_limits();
    if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "cudaFuncSetAttribute"));
    // pattern tiles: 16 copies each, each long enough for any phase plus a full
    // segment; the primes 7..19, then the further patterns 23..31, 37..43, 47..59
    const uint64_t len = tile_copy_bytes(kTilePeriod);
    ctx->tile_stride = len;
    int rc = dev_alloc(ctx, &ctx->d_tile,
                       (len + kXTileStride0 + kXTileStride1 + kXTileStride2 + kXTileStride3) * kTileCopies);
    if (rc) return bail(rc);
    {
        static const uint32_t pa[] = {7, 11, 13, 17, 19}, pb[] = {23, 29, 31}, pc[] = {37, 41, 43},
                              pd[] = {47, 53, 59};
        static const uint32_t pe[] = {61, 67, 71};
        uint8_t *x0 = ctx->d_tile + len * kTileCopies, *x1 = x0 + kXTileStride0 * kTileCopies,
                *x2 = x1 + kXTileStride1 * kTileCopies, *x3 = x2 + kXTileStride2 * kTileCopies;
        e = launch_build_tile(ctx->d_tile, len, (uint32_t)len, kTilePeriod, pa, 5, ctx->stream);
        if (e == cudaSuccess) e = launch_build_tile(x0, kXTileStride0, (uint32_t)kXTileStride0, kXTilePeriod0, pb, 3,
                                                    ctx->stream);
        if (e == cudaSuccess) e = launch_build_tile(x1, kXTileStride1, (uint32_t)kXTileStride1, kXTilePeriod1, pc, 3,
                                                    ctx->stream);
        if (e == cudaSuccess) e = launch_build_tile(x2, kXTileStride2, (uint32_t)kXTileStride2, kXTilePeriod2, pd, 3,
                                                    ctx->stream);
        if (e == cudaSuccess) e = launch_build_tile(x3, kXTileStride3, (uint32_t)kXTileStride3, kXTilePeriod3, pe, 3,
                                                    ctx->stream);
        if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "build tile"));
    }
    // the mod-210 count path: class tables and the 16 shifted copies of its pattern
    {
        e = set_sieve210_smem_limit();
        if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "cudaFuncSetAttribute"));
        W210Tables t;
        build_w210_tables(&t);
        rc = dev_alloc(ctx, &ctx->d_tab210, 1);
        if (rc) return bail(rc);
        e = cudaMemcpyAsync(ctx->d_tab210, &t, sizeof t, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "copy tables"));
        const uint64_t len210 = ((uint64_t)kW210PeriodBytes + kW210MaxSmemBytes + 32 + 15) & ~15ull;
        ctx->tile210_stride = len210;
        rc = dev_alloc(ctx, &ctx->d_tile210, len210 * kTileCopies);
        if (rc) return bail(rc);
        e = launch_build_tile210(ctx->d_tab210, ctx->d_tile210, ctx->tile210_stride, (uint32_t)len210, ctx->stream);
        if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "build tile"));
        e = cudaStreamSynchronize(ctx->stream);  // t is on this stack frame
        if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "build tables"));
    }
    rc = make_base_primes(ctx);
    if (rc) return bail(rc);
    *out = ctx;
    return SIEVE_OK;
}

void sieve_destroy(sieve_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    if (!ctx->shadow) {
        cudaFree(ctx->d_primes);
        cudaFree(ctx->d_magic);
        cudaFree(ctx->d_tile);
        cudaFree(ctx->d_tile210);
        cudaFree(ctx->d_tab210);
    }
    cudaFree(ctx->d_bitmap);
    cudaFree(ctx->buckets.d);
    cudaFree(ctx->cursors.d);
    cudaFree(ctx->mr.d);
    free_launch_buffers(ctx, ctx->lb);
    free_launch_buffers(ctx, ctx->lb210);
    free_compact_scratch(ctx, ctx->cs);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int sieve_count(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *count) {
    if (!count) return fail(ctx, SIEVE_EINVAL, "null count");
    int rc = check_range(ctx, lo, hi);
    if (rc) return rc;
    if ((rc = set_device(ctx))) return rc;
    if (lo == hi) {
        *count = 0;
        return SIEVE_OK;
    }
    rc = ensure_launch(ctx, 1);
    if (rc) return rc;
    if (ctx->params.wheel == 210) {
        ctx->lb.h_ranges()[0] = plan_range210(ctx, lo, hi, w210_segment_words(ctx->params));
        rc = launch_ranges210(ctx, ctx->stream, ctx->params, ctx->lb, 1, &ctx->cursors);
        int of = 0;
        if (!rc) rc = finish(ctx, ctx->lb, 1, &of);
        if (rc) return rc;
        *count = ctx->lb.h_acc[0];
        return SIEVE_OK;
    }
    const Params prm = single_range_params(ctx, lo, hi);
    ctx->lb.h_ranges()[0] = plan_range(ctx, lo, hi, prm.seg_bytes, kModeCount, nullptr);
    rc = run_sync(ctx, prm, kModeCount, 1);
    if (rc) return rc;
    *count = ctx->lb.h_acc[0];
    return SIEVE_OK;
}

int sieve_count_dev(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *count_dev) {
    if (!count_dev) return fail(ctx, SIEVE_EINVAL, "null count");
    int rc = check_range(ctx, lo, hi);
    if (rc) return rc;
    if ((rc = set_device(ctx))) return rc;
    rc = ensure_launch(ctx, 1);
    if (rc) return rc;
    if (ctx->params.wheel == 210) {
        ctx->lb.h_ranges()[0] = plan_range210(ctx, lo, hi, w210_segment_words(ctx->params));
        rc = launch_ranges210(ctx, ctx->stream, ctx->params, ctx->lb, 1, &ctx->cursors);
    } else {
        const Params prm = single_range_params(ctx, lo, hi);
        ctx->lb.h_ranges()[0] = plan_range(ctx, lo, hi, prm.seg_bytes, kModeCount, nullptr);
        rc = launch_ranges(ctx, ctx->stream, prm, kModeCount, ctx->lb, 1, &ctx->buckets, &ctx->cursors);
    }
    if (rc) return rc;
    // the count, or UINT64_MAX if a bucket list overflowed
    CK(launch_finalize_count(ctx->lb.d_acc + 1, reinterpret_cast<const unsigned *>(ctx->lb.d_acc + 2), count_dev,
                             ctx->stream));
    return SIEVE_OK;
}

int sieve_bitmap(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t *out_dev, size_t out_words, uint64_t *count) {
    int rc = check_range(ctx, lo, hi);
    if (rc) return rc;
    if ((rc = set_device(ctx))) return rc;
    const uint64_t need = bitmap_words_of(lo, hi);
    if (out_words < need) return fail(ctx, SIEVE_ETRUNC, "bitmap capacity too small");
    if (need && !out_dev) return fail(ctx, SIEVE_EINVAL, "null bitmap");
    if (lo == hi) {
        if (count) *count = 0;
        return SIEVE_OK;
    }
    return bitmap_into(ctx, lo, hi, out_dev, count);
}

static int list_impl(sieve_ctx *ctx, uint64_t lo, uint64_t hi, void *out_dev, size_t cap, uint64_t *n, int out64) {
    if (!n) return fail(ctx, SIEVE_EINVAL, "null n");
    int rc = check_range(ctx, lo, hi);
    if (rc) return rc;
    if (!out64 && hi > (1ull << 32)) return fail(ctx, SIEVE_ERANGE, "uint32 list needs hi <= 2^32");
    if ((rc = set_device(ctx))) return rc;
    if (lo == hi) {
        *n = 0;
        return SIEVE_OK;
    }
    rc = ensure_bitmap(ctx, bitmap_words_of(lo, hi));
    if (rc) return rc;
    rc = bitmap_into(ctx, lo, hi, ctx->d_bitmap, nullptr);
    if (rc) return rc;
    return compact_with(ctx, ctx->stream, ctx->cs, ctx->d_bitmap, lo, hi, out_dev, cap, n, out64);
}

int sieve_list(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t *out_dev, size_t cap, uint64_t *n) {
    return list_impl(ctx, lo, hi, out_dev, cap, n, 0);
}

int sieve_list64(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *out_dev, size_t cap, uint64_t *n) {
    return list_impl(ctx, lo, hi, out_dev, cap, n, 1);
}

int sieve_bitmap_dev(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t *out_dev, size_t out_words,
                     uint64_t *count_dev) {
    if (!ctx) return SIEVE_EINVAL;
    if (!count_dev) return fail(ctx, SIEVE_EINVAL, "null count");
    int rc = check_range(ctx, lo, hi);
    if (rc) return rc;
    if ((rc = set_device(ctx))) return rc;
    const uint64_t need = bitmap_words_of(lo, hi);
    if (out_words < need) return fail(ctx, SIEVE_ETRUNC, "bitmap capacity too small");
    if (need && !out_dev) return fail(ctx, SIEVE_EINVAL, "null bitmap");
    if (lo == hi) {
        CK(launch_store_count(nullptr, 0, count_dev, ctx->stream));
        return SIEVE_OK;
    }
    rc = ensure_launch(ctx, 1);
    if (rc) return rc;
    const Params prm = single_range_params(ctx, lo, hi);
    ctx->lb.h_ranges()[0] = plan_range(ctx, lo, hi, prm.seg_bytes, kModeBitmap, out_dev);
    rc = launch_ranges(ctx, ctx->stream, prm, kModeBitmap, ctx->lb, 1, &ctx->buckets, &ctx->cursors);
    if (rc) return rc;
    // the count, or UINT64_MAX if a bucket list overflowed or a device-side wait gave up
    CK(launch_finalize_count(ctx->lb.d_acc + 1, reinterpret_cast<const unsigned *>(ctx->lb.d_acc + 2), count_dev,
                             ctx->stream));
    return SIEVE_OK;
}

int sieve_compact_dev(sieve_ctx *ctx, const uint32_t *bitmap_dev, uint64_t lo, uint64_t hi, uint32_t *out_dev,
                      size_t cap, uint64_t *n_dev) {
    if (!ctx) return SIEVE_EINVAL;
    if (!n_dev) return fail(ctx, SIEVE_EINVAL, "null n");
    int rc = check_range(ctx, lo, hi);
    if (rc) return rc;
    if (hi > (1ull << 32)) return fail(ctx, SIEVE_ERANGE, "uint32 list needs hi <= 2^32");
    if (bitmap_words_of(lo, hi) && !bitmap_dev) return fail(ctx, SIEVE_EINVAL, "null bitmap");
    if (!out_dev && cap) return fail(ctx, SIEVE_EINVAL, "null output with a nonzero capacity");
    if ((rc = set_device(ctx))) return rc;
    return compact_async(ctx, ctx->stream, ctx->cs, bitmap_dev, lo, hi, out_dev, cap, n_dev, 0);
}

int sieve_compact(sieve_ctx *ctx, const uint32_t *bitmap_dev, uint64_t lo, uint64_t hi, uint32_t *out_dev,
                  size_t cap, uint64_t *n) {
    if (!n) return fail(ctx, SIEVE_EINVAL, "null n");
    int rc = check_range(ctx, lo, hi);
    if (rc) return rc;
    if (hi > (1ull << 32)) return fail(ctx, SIEVE_ERANGE, "uint32 list needs hi <= 2^32");
    if (bitmap_words_of(lo, hi) && !bitmap_dev) return fail(ctx, SIEVE_EINVAL, "null bitmap");
    if ((rc = set_device(ctx))) return rc;
    return compact_with(ctx, ctx->stream, ctx->cs, bitmap_dev, lo, hi, out_dev, cap, n, 0);
}

int sieve_batch_count(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi, size_t m, uint64_t *counts,
                      uint32_t *const *bitmaps_dev) {
    return sieve_batch_count_params(ctx, lo, hi, m, nullptr, counts, bitmaps_dev);
}

int sieve_batch_count_params(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi, size_t m,
                             const sieve_range_params *params, uint64_t *counts, uint32_t *const *bitmaps_dev) {
    if (!ctx) return SIEVE_EINVAL;
    if (m == 0) return SIEVE_OK;
    if (!lo || !hi || !counts) return fail(ctx, SIEVE_EINVAL, "null array");
    for (size_t i = 0; i < m; ++i) {
        int rc = check_range(ctx, lo[i], hi[i]);
        if (rc) return rc;
        if (params) {
            const sieve_range_params &q = params[i];
            if (q.seg_bytes && (q.seg_bytes < 1024 || q.seg_bytes > kMaxSegmentBytes || q.seg_bytes % 32))
                return fail(ctx, SIEVE_EINVAL, "range segment bytes");
            if (q.wheel && q.wheel != 30 && q.wheel != 210) return fail(ctx, SIEVE_EINVAL, "range wheel (30 or 210)");
            if (q.mid_limit > (1u << 31)) return fail(ctx, SIEVE_EINVAL, "range mid limit");
        }
    }
    int rc = set_device(ctx);
    if (rc) return rc;
    return batch_impl(ctx, lo, hi, m, params, counts, bitmaps_dev);
}

int sieve_set_param(sieve_ctx *ctx, int param, int64_t v) {
    if (!ctx) return SIEVE_EINVAL;
    Params &p = ctx->params;
    switch (param) {
        case SIEVE_PARAM_SEGMENT_BYTES:
            if (v < 1024 || v > (int64_t)kMaxSegmentBytes || v % 32) return fail(ctx, SIEVE_EINVAL, "segment bytes");
            p.seg_bytes = (uint32_t)v;
            break;
        case SIEVE_PARAM_THREADS:
            if (v != 256 && v != 512 && v != 1024) return fail(ctx, SIEVE_EINVAL, "threads");
            p.threads = (int)v;
            break;
        case SIEVE_PARAM_SMALL_LIMIT:
            if (v < 23 || v > 65536) return fail(ctx, SIEVE_EINVAL, "small limit");
            p.small_limit = (uint32_t)v;
            break;
        case SIEVE_PARAM_CTAS_PER_SM:
            if (v < 1 || v > 8) return fail(ctx, SIEVE_EINVAL, "ctas per sm");
            p.ctas_per_sm = (int)v;
            break;
        case SIEVE_PARAM_CHUNK_SEGMENTS:
            if (v < 1 || v > (int64_t)kMaxChunkSegments) return fail(ctx, SIEVE_EINVAL, "chunk segments");
            p.chunk_segs = (uint32_t)v;
            break;
        case SIEVE_PARAM_BUCKET_LIMIT:
            if (v < 0) return fail(ctx, SIEVE_EINVAL, "bucket limit");
            p.bucket_limit = (uint64_t)v;
            break;
        case SIEVE_PARAM_CURSOR_MB:
            if (v < 0 || v > 4096) return fail(ctx, SIEVE_EINVAL, "cursor budget");
            p.cursor_mb = (uint32_t)v;
            break;
        case SIEVE_PARAM_MID_LIMIT:
            if (v < 0 || v > (1ll << 31)) return fail(ctx, SIEVE_EINVAL, "mid limit");
            p.mid_limit = (uint32_t)v;
            break;
        case SIEVE_PARAM_MR_PERCENT:
            if (v < 0 || v > 1000000) return fail(ctx, SIEVE_EINVAL, "Miller-Rabin percent");
            p.mr_percent = (uint32_t)v;
            break;
        case SIEVE_PARAM_WHEEL:
            if (v != 30 && v != 210) return fail(ctx, SIEVE_EINVAL, "wheel (30 or 210)");
            p.wheel = (int)v;
            break;
        case SIEVE_PARAM_BATCH_ORDER:
            if (v < 0 || v > 2) return fail(ctx, SIEVE_EINVAL, "batch order (0, 1 or 2)");
            p.batch_order = (int)v;
            break;
        case SIEVE_PARAM_FAULT_WAIT:
            if (v != 0 && v != 1) return fail(ctx, SIEVE_EINVAL, "fault hook (0 or 1)");
            p.fault_wait = (int)v;
            break;
        case SIEVE_PARAM_PRESIEVE:
            if (v != 19 && v != 59 && v != 71) return fail(ctx, SIEVE_EINVAL, "pre-sieve limit (19, 59 or 71)");
            p.presieve = (uint32_t)v;
            break;
        case SIEVE_PARAM_SMALL_LIMIT_210:
            if (v < 0 || v > (1 << 20)) return fail(ctx, SIEVE_EINVAL, "small limit (mod 210)");
            p.small_limit210 = (uint32_t)v;
            break;
        case SIEVE_PARAM_MID_LIMIT_210:
            if (v < 0 || v > (1ll << 31)) return fail(ctx, SIEVE_EINVAL, "mid limit (mod 210)");
            p.mid_limit210 = (uint32_t)v;
            break;
        default:
            return fail(ctx, SIEVE_EINVAL, "unknown parameter");
    }
    drop_graphs(ctx);  // captured launches bake in the launch shape
    return SIEVE_OK;
}

int sieve_get_param(sieve_ctx *ctx, int param, int64_t *v) {
    if (!ctx || !v) return SIEVE_EINVAL;
    const Params &p = ctx->params;
    switch (param) {
        case SIEVE_PARAM_SEGMENT_BYTES: *v = p.seg_bytes; return SIEVE_OK;
        case SIEVE_PARAM_THREADS: *v = p.threads; return SIEVE_OK;
        case SIEVE_PARAM_SMALL_LIMIT: *v = p.small_limit; return SIEVE_OK;
        case SIEVE_PARAM_CTAS_PER_SM: *v = p.ctas_per_sm; return SIEVE_OK;
        case SIEVE_PARAM_CHUNK_SEGMENTS: *v = p.chunk_segs; return SIEVE_OK;
        case SIEVE_PARAM_BUCKET_LIMIT: *v = (int64_t)p.bucket_limit; return SIEVE_OK;
        case SIEVE_PARAM_CURSOR_MB: *v = p.cursor_mb; return SIEVE_OK;
        case SIEVE_PARAM_MR_PERCENT: *v = p.mr_percent; return SIEVE_OK;
        case SIEVE_PARAM_MID_LIMIT: *v = p.mid_limit; return SIEVE_OK;
        case SIEVE_PARAM_WHEEL: *v = p.wheel; return SIEVE_OK;
        case SIEVE_PARAM_BATCH_ORDER: *v = p.batch_order; return SIEVE_OK;
        case SIEVE_PARAM_FAULT_WAIT: *v = p.fault_wait; return SIEVE_OK;
        case SIEVE_PARAM_PRESIEVE: *v = p.presieve; return SIEVE_OK;
        case SIEVE_PARAM_SMALL_LIMIT_210: *v = p.small_limit210; return SIEVE_OK;
        case SIEVE_PARAM_MID_LIMIT_210: *v = p.mid_limit210; return SIEVE_OK;
        default: return fail(ctx, SIEVE_EINVAL, "unknown parameter");
    }
}

int sieve_get_info(sieve_ctx *ctx, sieve_info *info) {
    if (!ctx || !info) return SIEVE_EINVAL;
    info->hi_max = ctx->hi_max;
    info->prime_limit = ctx->prime_limit;
    info->n_base_primes = ctx->h_primes.size();
    info->device = ctx->device;
    info->num_sms = ctx->num_sms;
    info->device_bytes = ctx->device_bytes;
    return SIEVE_OK;
}

int sieve_base_primes(sieve_ctx *ctx, uint32_t *out, size_t cap, uint64_t *n) {
    if (!ctx || !n) return SIEVE_EINVAL;
    *n = ctx->h_primes.size();
    if (out) std::memcpy(out, ctx->h_primes.data(), std::min<size_t>(cap, ctx->h_primes.size()) * sizeof(uint32_t));
    return SIEVE_OK;
}

int sieve_selftest_wait(sieve_ctx *ctx, int arm, uint32_t limit, int *timed_out) {
    if (!ctx || !timed_out || limit == 0) return SIEVE_EINVAL;
    int rc = set_device(ctx);
    if (rc) return rc;
    int *d_status = nullptr;
    rc = dev_alloc(ctx, &d_status, 1);
    if (rc) return rc;
    int h_status = -1;
    cudaError_t e = launch_wait_selftest(ctx->d_tile, 4096, arm ? 1 : 0, limit, d_status, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, d_status, 1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wait self-test");
    *timed_out = h_status;
    return SIEVE_OK;
}

int sieve_crossing_work_ge(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t pmin, uint64_t *clears) {
    if (!clears) return fail(ctx, SIEVE_EINVAL, "null clears");
    int rc = check_range(ctx, lo, hi);
    if (rc) return rc;
    // For each base prime p >= max(pmin, 23): #{ m : m >= p, gcd(m, W) = 1, lo <= p m < hi },
    // W the wheel of the count path (30, or 210 when SIEVE_PARAM_WHEEL is 210).
    const uint64_t W = ctx->params.wheel == 210 ? 210 : 30;
    uint64_t cum[211] = {0};  // cum[r] = #{ 1 <= m < r : gcd(m, W) = 1 }
    for (uint64_t r = 1; r <= W; ++r) cum[r] = cum[r - 1] + ((r - 1) % 2 && (r - 1) % 3 && (r - 1) % 5 && (W == 30 || (r - 1) % 7));
    auto coprime_below = [&](uint64_t x) -> uint64_t {  // #{ 1 <= m < x : gcd(m, W) = 1 }
        return (x / W) * cum[W] + cum[x % W];
    };
    uint64_t total = 0;
    const uint32_t n_use = primes_needed(ctx, hi);
    for (uint32_t i = kFirstCrossingPrime; i < n_use; ++i) {
        const uint64_t p = ctx->h_primes[i];
        if (p < pmin) continue;
        uint64_t m_lo = std::max<uint64_t>(p, (lo + p - 1) / p);
        uint64_t m_hi = (hi + p - 1) / p;  // m < m_hi  <=>  p m < hi
        if (m_hi > m_lo) total += coprime_below(m_hi) - coprime_below(m_lo);
    }
    *clears = total;
    return SIEVE_OK;
}

int sieve_crossing_work(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *clears) {
    return sieve_crossing_work_ge(ctx, lo, hi, 23, clears);
}

}  // extern "C"
