// host.h -- host-side state shared by the C ABI (sieve_api.cu) and the
// request server (sieve_server.cu).  Not part of the public interface.
#pragma once

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gbsieve.h"
#include "internal.h"

namespace gbs {

// Launch parameters (copied by the server at creation).
struct Params {
    uint32_t seg_bytes = kMaxSegmentBytes;
    int threads = 1024;
    uint32_t small_limit = 304;   // measured best on pi(10^12) with the patterns up to 71: swept 208..544 in
                                  // steps of 16 (448 was best with the patterns up to 59)
    uint32_t mid_limit = 0;       // primes below this use per-phase sub-progressions; 0: segment bytes / 3
    int ctas_per_sm = 1;
    uint32_t chunk_segs = 32;      // segments per work item (24, 32: within 0.05 ms; 64 and 16 slower)
    uint64_t bucket_limit = 1ull << 62;  // primes >= this use the bucket lists; 0: the segment size
    uint32_t cursor_mb = 1024;           // budget for per-CTA large-prime cursors (0: recompute every segment)
    uint32_t mr_percent = 0;             // Miller-Rabin path when width < this % of the skipped primes (0: off)
    int wheel = 30;                      // count-only launches on the mod-30 or the mod-210 wheel
    uint32_t small_limit210 = 128;       // mod-210: primes below this are crossed warp-cooperatively
    uint32_t mid_limit210 = 0;           // mod-210: primes below this use per-class sub-progressions; 0: words / 6
    int batch_order = 0;                 // batches: 0 as given, 1 heaviest first, 2 heaviest/lightest alternating
    int fault_wait = 0;                  // test hook: synchronous launches report a device-wait failure
    uint32_t presieve = 59;              // mod-30: largest prime applied as a pattern (19, 59 or 71); with
                                         // the small limit re-tuned, 71 is 0.15 % faster on pi(10^12) but its
                                         // 8 MB of pattern copies evict the cursors: 7x the DRAM traffic
};

// Everything one sieve launch reads and writes besides the resident state:
// a pinned host block and its device copy ([SieveLaunch | RangeDesc x m]),
// and the accumulators ([0] work counter, [1..m] counts, [m+1] overflow flag).
struct LaunchBuffers {
    unsigned char *h_block = nullptr;
    unsigned char *d_block = nullptr;
    unsigned long long *d_acc = nullptr;
    unsigned long long *h_acc = nullptr;  // pinned, [0..m] = counts, overflow
    size_t cap = 0;                        // ranges
    // recorded on the stream after the block's host-to-device copies: an
    // asynchronous call may return before they run, so the next writer of
    // h_block waits for it (block_wait)
    cudaEvent_t consumed = nullptr;
    RangeDesc *h_ranges() const { return reinterpret_cast<RangeDesc *>(h_block + kLaunchHeader); }
    RangeDesc *d_ranges() const { return reinterpret_cast<RangeDesc *>(d_block + kLaunchHeader); }
    // after the ranges: the indices of the ranges on the Miller-Rabin path, then the
    // cap + 1 prefix sums of their word counts
    uint32_t *h_mr() const { return reinterpret_cast<uint32_t *>(h_block + kLaunchHeader + cap * sizeof(RangeDesc)); }
    uint32_t *d_mr() const { return reinterpret_cast<uint32_t *>(d_block + kLaunchHeader + cap * sizeof(RangeDesc)); }
    uint32_t *h_mrw() const { return h_mr() + cap; }
    uint32_t *d_mrw() const { return d_mr() + cap; }
    static size_t block_bytes(size_t cap) {
        return kLaunchHeader + cap * (sizeof(RangeDesc) + 2 * sizeof(uint32_t)) + sizeof(uint32_t);
    }
};

// Words the Miller-Rabin path needs for ranges without an output bitmap.
struct MrScratch {
    uint32_t *d = nullptr;
    size_t words = 0;
};

// Scratch of the bitmap -> list compaction.
struct CompactScratch {
    uint32_t *counts = nullptr;
    uint64_t *offsets = nullptr;
    unsigned long long *d_total = nullptr;
    unsigned long long *h_total = nullptr;  // pinned
    unsigned long long *status = nullptr;   // cap + 1 words: the single-pass compaction's tile states
    size_t cap = 0;                          // tiles
};

struct BucketStore {
    uint32_t *d = nullptr;
    size_t entries = 0;
    double slack = 1.15;  // capacity = slack x expected hits + 4096, raised on overflow
};

struct CursorStore {
    uint32_t *d = nullptr;
    size_t entries = 0;
};

// A captured batch: m ranges on the mod-30 wheel in `mode` (count or bitmap)
// with `smem` bytes of shared memory per CTA, and m210 count-only ranges on the
// mod-210 wheel with smem210 bytes.
struct GraphKey {
    size_t m, m210;
    int mode;
    uint32_t smem, smem210;
    bool operator<(const GraphKey &o) const {
        if (m != o.m) return m < o.m;
        if (m210 != o.m210) return m210 < o.m210;
        if (mode != o.mode) return mode < o.mode;
        if (smem != o.smem) return smem < o.smem;
        return smem210 < o.smem210;
    }
};

// Per-range overrides of a launch's parameters (0: the launch's Params).  The
// segment size of a range is its RangeDesc::seg_bytes, set when it is planned.
struct RangeOverride {
    uint32_t mid_limit = 0;      // primes below this use the per-phase (mod 30) / per-class (mod 210) tier
    uint64_t bucket_limit = 0;   // primes >= this go through the bucket lists (mod 30)
    uint32_t mr_percent = 0;     // Miller-Rabin threshold; UINT32_MAX: never
};

}  // namespace gbs

struct sieve_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t capture_stream = nullptr;  // graphs are captured here (never on the legacy stream)
    uint64_t hi_max = 0;
    uint64_t prime_limit = 0;

    // resident state: base primes (2 first), their Barrett constants, the pattern tile
    uint32_t *d_primes = nullptr;
    uint64_t *d_magic = nullptr;
    std::vector<uint32_t> h_primes;
    std::vector<uint32_t> h_prime_bucket;  // [b]: index of the first base prime >= 1024 b
    uint8_t *d_tile = nullptr;
    uint64_t tile_stride = 0;
    // the same for the mod-210 count path: pattern of 11..19 and the class tables
    uint8_t *d_tile210 = nullptr;
    uint64_t tile210_stride = 0;
    gbs::W210Tables *d_tab210 = nullptr;

    gbs::Params params;
    gbs::LaunchBuffers lb;
    gbs::LaunchBuffers lb210;  // the mod-210 ranges of a batch whose ranges use both wheels
    gbs::CompactScratch cs;
    gbs::BucketStore buckets;
    gbs::CursorStore cursors;
    gbs::MrScratch mr;
    std::vector<uint32_t> batch_order;  // launch position -> caller's index, last batch
    uint32_t *d_bitmap = nullptr;  // list scratch
    size_t bitmap_cap = 0;         // words

    // batched launches replayed from graphs, per (ranges, mode); invalidated
    // when a buffer they reference is reallocated or a parameter changes
    std::map<gbs::GraphKey, cudaGraphExec_t> graphs;

    std::atomic<uint64_t> device_bytes{0};
    bool shadow = false;  // a server's private view: resident arrays are borrowed, not owned
    // the last failure's message; server threads share a view, so writes are serialised
    std::mutex err_mu;
    char last_error[256] = {0};
};

namespace gbs {

int fail(sieve_ctx *c, int code, const std::string &msg);
int cuda_fail(sieve_ctx *c, cudaError_t e, const char *where);
uint64_t isqrt64(uint64_t n);
uint64_t bitmap_words_of(uint64_t lo, uint64_t hi);
RangeDesc plan_range(const sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t seg_bytes, int mode,
                     uint32_t *bitmap);
int alloc_launch_buffers(sieve_ctx *ctx, LaunchBuffers &lb, size_t m);
void free_launch_buffers(sieve_ctx *ctx, LaunchBuffers &lb);
int block_wait(sieve_ctx *ctx, LaunchBuffers &lb);  // until lb.h_block may be rewritten
int alloc_compact_scratch(sieve_ctx *ctx, CompactScratch &cs, size_t tiles);
void free_compact_scratch(sieve_ctx *ctx, CompactScratch &cs);

// Sieve the m ranges lb.h_ranges()[0..m) (planned with plan_range) on
// `stream`: fills in the launch header, copies the block, clears the
// accumulators and launches.  Bucket lists are used only if `bs` is given.
RangeDesc plan_range210(const sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t seg_words);
uint32_t w210_segment_words(const Params &prm);
// ro (optional) holds per-range overrides of prm, one per range of lb.
int launch_ranges210(sieve_ctx *ctx, cudaStream_t stream, const Params &prm, LaunchBuffers &lb, size_t m,
                     CursorStore *cs, const RangeOverride *ro = nullptr);
int launch_ranges(sieve_ctx *ctx, cudaStream_t stream, const Params &prm, int mode, LaunchBuffers &lb, size_t m,
                  BucketStore *bs, CursorStore *cs = nullptr, const RangeOverride *ro = nullptr);

// Compact the odd-only bitmap of [lo, hi) into out_dev (uint32 or uint64): the
// values p - sub (sub = 0: the primes; sub = lo: their offsets from lo, which a
// uint32 list can hold whenever hi - lo <= 2^32).  *n = primes in the range (2
// included); SIEVE_ETRUNC if cap < *n.  Synchronises `stream`.
int compact_with(sieve_ctx *ctx, cudaStream_t stream, CompactScratch &cs, const uint32_t *bitmap_dev, uint64_t lo,
                 uint64_t hi, void *out_dev, size_t cap, uint64_t *n, int out64, uint64_t sub = 0);

}  // namespace gbs
