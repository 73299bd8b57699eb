// internal.h -- types shared by the kernels and the host side of gbsieve.
//
// Layout of the mod-30 wheel used by every sieving kernel: wheel byte b holds
// the eight integers 30 b + r, r in {1, 7, 11, 13, 17, 19, 23, 29} (the
// residues coprime to 30), bit k <-> residue k in that order.  Multiples of 2,
// 3 and 5 have no bit.  A segment is a run of consecutive wheel bytes held in
// shared memory.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gbs {

// Pre-sieve period: 7 * 11 * 13 * 17 * 19 wheel bytes.
constexpr uint32_t kTilePeriod = 323323u;
// Largest shared-memory segment a launch may use, bytes (227 KB opt-in limit
// per CTA minus the kernel's static shared memory).
constexpr uint32_t kMaxSegmentBytes = 229376u;
// Most segments one work item (a chunk) may hold; bucket lists are per segment of a chunk.
constexpr uint32_t kMaxChunkSegments = 64u;
// Small primes whose per-segment residue B0 mod p is cached in shared memory.
constexpr uint32_t kSmallResidues = 96u;
// Number of byte-shifted copies of the pattern (one per 16-byte phase).
constexpr uint32_t kTileCopies = 16u;
// Index of the first base prime >= 23 in the base-prime array (2, 3, 5, 7,
// 11, 13, 17, 19 come first).
constexpr uint32_t kFirstCrossingPrime = 8u;
// Three further pre-sieve patterns for the mod-30 kernels, ANDed into a segment
// after the first one: the wheel bytes of 23 * 29 * 31, 37 * 41 * 43 and 47 * 53 * 59.
// Each is stored like the first (kTileCopies byte-shifted copies, each a period
// plus a full segment long), after it in the same allocation.
constexpr uint32_t kXTilePeriod0 = 20677u;  // 23 * 29 * 31
constexpr uint32_t kXTilePeriod1 = 65231u;  // 37 * 41 * 43
constexpr uint32_t kXTilePeriod2 = 146969u; // 47 * 53 * 59
constexpr uint32_t kXTilePeriod3 = 290177u; // 61 * 67 * 71 (a fourth pattern, SIEVE_PARAM_PRESIEVE = 71)
constexpr uint64_t tile_copy_bytes(uint32_t period) {
    return ((uint64_t)period + kMaxSegmentBytes + 32 + 15) & ~15ull;
}
constexpr uint64_t kXTileStride0 = tile_copy_bytes(kXTilePeriod0);
constexpr uint64_t kXTileStride1 = tile_copy_bytes(kXTilePeriod1);
constexpr uint64_t kXTileStride2 = tile_copy_bytes(kXTilePeriod2);
constexpr uint64_t kXTileStride3 = tile_copy_bytes(kXTilePeriod3);
// Index of the first base prime >= 61: the first one crossed when the
// further patterns are applied.
constexpr uint32_t kFirstCrossingPrimeX = 17u;
// Index of the first base prime >= 73: the first one crossed with the fourth pattern.
constexpr uint32_t kFirstCrossingPrimeX4 = 20u;

// One range of a launch.  Segment s of the range covers wheel bytes
// [Bbase + s S, Bbase + (s + 1) S); Bbase is chosen so that 30 Bbase + 1 is
// congruent to o0 = lo | 1 modulo 64 and 30 Bbase <= lo (Bbase may be
// negative, >= -32, when lo < 960): every group of 32 wheel bytes then maps
// to exactly 15 whole words of the odd-only output bitmap.
struct RangeDesc {
    int64_t Bbase;          // wheel byte of segment 0
    uint64_t lo, hi;        // the half-open range
    uint64_t item_first;    // launch-wide index of this range's first chunk
    uint64_t nseg;          // segments in this range
    uint32_t *bitmap;       // odd-only output (bitmap mode); null: count only
    uint64_t bitmap_words;  // words of the odd-only bitmap of [lo, hi)
    uint64_t corr;          // primes the wheel cannot hold (2, 3, 5) in range
    uint32_t n_use;         // base primes with p * p < hi (prefix length)
    uint32_t mr;            // 1: sieve with the primes below 2^16, then Miller-Rabin (one segment)
    // this range's launch parameters (ranges of one launch may differ):
    uint32_t seg_bytes;     // segment size S (bytes; <= the launch's SieveLaunch::seg_bytes)
    uint32_t mid_end;       // primes [small_end, mid_end) per-phase tier, [mid_end, ...) wheel walk
    uint32_t bucket_first;  // primes [bucket_first, n_use) through the bucket lists (0xffffffff: none)
    uint32_t reserved;
};
static_assert(sizeof(RangeDesc) == 88, "RangeDesc layout");

enum SieveMode : int { kModeCount = 0, kModeBitmap = 1 };

struct SieveLaunch {
    const RangeDesc *ranges;
    uint32_t n_ranges;
    uint64_t n_items;                    // total chunks over all ranges
    unsigned long long *item_counter;    // zeroed before the launch
    unsigned long long *counts;          // one per range, zeroed before the launch
    const uint32_t *primes;              // base primes, ascending, 2 first
    const uint64_t *magic;               // floor((2^64 - 1) / p) per prime
    uint32_t small_end;                  // primes [small_first, small_end) crossed warp-cooperatively
    uint32_t mid_end;                    // the largest RangeDesc::mid_end of the launch (cost table end)
    uint32_t bucket_first;               // the smallest RangeDesc::bucket_first of the launch
    uint32_t chunk_segs;                 // segments per work item, <= kMaxChunkSegments
    uint32_t *buckets;                   // grid x chunk_segs x bucket_cap entries
    uint32_t bucket_cap;                 // entries per segment list
    unsigned *overflow;                  // set to 1 if a list overflowed (zeroed before the launch)
    uint32_t mr_end;                     // index of the first base prime >= 2^16
    uint64_t mr_square;                  // that prime squared: survivors below it need no test
    const uint32_t *mr_list;             // ranges on the Miller-Rabin path
    const uint32_t *mr_words;            // n_mr + 1 prefix sums of their words (the filter's flat index)
    uint32_t n_mr;
    uint32_t *cursors;                   // null, or grid x cursor_stride wheel cursors of the large primes
    uint32_t cursor_stride;              // large primes per CTA (from mid_end)
    const uint8_t *tile;                 // kTileCopies shifted copies of the pattern
    uint64_t tile_stride;                // bytes between copies
    uint32_t seg_bytes;                  // the largest RangeDesc::seg_bytes (shared memory per CTA)
    uint32_t small_first;                // first prime of the small tier: kFirstCrossingPrime, or
                                         // kFirstCrossingPrimeX with the further patterns
    const uint8_t *xtile0, *xtile1, *xtile2;  // null, or copy 0 of each further pattern (mod-30 kernels)
    const uint8_t *xtile3;                    // null, or copy 0 of the fourth pattern (61 * 67 * 71)
};
// Bytes reserved for the SieveLaunch at the head of a launch block; the
// RangeDescs follow it.
constexpr size_t kLaunchHeader = 256;
static_assert(sizeof(SieveLaunch) <= kLaunchHeader, "launch header");

// Kernel launchers (sieve_kernels.cu).  All enqueue on `stream` and return the
// CUDA launch status.
// Pattern of the primes ps[0 .. np) (np <= 5, product = period) on the mod-30 wheel:
// kTileCopies copies, copy k holding pattern byte (i + k) mod period at offset i < len.
cudaError_t launch_build_tile(uint8_t *tile, uint64_t stride, uint32_t len, uint32_t period, const uint32_t *ps,
                              int np, cudaStream_t stream);
cudaError_t launch_tiny_primes(uint32_t *out, uint32_t *n_out, cudaStream_t stream);
cudaError_t launch_magic(const uint32_t *primes, uint64_t *magic, uint64_t n, cudaStream_t stream);
// Launch parameters live in device memory (d_launch) so that a captured graph
// can be replayed with new ranges; d_launch->n_items may be 0.
cudaError_t launch_sieve(int mode, const SieveLaunch *d_launch, int grid, int threads, uint32_t seg_bytes,
                         cudaStream_t stream);
cudaError_t set_sieve_smem_limits();
// Miller-Rabin test of the survivors of the ranges in d_launch->mr_list.
cudaError_t launch_mr_filter(int mode, const SieveLaunch *d_launch, int grid, cudaStream_t stream);

// Count path on the mod-210 wheel (sieve_w210.cu): 48 bits per group of 210
// integers, bit 48 g + i <-> 210 g + r_i (r_i the residues coprime to 210,
// ascending), packed LSB-first into 32-bit words; segments of a multiple of 3
// words (2 whole groups per 3 words).  The launch block and RangeDesc are
// shared with the mod-30 kernels: Bbase is the first group (lo / 210), corr
// counts 2, 3, 5 and 7, and SieveLaunch::seg_bytes is the segment's size in
// bytes (a multiple of 12).
constexpr uint32_t kW210Period = 46189u;            // 11 * 13 * 17 * 19 groups
constexpr uint32_t kW210PeriodBytes = 277134u;      // 6 bytes per group
constexpr uint32_t kW210MaxSegmentBytes = 229368u;  // 57342 words (a multiple of 3)
constexpr uint32_t kW210MaxSmemBytes = 229376u;     // the segment rounded up to 16-byte copies
// Group 0 as it must read after sieving: the residues 1, 121, 143, 169, 187 and
// 209 (bits 0, 27, 32, 38, 42, 47) are not prime, the other 42 are.
constexpr uint32_t kW210Group0Lo = 0xf7fffffeu;  // bits 0..31
constexpr uint32_t kW210Group0Hi = 0x7bbeu;      // bits 32..47
struct W210Tables {
    uint16_t step[48 * 48];  // [class of p][k]: bit of class k | dadj_k << 6 | (gap_k / 2) << 10
    uint8_t adj[48 * 48];    // [class of p][k]: floor(r_pc r_k / 210)
    uint8_t bit[48 * 48];    // [class of p][k]: index of (r_pc r_k) mod 210
    uint8_t idx[210];        // residue -> index, 0xff if not coprime to 210
    uint8_t cnt[210];        // v -> #{ i : r_i <= v }
    uint8_t r48[48];         // the residues
};
void build_w210_tables(W210Tables *t);  // host
cudaError_t set_sieve210_smem_limit();
cudaError_t launch_sieve210(const SieveLaunch *d_launch, const W210Tables *tab, const uint8_t *tile,
                            uint64_t tile_stride, int grid, int threads, uint32_t seg_bytes, cudaStream_t stream);
cudaError_t launch_build_tile210(const W210Tables *tab, uint8_t *tile, uint64_t stride, uint32_t len,
                                 cudaStream_t stream);

// Self-test of the bounded mbarrier wait used by the sieve's bulk copies
// (sieve_kernels.cu): *status_dev = 0 if the wait completed, 1 if it hit `limit`.
cudaError_t launch_wait_selftest(const void *src, uint32_t bytes, int arm, uint32_t limit, int *status_dev,
                                 cudaStream_t stream);

// Compaction of an odd-only bitmap into a prime list.
constexpr uint32_t kCompactTileWords = 2048;  // 256 threads x 8 words
cudaError_t launch_tile_popc(const uint32_t *bitmap, uint64_t nwords, uint32_t *tile_counts,
                             uint64_t ntiles, int grid, cudaStream_t stream);
cudaError_t launch_tile_scan(uint32_t *tile_counts, uint64_t *tile_offsets, uint64_t ntiles,
                             unsigned long long *total, cudaStream_t stream);
// Single-pass compaction (tile offsets by decoupled look-back, no popcount pass or
// scan): the first min(n, cap) values written, n (or UINT64_MAX if a look-back gave
// up) to *n_out.  status: ntiles + 1 words, zeroed before the launch.
cudaError_t launch_emit_onepass(const uint32_t *bitmap, uint64_t nwords, uint64_t ntiles, uint64_t o0,
                                uint32_t base_index, void *out, int out64, int num_sms, cudaStream_t stream, uint64_t cap,
                                uint64_t two, unsigned long long *status, uint64_t *n_out);
// *n = (*total, or 0 if total is null) + add: the device-side count of the asynchronous compaction.
cudaError_t launch_store_count(const unsigned long long *total, uint32_t add, uint64_t *n, cudaStream_t stream);
// With total != null, writes only if *total + base_index <= cap (else nothing).
// base_index = 1 also puts `two` at out[0]; n_out (if set) = *total + base_index.
cudaError_t launch_emit(const uint32_t *bitmap, uint64_t nwords, const uint64_t *tile_offsets,
                        uint64_t ntiles, uint64_t o0, uint32_t base_index, void *out,
                        int out64, int num_sms, cudaStream_t stream,
                        const unsigned long long *total = nullptr, uint64_t cap = 0, uint64_t two = 2,
                        uint64_t *n_out = nullptr);
// out[0] = 2 - sub (sub: the value base a list is written relative to, 0 for primes).
cudaError_t launch_put_two(void *out, int out64, cudaStream_t stream, uint64_t sub = 0);
// A launch block of at most kUploadMaxBytes (a multiple of 8), copied from host
// memory into the kernel's parameters at the call, written to dst; acc[0 .. acc_n)
// zeroed.  The host block may be rewritten as soon as this returns.
constexpr size_t kUploadMaxBytes = 2048;
cudaError_t launch_upload(void *dst, const void *src, size_t bytes, unsigned long long *acc, size_t acc_n,
                          cudaStream_t stream);
// *out = *count, or UINT64_MAX when *overflow is set.
cudaError_t launch_finalize_count(const unsigned long long *count, const unsigned *overflow, uint64_t *out,
                                  cudaStream_t stream);

}  // namespace gbs
