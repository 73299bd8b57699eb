// sieve_compact.cu -- odd-only bitmap -> ascending prime list.
//
// The bitmap is cut into tiles of kCompactTileWords words.  Pass 1 counts the
// set bits of every tile, pass 2 scans the tile counts into tile offsets (one
// CTA), pass 3 re-reads each tile and writes, for bit i of the bitmap, the
// prime o0 + 2 i at its rank.  In passes 1 and 3 a CTA of 256 threads takes a
// tile and warp w the tile's words [256 w, 256 w + 256).  In pass 1 lane l
// holds word 32 k + l of chunk k (every load instruction reads 128 contiguous
// bytes); in pass 3 it holds eight consecutive words (k_emit).
#include "internal.h"

#include <atomic>

namespace gbs {
namespace {

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_inclusive_scan_u32(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

static_assert(kCompactTileWords == 256 * 8, "a tile is 8 warps x 8 chunks x 32 words");

__global__ void __launch_bounds__(256) k_tile_popc(const uint32_t *__restrict__ bitmap, uint64_t nwords,
                                                   uint32_t *__restrict__ tile_counts, uint64_t ntiles) {
    __shared__ uint32_t s_warp[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t base = t * kCompactTileWords + 256ull * warp + lane;
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint64_t w = base + 32ull * k;
            if (w < nwords) c += __popc(__ldg(bitmap + w));
        }
        c = warp_sum_u32(c);
        if (lane == 0) s_warp[warp] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t total = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) total += s_warp[i];
            tile_counts[t] = total;
        }
        __syncthreads();
    }
}

// Exclusive scan of the tile counts and the grand total: one CTA of 1024
// threads, 32 counts per thread per round (32768 tiles a round, the 2^26 words
// of [0, 2^32) in one).  A round stages its counts in shared memory with a
// coalesced load, count i at i + i / 32 (so that the 32 consecutive counts a
// thread scans lie in 32 different banks), scans them there, and writes the
// offsets with a coalesced store.  Within a round the prefixes fit 32 bits: a
// tile holds at most 65536 set bits.
constexpr uint32_t kScanItems = 32;
constexpr uint32_t kScanThreads = 1024;
constexpr uint32_t kScanRound = kScanThreads * kScanItems;
constexpr uint32_t kScanSmemBytes = (kScanRound + kScanRound / 32) * sizeof(uint32_t);

__device__ __forceinline__ uint32_t scan_slot(uint32_t i) { return i + (i >> 5); }

__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const uint32_t *tile_counts, uint64_t *tile_offsets,
                                                            uint64_t ntiles, unsigned long long *total) {
    extern __shared__ uint32_t s_cnt[];  // kScanRound counts, padded
    __shared__ uint32_t s_warp[32];
    __shared__ unsigned long long s_run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_run = 0;
    for (uint64_t base = 0; base < ntiles; base += kScanRound) {
#pragma unroll 8
        for (uint32_t i = threadIdx.x; i < kScanRound; i += kScanThreads)  // 8 loads in flight per thread
            s_cnt[scan_slot(i)] = base + i < ntiles ? tile_counts[base + i] : 0u;
        __syncthreads();
        const uint32_t t0 = threadIdx.x * kScanItems;
        uint32_t sum = 0;
#pragma unroll 8
        for (uint32_t k = 0; k < kScanItems; ++k) sum += s_cnt[scan_slot(t0 + k)];
        const uint32_t incl = warp_inclusive_scan_u32(sum, lane);
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t wbase = 0, all = 0;
        for (int w = 0; w < (int)(kScanThreads / 32); ++w) {
            const uint32_t x = s_warp[w];
            if (w < warp) wbase += x;
            all += x;
        }
        uint32_t run = wbase + incl - sum;  // exclusive prefix of this thread's first count
#pragma unroll 8
        for (uint32_t k = 0; k < kScanItems; ++k) {
            const uint32_t slot = scan_slot(t0 + k), c = s_cnt[slot];
            s_cnt[slot] = run;
            run += c;
        }
        __syncthreads();
        const unsigned long long r0 = s_run;
        for (uint32_t i = threadIdx.x; i < kScanRound && base + i < ntiles; i += kScanThreads)
            tile_offsets[base + i] = r0 + s_cnt[scan_slot(i)];
        __syncthreads();  // every thread has read s_run and s_cnt
        if (threadIdx.x == 0) s_run = r0 + all;
    }
    __syncthreads();
    if (threadIdx.x == 0) *total = s_run;
}

// Primes a warp stages in shared memory before writing them out as one
// contiguous run (a warp's 256 words hold more only near 0; then it writes
// directly).
constexpr uint32_t kEmitStage = 1024;

// The primes of one lane's eight words, written downwards from p (exclusive):
// words 7 .. 0, in each word its set bits from the highest, so the values land
// in ascending order.  v is the integer of bit 0 of word 0.
template <typename T, typename V>
__device__ __forceinline__ void emit_lane_desc(const uint32_t (&w)[8], V v, T *p) {
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        const V vk = v + (V)(64u * (uint32_t)k);
        for (uint32_t x = w[k]; x;) {
            const uint32_t b = 31u - (uint32_t)__clz(x);
            *--p = (T)(vk + (V)(2u * b));
            x ^= 1u << b;
        }
    }
}

// Pass 3.  Warp w of a CTA takes words [256 w, 256 w + 256) of the tile, lane l
// the eight consecutive words 8 l .. 8 l + 7 of those (two 16-byte loads per
// lane, so a load instruction reads 512 contiguous bytes).  One warp scan of the
// lanes' popcounts ranks every prime of the warp's words; each lane writes its
// primes into the warp's stage in shared memory, and the warp copies the stage
// out as one contiguous run.  The warps' prime counts go through a two-slot
// table (by tile parity), so one barrier per tile suffices: a warp can be at
// most one tile ahead of another.  With total != null the list is written only
// if it fits: *total (from k_tile_scan) + base_index <= cap; otherwise the
// kernel writes nothing, so the host can launch it before it has read the total.
// base_index = 1 puts `two` (the prime 2, less the value base) at out[0]; n_out,
// if set, receives *total + base_index, the list's length.
template <typename T>
__global__ void __launch_bounds__(256) k_emit(const uint32_t *__restrict__ bitmap, uint64_t nwords,
                                              const uint64_t *__restrict__ tile_offsets, uint64_t ntiles,
                                              uint64_t o0, uint32_t base_index, T *__restrict__ out,
                                              const unsigned long long *total, uint64_t cap, T two,
                                              uint64_t *n_out) {
    __shared__ uint32_t s_warp[2][8];
    extern __shared__ __align__(16) unsigned char s_dyn[];  // 8 stages of kEmitStage entries
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (n_out) *n_out = (total ? *total : 0ull) + base_index;
        if (base_index && (!total || *total + base_index <= cap)) out[0] = two;
    }
    if (total && *total + base_index > cap) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(bitmap) & 15u) == 0;
    T *const stage = reinterpret_cast<T *>(s_dyn) + (size_t)warp * kEmitStage;
    uint32_t par = 0;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, par ^= 1u) {
        const uint64_t w0 = t * kCompactTileWords + 256ull * warp + 8ull * lane;  // this lane's first word
        const uint64_t toff = tile_offsets[t];
        uint32_t w[8];
        if (vec && w0 + 8 <= nwords) {
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(bitmap + w0));
            const uint4 b = __ldg(reinterpret_cast<const uint4 *>(bitmap + w0) + 1);
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
            w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) w[k] = w0 + k < nwords ? __ldg(bitmap + w0 + k) : 0u;
        }
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) c += __popc(w[k]);
        const uint32_t incl = warp_inclusive_scan_u32(c, lane);
        const uint32_t n = __shfl_sync(0xffffffffu, incl, 31);  // primes in the warp's 256 words
        if (lane == 0) s_warp[par][warp] = n;
        __syncthreads();
        uint64_t first = base_index + toff;  // rank of the warp's first prime
        for (int i = 0; i < warp; ++i) first += s_warp[par][i];
        const uint64_t v = o0 + 64ull * w0;  // integer of bit 0 of the lane's first word
        if (n <= kEmitStage) {
            if (sizeof(T) == 4)
                emit_lane_desc(w, (uint32_t)v, stage + incl);  // a 32-bit list holds values below 2^32
            else
                emit_lane_desc(w, v, stage + incl);
            __syncwarp();
            T *const o = out + first;
            uint32_t i = lane;
            for (; i + 96 < n; i += 128) {
                const T a0 = stage[i], a1 = stage[i + 32], a2 = stage[i + 64], a3 = stage[i + 96];
                o[i] = a0; o[i + 32] = a1; o[i + 64] = a2; o[i + 96] = a3;
            }
            for (; i < n; i += 32) o[i] = stage[i];
            __syncwarp();  // the stage is refilled by the next tile
        } else {
            if (sizeof(T) == 4)
                emit_lane_desc(w, (uint32_t)v, out + first + incl);
            else
                emit_lane_desc(w, v, out + first + incl);
        }
    }
}

}  // namespace

cudaError_t launch_tile_popc(const uint32_t *bitmap, uint64_t nwords, uint32_t *tile_counts, uint64_t ntiles,
                             int grid, cudaStream_t stream) {
    if (ntiles == 0) return cudaSuccess;
    const unsigned g = (unsigned)(ntiles < (uint64_t)grid ? ntiles : (uint64_t)grid);
    k_tile_popc<<<g, 256, 0, stream>>>(bitmap, nwords, tile_counts, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_tile_scan(uint32_t *tile_counts, uint64_t *tile_offsets, uint64_t ntiles,
                             unsigned long long *total, cudaStream_t stream) {
    // 132 KiB of counts: above the default 48 KiB (the attribute belongs to the current device)
    cudaError_t e = cudaFuncSetAttribute(k_tile_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, kScanSmemBytes);
    if (e != cudaSuccess) return e;
    k_tile_scan<<<1, kScanThreads, kScanSmemBytes, stream>>>(tile_counts, tile_offsets, ntiles, total);
    return cudaGetLastError();
}

// As emit_lane_desc, for a list truncated at cap: the lane's primes have ranks
// [end - count, end); only those below cap are written.
template <typename T, typename V>
__device__ __forceinline__ void emit_lane_desc_capped(const uint32_t (&w)[8], V v, T *out, uint64_t end,
                                                      uint64_t cap) {
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        const V vk = v + (V)(64u * (uint32_t)k);
        for (uint32_t x = w[k]; x;) {
            const uint32_t b = 31u - (uint32_t)__clz(x);
            if (--end < cap) out[end] = (T)(vk + (V)(2u * b));
            x ^= 1u << b;
        }
    }
}

// Tile status words of the single-pass compaction: the top two bits say what the
// low 62 hold (0: nothing yet, 1: the tile's own count, 2: the count of all tiles
// up to and including it); an all-ones value is a poisoned prefix.
constexpr unsigned long long kTileAgg = 1ull << 62, kTilePrefix = 2ull << 62;
constexpr unsigned long long kTileValue = (1ull << 62) - 1;
// Polls of one predecessor's status before the look-back gives up (about a second).
constexpr uint32_t kLookbackPolls = 1u << 20;

// Single-pass compaction (decoupled look-back; Merrill and Garland, "Single-pass
// parallel prefix scan with decoupled look-back", 2016).  CTAs claim tiles in
// order from a counter (status[ntiles]); a tile's count is published at once,
// then its first thread adds up the counts of the tiles before it, walking back
// to the nearest published prefix, and publishes its own.  A tile is claimed only
// by a running CTA, so every status a look-back waits for is being written.  The
// primes are emitted as in k_emit; ranks at or above cap are not written (a list
// that does not fit is truncated).  base_index = 1 puts `two` at out[0]; the last
// tile writes the list's length (or UINT64_MAX if a look-back gave up) to *n_out.
// status: ntiles + 1 words, zeroed before the launch.
// CTA of the single-pass compaction: eight warps that emit (as in k_emit) and
// one that publishes the tile's count and looks back for its offset meanwhile.
constexpr uint32_t kOnePassThreads = 288;

template <typename T>
__global__ void __launch_bounds__(kOnePassThreads) k_emit_onepass(const uint32_t *__restrict__ bitmap, uint64_t nwords,
                                                      uint64_t ntiles, uint64_t o0, uint32_t base_index,
                                                      T *__restrict__ out, uint64_t cap, T two,
                                                      unsigned long long *status, uint64_t *n_out) {
    __shared__ uint32_t s_warp[2][8];
    __shared__ unsigned long long s_tile, s_prefix;
    extern __shared__ __align__(16) unsigned char s_dyn[];  // 8 stages of kEmitStage entries
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;  // warp 8 looks back
    const bool vec = (reinterpret_cast<uintptr_t>(bitmap) & 15u) == 0;
    T *const stage = reinterpret_cast<T *>(s_dyn) + (size_t)(warp < 8 ? warp : 0) * kEmitStage;
    if (blockIdx.x == 0 && threadIdx.x == 0 && base_index && cap) out[0] = two;
    uint32_t par = 0;
    for (;; par ^= 1u) {
        if (threadIdx.x == 0) s_tile = atomicAdd(status + ntiles, 1ull);
        __syncthreads();
        const uint64_t t = s_tile;
        if (t >= ntiles) break;
        const uint64_t w0 = t * kCompactTileWords + 256ull * warp + 8ull * lane;  // this lane's first word
        uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        uint32_t c = 0, incl = 0, n = 0;
        if (warp < 8) {
            if (vec && w0 + 8 <= nwords) {
                const uint4 a = __ldg(reinterpret_cast<const uint4 *>(bitmap + w0));
                const uint4 b = __ldg(reinterpret_cast<const uint4 *>(bitmap + w0) + 1);
                w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
                w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) w[k] = w0 + k < nwords ? __ldg(bitmap + w0 + k) : 0u;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) c += __popc(w[k]);
            incl = warp_inclusive_scan_u32(c, lane);
            n = __shfl_sync(0xffffffffu, incl, 31);
            if (lane == 0) s_warp[par][warp] = n;
        }
        __syncthreads();
        const uint64_t v = o0 + 64ull * w0;
        if (warp == 8) {  // the look-back, 32 statuses per step
            unsigned long long agg = 0;
            for (int i = 0; i < 8; ++i) agg += s_warp[par][i];
            unsigned long long prefix = 0;
            bool poisoned = false;
            const unsigned long long published = t == 0 ? 2ull << 62 : 1ull << 62;  // prefix, or own count
            if (lane == 0) atomicExch(status + t, published | agg);
            if (t > 0) {
                for (int64_t hi_j = (int64_t)t - 1;; hi_j -= 32) {
                    const int64_t j = hi_j - lane;  // lane 0 reads the nearest tile
                    volatile unsigned long long *sj = status + (j >= 0 ? j : 0);
                    unsigned long long x0 = 2ull << 62;  // before tile 0: a prefix of 0
                    if (j >= 0) x0 = *sj;
                    for (uint32_t polls = 0; __any_sync(0xffffffffu, (x0 >> 62) == 0);) {
                        if (++polls >= kLookbackPolls) break;
                        __nanosleep(64);
                        if ((x0 >> 62) == 0) x0 = *sj;
                    }
                    const bool bad = (x0 >> 62) == 0 || x0 == (kTilePrefix | kTileValue);
                    if (__any_sync(0xffffffffu, bad)) {  // gave up, or a poisoned prefix
                        poisoned = true;
                        break;
                    }
                    const uint32_t pm = __ballot_sync(0xffffffffu, (x0 >> 62) == 2);
                    const int stop = pm ? __ffs(pm) - 1 : 31;  // the nearest prefix, or the whole window
                    unsigned long long x = lane <= stop ? (x0 & kTileValue) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                    prefix += x;
                    if (pm) break;
                }
                if (lane == 0) {
                    __threadfence();
                    atomicExch(status + t, kTilePrefix | (poisoned ? kTileValue : (prefix + agg) & kTileValue));
                }
            }
            if (lane == 0) {
                s_prefix = poisoned ? ~0ull : prefix;
                if (t == ntiles - 1 && n_out) *n_out = poisoned ? ~0ull : prefix + agg + base_index;
            }
        } else if (n <= kEmitStage) {  // meanwhile the primes into the stages (no offset needed)
            if (sizeof(T) == 4)
                emit_lane_desc(w, (uint32_t)v, stage + incl);
            else
                emit_lane_desc(w, v, stage + incl);
        }
        __syncthreads();
        if (warp == 8) continue;
        const unsigned long long prefix = s_prefix;
        if (prefix == ~0ull) continue;  // a look-back gave up: this tile writes nothing
        uint64_t first = base_index + prefix;  // rank of the warp's first prime
        for (int i = 0; i < warp; ++i) first += s_warp[par][i];
        if (first >= cap) continue;
        if (n <= kEmitStage) {
            const uint32_t lim = first + n <= cap ? n : (uint32_t)(cap - first);
            T *const o = out + first;
            uint32_t i = lane;
            for (; i + 96 < lim; i += 128) {
                const T a0 = stage[i], a1 = stage[i + 32], a2 = stage[i + 64], a3 = stage[i + 96];
                o[i] = a0; o[i + 32] = a1; o[i + 64] = a2; o[i + 96] = a3;
            }
            for (; i < lim; i += 32) o[i] = stage[i];
        } else if (sizeof(T) == 4) {
            emit_lane_desc_capped(w, (uint32_t)v, out, first + incl, cap);
        } else {
            emit_lane_desc_capped(w, v, out, first + incl, cap);
        }
    }
}

namespace {
// CTAs of kernel k (k_emit<T> or k_emit_onepass<T>) resident per SM with its
// stage (the grid is that many per SM: one wave, no tail of CTAs that start
// after the first ones have finished).  The shared-memory attribute is set on
// every call (it belongs to the current device); the occupancy is the same on
// every device of the one supported architecture.
template <typename T, typename K>
cudaError_t ctas_per_sm(K k, int threads, std::atomic<int> &cached, int *per_sm) {
    const int smem = 8 * kEmitStage * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int n = cached.load(std::memory_order_relaxed);
    if (n <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem);
        if (e != cudaSuccess) return e;
        if (n <= 0) n = 1;
        cached.store(n, std::memory_order_relaxed);
    }
    *per_sm = n;
    return cudaSuccess;
}

template <typename T>
cudaError_t emit_ctas_per_sm(int *per_sm) {
    static std::atomic<int> cached{0};
    return ctas_per_sm<T>(k_emit<T>, 256, cached, per_sm);
}

template <typename T>
cudaError_t onepass_ctas_per_sm(int *per_sm) {
    static std::atomic<int> cached{0};
    return ctas_per_sm<T>(k_emit_onepass<T>, (int)kOnePassThreads, cached, per_sm);
}
}  // namespace

cudaError_t launch_emit(const uint32_t *bitmap, uint64_t nwords, const uint64_t *tile_offsets, uint64_t ntiles,
                        uint64_t o0, uint32_t base_index, void *out, int out64, int num_sms, cudaStream_t stream,
                        const unsigned long long *total, uint64_t cap, uint64_t two, uint64_t *n_out) {
    if (ntiles == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = out64 ? emit_ctas_per_sm<uint64_t>(&per_sm) : emit_ctas_per_sm<uint32_t>(&per_sm);
    if (e != cudaSuccess) return e;
    const uint64_t grid = (uint64_t)num_sms * per_sm;
    const unsigned g = (unsigned)(ntiles < grid ? ntiles : grid);
    if (out64) {
        const int smem = 8 * kEmitStage * sizeof(uint64_t);  // 64 KiB: above the default 48 KiB
        k_emit<uint64_t><<<g, 256, smem, stream>>>(bitmap, nwords, tile_offsets, ntiles, o0, base_index,
                                                   static_cast<uint64_t *>(out), total, cap, two, n_out);
    } else {
        const int smem = 8 * kEmitStage * sizeof(uint32_t);
        k_emit<uint32_t><<<g, 256, smem, stream>>>(bitmap, nwords, tile_offsets, ntiles, o0, base_index,
                                                   static_cast<uint32_t *>(out), total, cap, (uint32_t)two, n_out);
    }
    return cudaGetLastError();
}

cudaError_t launch_emit_onepass(const uint32_t *bitmap, uint64_t nwords, uint64_t ntiles, uint64_t o0,
                                uint32_t base_index, void *out, int out64, int num_sms, cudaStream_t stream, uint64_t cap,
                                uint64_t two, unsigned long long *status, uint64_t *n_out) {
    if (ntiles == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = out64 ? onepass_ctas_per_sm<uint64_t>(&per_sm) : onepass_ctas_per_sm<uint32_t>(&per_sm);
    if (e != cudaSuccess) return e;
    const uint64_t grid = (uint64_t)num_sms * per_sm;
    const unsigned g = (unsigned)(ntiles < grid ? ntiles : grid);
    if (out64) {
        k_emit_onepass<uint64_t><<<g, kOnePassThreads, 8 * kEmitStage * sizeof(uint64_t), stream>>>(
            bitmap, nwords, ntiles, o0, base_index, static_cast<uint64_t *>(out), cap, two, status, n_out);
    } else {
        k_emit_onepass<uint32_t><<<g, kOnePassThreads, 8 * kEmitStage * sizeof(uint32_t), stream>>>(
            bitmap, nwords, ntiles, o0, base_index, static_cast<uint32_t *>(out), cap, (uint32_t)two, status, n_out);
    }
    return cudaGetLastError();
}

namespace {
__global__ void k_store_count(const unsigned long long *total, uint32_t add, uint64_t *n) {
    *n = (total ? *total : 0ull) + add;
}
}  // namespace

cudaError_t launch_store_count(const unsigned long long *total, uint32_t add, uint64_t *n, cudaStream_t stream) {
    k_store_count<<<1, 1, 0, stream>>>(total, add, n);
    return cudaGetLastError();
}

}  // namespace gbs
