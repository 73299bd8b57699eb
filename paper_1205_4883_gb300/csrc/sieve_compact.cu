// sieve_compact.cu -- odd-only bitmap -> ascending prime list.
//
// The bitmap is cut into tiles of kCompactTileWords words.  Pass 1 counts the
// set bits of every tile, pass 2 scans the tile counts into tile offsets (one
// CTA), pass 3 re-reads each tile and writes, for bit i of the bitmap, the
// prime o0 + 2 i at its rank.  In passes 1 and 3 a CTA of 256 threads takes a
// tile; warp w takes the tile's words [256 w, 256 w + 256) as eight chunks of
// 32, lane l holding word 32 k + l of chunk k, so every load instruction reads
// 128 contiguous bytes.  The primes of a chunk are ranked by a warp scan in
// word order, gathered in shared memory and written out as one contiguous run.
#include "internal.h"

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
// threads, each taking 8 consecutive counts per round (8192 tiles a round).
constexpr uint32_t kScanItems = 8;

__global__ void __launch_bounds__(1024) k_tile_scan(const uint32_t *tile_counts, uint64_t *tile_offsets,
                                                    uint64_t ntiles, unsigned long long *total) {
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (uint64_t base = 0; base < ntiles; base += (uint64_t)blockDim.x * kScanItems) {
        const uint64_t t0 = base + (uint64_t)threadIdx.x * kScanItems;
        uint32_t v[kScanItems];
        unsigned long long sum = 0;
#pragma unroll
        for (uint32_t i = 0; i < kScanItems; ++i) {
            v[i] = t0 + i < ntiles ? tile_counts[t0 + i] : 0u;
            sum += v[i];
        }
        unsigned long long x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        unsigned long long wbase = 0, all = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) wbase += s_warp[w];
            all += s_warp[w];
        }
        unsigned long long run = s_run + wbase + x - sum;
#pragma unroll
        for (uint32_t i = 0; i < kScanItems; ++i) {
            if (t0 + i < ntiles) tile_offsets[t0 + i] = run;
            run += v[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_run += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s_run;
}

// Primes a warp stages in shared memory per chunk before writing them out as
// one contiguous run (a denser chunk is written directly).
constexpr uint32_t kEmitStage = 512;

template <typename T>
__global__ void __launch_bounds__(256) k_emit(const uint32_t *__restrict__ bitmap, uint64_t nwords,
                                              const uint64_t *__restrict__ tile_offsets, uint64_t ntiles,
                                              uint64_t o0, uint32_t base_index, T *__restrict__ out) {
    __shared__ uint32_t s_warp[8];
    __shared__ T s_stage[8][kEmitStage];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t base = t * kCompactTileWords + 256ull * warp;
        uint32_t w[8];
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint64_t i = base + 32ull * k + lane;
            w[k] = i < nwords ? __ldg(bitmap + i) : 0u;
            c += __popc(w[k]);
        }
        c = warp_sum_u32(c);
        if (lane == 0) s_warp[warp] = c;
        __syncthreads();
        uint32_t before = 0;  // primes of the tile's earlier warps
        for (int i = 0; i < warp; ++i) before += s_warp[i];
        uint64_t chunk = base_index + tile_offsets[t] + before;  // rank of the chunk's first prime
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t v = w[k], cv = __popc(v);
            const uint32_t incl = warp_inclusive_scan_u32(cv, lane);
            const uint32_t n = __shfl_sync(0xffffffffu, incl, 31);  // primes in the chunk
            const uint64_t first = o0 + 64ull * (base + 32ull * k + lane);  // integer of the word's bit 0
            if (n <= kEmitStage) {
                T *stage = s_stage[warp];
                uint32_t j = incl - cv;
                for (uint32_t x = v; x; x &= x - 1) stage[j++] = (T)(first + 2ull * (uint32_t)(__ffs(x) - 1));
                __syncwarp();
                for (uint32_t i = lane; i < n; i += 32) out[chunk + i] = stage[i];
                __syncwarp();
            } else {
                uint64_t pos = chunk + incl - cv;
                for (uint32_t x = v; x; x &= x - 1) out[pos++] = (T)(first + 2ull * (uint32_t)(__ffs(x) - 1));
            }
            chunk += n;
        }
        __syncthreads();
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
    k_tile_scan<<<1, 1024, 0, stream>>>(tile_counts, tile_offsets, ntiles, total);
    return cudaGetLastError();
}

cudaError_t launch_emit(const uint32_t *bitmap, uint64_t nwords, const uint64_t *tile_offsets, uint64_t ntiles,
                        uint64_t o0, uint32_t base_index, void *out, int out64, int grid, cudaStream_t stream) {
    if (ntiles == 0) return cudaSuccess;
    const unsigned g = (unsigned)(ntiles < (uint64_t)grid ? ntiles : (uint64_t)grid);
    if (out64)
        k_emit<uint64_t><<<g, 256, 0, stream>>>(bitmap, nwords, tile_offsets, ntiles, o0, base_index,
                                                static_cast<uint64_t *>(out));
    else
        k_emit<uint32_t><<<g, 256, 0, stream>>>(bitmap, nwords, tile_offsets, ntiles, o0, base_index,
                                                static_cast<uint32_t *>(out));
    return cudaGetLastError();
}

}  // namespace gbs
