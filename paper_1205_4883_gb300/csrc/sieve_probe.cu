// sieve_probe.cu -- measured roofline denominators for the sieve's kernels.
//
// The count kernel's work is single-bit clears in shared memory (atomicAnd on
// 32-bit words), and the bitmap and list kernels write HBM.  These probes
// measure what one GB300 sustains for those operations, so that a kernel's
// rate can be set against a measured ceiling as well as the nominal one
// (32 lanes per clock per SM):
//   - shared-memory atomicAnd, each lane of a warp on its own bank (no
//     conflicts), and on random words (the access pattern of one lane per
//     prime);
//   - conflict-free plain 32-bit shared-memory stores;
//   - write-only HBM bandwidth, 16-byte stores over a caller buffer.
// The shared-memory probes run one CTA of 1024 threads per SM on 64 KiB of
// words and time themselves with clock64(), so they report lane operations
// per SM clock, independent of the clock the GPU runs at.

#include <cstdint>

#include "gbsieve.h"
#include "host.h"

namespace gbs {
namespace {

constexpr uint32_t kProbeWords = 16384;  // 64 KiB of shared memory
constexpr uint32_t kProbeThreads = 1024;

// A 32-bit mixing step (the "lowbias32" finaliser: xor-shift-multiply rounds).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// kind 1: conflict-free atomicAnd; 2: random-word atomicAnd; 3: conflict-free store.
// cycles[blockIdx.x] = SM clocks between the two barriers around the loop.  The
// loops are unrolled eight ways with immediate offsets so that address arithmetic
// stays well below one instruction per operation: the probe measures the shared
// memory pipe, not the issue rate.
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, 1) k_smem_probe(uint32_t iters, unsigned long long *cycles,
                                                                 uint32_t *sink) {
    extern __shared__ uint32_t w[];  // kProbeWords words (dynamic: above the 48 KiB static limit)
    for (uint32_t i = threadIdx.x; i < kProbeWords; i += blockDim.x) w[i] = 0xffffffffu;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t mask = ~(1u << lane);
    // conflict-free: lane l on bank l, rows r .. r + 7 of 504 (so r + 7 < 512 needs no wrap)
    uint32_t r = (warp * 17u) % 504u;
    // random: eight independent linear congruential streams, each one step per round
    uint32_t h[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) h[u] = mix32(threadIdx.x * 8u + u + 977u * blockIdx.x);
    __syncthreads();
    const long long t0 = clock64();
    for (uint32_t i = 0; i < iters; i += 8) {
        if (KIND == 2) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                h[u] = h[u] * 1664525u + 1013904223u;
                atomicAnd(&w[h[u] >> 18], mask);
            }
        } else {
            uint32_t *row = w + 32u * r + lane;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (KIND == 1)
                    atomicAnd(row + 32 * u, mask);
                else
                    row[32 * u] = i + u;
            }
            r += 8;
            if (r >= 504u) r -= 504u;
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
    uint32_t acc = 0;
    for (uint32_t i = threadIdx.x; i < kProbeWords; i += blockDim.x) acc ^= w[i];
    if (acc == 0x12345678u) sink[0] = acc;  // keeps the loop's results observable
}

__global__ void k_hbm_write(uint4 *buf, uint64_t n16, uint32_t v) {
    const uint4 x = make_uint4(v, v ^ 1u, v ^ 2u, v ^ 3u);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16; i += (uint64_t)gridDim.x * blockDim.x)
        buf[i] = x;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" int sieve_probe(sieve_ctx *ctx, int kind, void *buf_dev, uint64_t bytes, double *value) {
    if (!ctx || !value) return SIEVE_EINVAL;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const int sms = ctx->num_sms;
    cudaStream_t st = ctx->stream;
    if (kind == SIEVE_PROBE_HBM_WRITE) {
        if (!buf_dev || bytes < (1u << 20) || (reinterpret_cast<uintptr_t>(buf_dev) & 15u))
            return fail(ctx, SIEVE_EINVAL, "probe buffer: 16-byte aligned, at least 1 MiB");
        const uint64_t n16 = bytes / 16;
        cudaEvent_t a = nullptr, b = nullptr;
        if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            return cuda_fail(ctx, e, "cudaEventCreate");
        }
        float best = 0.f;
        for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
            cudaEventRecord(a, st);
            k_hbm_write<<<sms * 8, 512, 0, st>>>(static_cast<uint4 *>(buf_dev), n16, (uint32_t)rep);
            cudaEventRecord(b, st);
            e = cudaEventSynchronize(b);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // rep 0 is a warm-up
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "HBM write probe");
        *value = (double)(n16 * 16) / (best * 1e-3) / 1e9;  // GB/s
        return SIEVE_OK;
    }
    if (kind != SIEVE_PROBE_SMEM_AND_CONFLICT_FREE && kind != SIEVE_PROBE_SMEM_AND_RANDOM &&
        kind != SIEVE_PROBE_SMEM_STORE_CONFLICT_FREE)
        return fail(ctx, SIEVE_EINVAL, "unknown probe kind");
    unsigned long long *d_cycles = nullptr;
    uint32_t *d_sink = nullptr;
    if ((e = cudaMalloc(&d_cycles, sms * sizeof(unsigned long long))) != cudaSuccess)
        return cuda_fail(ctx, e, "cudaMalloc");
    if ((e = cudaMalloc(&d_sink, sizeof(uint32_t))) != cudaSuccess) {
        cudaFree(d_cycles);
        return cuda_fail(ctx, e, "cudaMalloc");
    }
    const uint32_t iters = 1u << 14;
    const int smem = (int)(kProbeWords * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_smem_probe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_smem_probe<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_smem_probe<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    double best = 0.0;
    std::vector<unsigned long long> cyc(sms);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        if (kind == SIEVE_PROBE_SMEM_AND_CONFLICT_FREE)
            k_smem_probe<1><<<sms, kProbeThreads, smem, st>>>(iters, d_cycles, d_sink);
        else if (kind == SIEVE_PROBE_SMEM_AND_RANDOM)
            k_smem_probe<2><<<sms, kProbeThreads, smem, st>>>(iters, d_cycles, d_sink);
        else
            k_smem_probe<3><<<sms, kProbeThreads, smem, st>>>(iters, d_cycles, d_sink);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cyc.data(), d_cycles, sms * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        unsigned long long mx = 1;
        for (int i = 0; i < sms; ++i) mx = cyc[i] > mx ? cyc[i] : mx;
        const double rate = (double)kProbeThreads * iters / (double)mx;  // lane-ops per clock per SM
        if (rate > best) best = rate;
    }
    cudaFree(d_cycles);
    cudaFree(d_sink);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "shared-memory probe");
    *value = best;
    return SIEVE_OK;
}
