// sieve_kernels.cu -- the GB300 kernels of the segmented sieve of Eratosthenes.
//
// Paper, Section 3.1: the sieve marks as composite the multiples of each
// prime; Section 1: primes <= sqrt(hi - 1) suffice for [lo, hi); Eq. 3: the
// integers are processed in blocks ("segments"), the last one short.
//
// Data layout: a segment is S consecutive mod-30 wheel bytes (30 S integers)
// in shared memory; wheel byte b, bit k <-> integer 30 b + r_k with
// r = {1, 7, 11, 13, 17, 19, 23, 29}.  Per segment a CTA
//   1. copies the pre-sieved pattern (multiples of 7, 11, 13, 17, 19 already
//      cleared; period 323323 bytes) from one of 16 byte-shifted copies held
//      in L2, so every copy is 16-byte aligned, with one cp.async.bulk;
//   2. crosses off, for every base prime p >= 23 and every wheel class j, the
//      arithmetic progression of multiples p m with m = r_j (mod 30), m >= p:
//      in wheel bytes it is c_j + p q (c_j = floor(p r_j / 30)) with a fixed
//      bit -- "small" primes (many hits per class) are crossed by a whole warp
//      striding over one progression, the rest by one thread per prime;
//   3. counts the surviving bits in [lo, hi) (__popc + warp shuffles) or
//      expands them into the odd-only bitmap in HBM.
// CTAs are persistent and take segments from a global counter.

#include "internal.h"

#include <cstring>

namespace gbs {
namespace {

__constant__ uint32_t c_res[8] = {1, 7, 11, 13, 17, 19, 23, 29};

struct WheelTables {
    uint16_t expand[256];  // wheel byte -> 15 odd-only bits (odd integers 30b+1 .. 30b+29)
    uint8_t adj[64];       // [class of p][j]: floor(r_c * r_j / 30)
    uint8_t bit[64];       // [class of p][j]: wheel bit of (r_c * r_j) mod 30
    uint8_t cls[32];       // residue mod 30 -> wheel class (0xff if not coprime)
    uint64_t adj40[8];     // [class of p]: adj[c][k] in 5-bit fields, k = 0..7
    uint32_t bits24[8];    // [class of p]: bit[c][k] in 3-bit fields, k = 0..7
    uint32_t dadj24[8];    // [class of p]: floor(r_c r_{k+1} / 30) - floor(r_c r_k / 30), 3-bit fields
};

// Gaps between consecutive residues coprime to 30 (1, 7, 11, ..., 29, 31) in
// 4-bit fields: 6, 4, 2, 4, 2, 4, 6, 2.
constexpr uint32_t kWheelGaps = 0x26424246u;
// Large primes a lane handles per pass of the large-prime loop (loads in flight).
constexpr uint32_t kLargeUnroll = 4;
// The residues 1, 7, 11, 13, 17, 19, 23, 29 in 5-bit fields.
constexpr uint64_t kRes40 = 1ull | 7ull << 5 | 11ull << 10 | 13ull << 15 | 17ull << 20 | 19ull << 25 | 23ull << 30 |
                            29ull << 35;

__device__ __forceinline__ int wheel_index(uint32_t r) {
    int k = -1;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (c_res[i] == r) k = i;
    return k;
}

__device__ void init_tables(WheelTables &t) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        uint32_t e = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (i & (1 << k)) e |= 1u << ((c_res[k] - 1) / 2);
        t.expand[i] = (uint16_t)e;
    }
    if (threadIdx.x < 64) {
        int c = threadIdx.x >> 3, j = threadIdx.x & 7;
        uint32_t prod = c_res[c] * c_res[j];
        t.adj[threadIdx.x] = (uint8_t)(prod / 30);
        t.bit[threadIdx.x] = (uint8_t)wheel_index(prod % 30);
    }
    if (threadIdx.x < 32) {
        int k = wheel_index(threadIdx.x);
        t.cls[threadIdx.x] = (uint8_t)(k < 0 ? 0xff : k);
    }
    if (threadIdx.x < 8) {
        const uint32_t rc = c_res[threadIdx.x];
        uint32_t bits = 0, dadj = 0;
        uint64_t adj = 0;
        for (int k = 0; k < 8; ++k) {
            adj |= (uint64_t)((rc * c_res[k]) / 30) << (5 * k);
            const uint32_t rk = c_res[k], rk1 = k < 7 ? c_res[k + 1] : 31u;
            bits |= (uint32_t)wheel_index((rc * rk) % 30) << (3 * k);
            dadj |= ((rc * rk1) / 30 - (rc * rk) / 30) << (3 * k);
        }
        t.adj40[threadIdx.x] = adj;
        t.bits24[threadIdx.x] = bits;
        t.dadj24[threadIdx.x] = dadj;
    }
    __syncthreads();
}

// x mod p by Barrett reduction with M = floor((2^64 - 1) / p): the quotient
// estimate umulhi(x, M) is floor(x / p) or one less, so one correction step.
__device__ __forceinline__ uint32_t mod_barrett(uint64_t x, uint32_t p, uint64_t M) {
    uint64_t q = __umul64hi(x, M);
    uint64_t r = x - q * (uint64_t)p;
    return (uint32_t)(r >= p ? r - p : r);
}

__device__ __forceinline__ void clear_bit(uint32_t *seg32, uint32_t off, uint32_t bit) {
    atomicAnd(&seg32[off >> 2], ~(1u << (((off & 3u) << 3) | bit)));
}

// Byte offset (relative to the segment start B0) of the first multiple of p
// in progression j, i.e. of the first p m >= max(p^2, 30 B0) with
// m = r_j (mod 30); R = max(B0, 0) mod p.  In wheel bytes the progression is
// c_j + p q with c_j = floor(p r_j / 30) = pq r_j + floor(r_c r_j / 30), so the
// offset is (c_j - R) mod p -- unless the segment starts before p^2 ("early",
// always the case when B0 < 0), when the start is clamped to the byte of the
// first multiple with m >= p.  Values >= L mean "no hit in this segment".
__device__ __forceinline__ uint32_t class_off(const WheelTables &t, uint32_t p, uint32_t pq, uint32_t pc, int j,
                                              uint32_t R, int64_t B0, bool early, uint32_t L) {
    const uint32_t rj = c_res[j];
    const uint32_t cj = pq * rj + (uint32_t)((t.adj40[pc] >> (5 * j)) & 31u);
    uint32_t d = cj - R;
    if ((int32_t)d < 0) d += p;
    if (!early) return d;
    const uint64_t Bc = B0 > 0 ? (uint64_t)B0 : 0;
    uint64_t start = Bc + d;
    const uint64_t q0 = p > rj ? (uint64_t)((p - rj + 29) / 30) : 0;  // m = 30 q + r_j >= p
    const uint64_t bmin = (uint64_t)p * q0 + cj;
    if (bmin > start) start = bmin;
    const int64_t off = (int64_t)start - B0;
    return off < (int64_t)L ? (uint32_t)off : L;
}

// All eight progressions of p in a segment that starts before p^2 (or before
// integer 0): the rare case, kept out of line so the common path stays short.
__device__ __noinline__ void cross_prime_early(const WheelTables &t, uint32_t *seg32, uint32_t p, uint32_t pq,
                                               uint32_t pc, uint32_t R, int64_t B0, uint32_t L) {
    for (int j = 0; j < 8; ++j) {
        const uint32_t off = class_off(t, p, pq, pc, j, R, B0, true, L);
        const uint32_t bit = t.bit[pc * 8 + j];
        for (uint32_t o = off; o < L; o += p) clear_bit(seg32, o, bit);
    }
}

// True when the segment starting at wheel byte B0 (Bc = max(B0, 0)) may begin
// before some progression's first allowed multiple p m, m >= p: those bytes are
// all below p^2 / 30 + 2 p, so 30 Bc >= p^2 + 60 p rules it out.
__device__ __forceinline__ bool is_early(int64_t B0, uint64_t Bc, uint32_t p) {
    return B0 < 0 || 30ull * Bc < (uint64_t)p * p + 60ull * p;
}

// Inverse of an odd p modulo 128 (Newton steps: p is its own inverse mod 8).
__device__ __forceinline__ uint32_t inv_mod128(uint32_t p) {
    uint32_t x = p;
    x *= 2u - p * x;  // mod 64
    x *= 2u - p * x;  // mod 4096
    return x & 127u;
}

// Bits of wheel word w (4 bytes at integers base .. base + 119, base relative
// to 30 B0) that lie in [lo_rel, hi_rel).
__device__ uint32_t range_mask(int64_t base, int64_t lo_rel, int64_t hi_rel) {
    uint32_t m = 0;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 8; ++k) {
            int64_t n = base + 30 * i + c_res[k];
            if (n >= lo_rel && n < hi_rel) m |= 1u << (8 * i + k);
        }
    return m;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Number of base primes among primes[0, n) with p^2 < E (a prefix, since the
// primes ascend), found by one warp with 32-way probing.  Every lane of the
// warp must call it; all lanes return the result.
__device__ uint32_t primes_with_square_below(const uint32_t *primes, uint32_t n, uint64_t E, int lane) {
    uint32_t a = 0, b = n;  // the answer lies in [a, b]
    while (b - a > 32) {
        const uint32_t step = (b - a + 31) / 32, idx = a + (uint32_t)lane * step;
        bool ok = false;
        if (idx < b) {
            const uint64_t q = __ldg(primes + idx);
            ok = q * q < E;
        }
        const int c = __popc(__ballot_sync(0xffffffffu, ok));
        if (c == 0) return a;
        const uint32_t na = a + (uint32_t)(c - 1) * step + 1, nb = a + (uint32_t)c * step;
        a = na;
        b = nb < b ? nb : b;
    }
    bool ok = false;
    if (a + lane < b) {
        const uint64_t q = __ldg(primes + a + lane);
        ok = q * q < E;
    }
    return a + __popc(__ballot_sync(0xffffffffu, ok));
}

// Wheel cursor of a prime p: its multiples p m with m coprime to 30 in
// increasing order.  In wheel bytes they are p a + c_k for a = 0, 1, ... and
// k = 0..7, with c_k = floor(p r_k / 30) ascending in k, so stepping k -> k + 1
// (and a -> a + 1 after k = 7) walks them in order.  wheel_start() returns the
// first one at or after wheel byte B0 that also has m >= p (crossing starts at
// p^2), as a byte offset from B0 (int64) and its class k.
struct WheelCursor {
    int64_t off;
    uint32_t k;
};

__device__ __forceinline__ WheelCursor wheel_start(const WheelTables &t, uint32_t p, uint64_t M, uint32_t pq,
                                                       uint32_t pc, int64_t B0) {
    const uint64_t Bc = B0 > 0 ? (uint64_t)B0 : 0;
    uint64_t Q = __umul64hi(Bc, M);
    uint32_t R = (uint32_t)(Bc - Q * p);
    if (R >= p) {
        R -= p;
        ++Q;
    }
    const uint64_t adj = t.adj40[pc];
    // first class with c_k >= R: c_j = floor(p r_j / 30) < R iff p r_j < 30 R, i.e.
    // r_j <= v = floor((30 R - 1) / p) < 30, so k = #{ j : r_j <= v }, read from
    // nibble v of a packed table (0x...6554 holds v = 16..29)
    uint32_t k = 0;
    if (R) {
        const uint64_t x = 30ull * R - 1;
        uint64_t v = __umul64hi(x, M);
        if (x - v * p >= p) ++v;
        k = (uint32_t)(((v < 16 ? 0x4443322221111110ull : 0x87777776666554ull) >> (4 * (v & 15))) & 15u);
    }
    uint64_t a = Q;
    if (k == 8) {
        k = 0;
        ++a;
    }
    if (a < pq || (a == pq && k < pc)) {  // not before m = p: (a, k) >= (pq, class of p)
        a = pq;
        k = pc;
    }
    const uint32_t c_k = pq * (uint32_t)((kRes40 >> (5 * k)) & 31u) + (uint32_t)((adj >> (5 * k)) & 31u);
    WheelCursor w;
    w.off = (int64_t)((uint64_t)p * a + c_k) - B0;
    w.k = k;
    return w;
}


// Byte distance from multiple (a, k) to the next one: pq gap_k + dadj_k.
__device__ __forceinline__ uint32_t wheel_step(uint32_t pq, uint32_t dadj, uint32_t k) {
    return pq * ((kWheelGaps >> (4 * k)) & 15u) + ((dadj >> (3 * k)) & 7u);
}

__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Bulk (TMA) copy of the pattern tile into shared memory, completed on an
// mbarrier: one thread arms the barrier with the byte count and issues one
// cp.async.bulk global -> shared; every thread waits on the barrier's phase.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Orders this thread's earlier shared-memory accesses (and, after a barrier,
// the block's) before its later async-proxy operations on shared memory.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Polls before a wait is declared failed (each try_wait may itself suspend the
// thread for a while): far beyond any copy of a few hundred KB from L2.
constexpr uint32_t kWaitLimit = 1u << 24;

// Self-test of the bounded wait: one CTA initialises an mbarrier, copies `bytes`
// from `src` into shared memory with the bulk copy when `arm` is set (else
// nothing will ever complete the phase), and every thread waits with the given
// limit.  *status = 0 when the phase completed, 1 when the limit was hit.
__global__ void k_wait_selftest(const uint4 *src, uint32_t bytes, int arm, uint32_t limit, int *status) {
    extern __shared__ uint4 buf[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t failed;
    if (threadIdx.x == 0) {
        failed = 0;
        mbar_init(&bar, 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
    if (threadIdx.x == 0 && arm) bulk_copy_g2s(buf, src, bytes, &bar);
    uint32_t tries = 0;
    while (!mbar_try_wait(&bar, 0) && ++tries < limit) {
    }
    if (tries >= limit) failed = 1;
    __syncthreads();
    if (threadIdx.x == 0) *status = failed ? 1 : 0;
}

// Medium primes [base, base + 32) below mid_end, lane l taking base + l, over
// the L bytes (a multiple of 32) at wheel byte B0 held at seg32: each of a
// prime's eight progressions (stride p bytes) is split into four
// sub-progressions of stride 4 p bytes = p words, one per byte phase, each
// crossed with one fixed mask.  The warp re-converges after every sub-loop.
__device__ __forceinline__ void cross_medium_group(const WheelTables &tab, const uint32_t *__restrict__ primes,
                                                   const uint64_t *__restrict__ magic, uint32_t *seg32,
                                                   uint32_t base, uint32_t mid_end, int lane, int64_t B0,
                                                   uint32_t L) {
    const uint64_t Bc = B0 > 0 ? (uint64_t)B0 : 0;
    const uint32_t i = base + lane;
    const bool valid = i < mid_end;
    const uint32_t p = valid ? __ldg(primes + i) : 1u;
    const uint64_t M = valid ? __ldg(magic + i) : ~0ull;
    const uint32_t R = mod_barrett(Bc, p, M);
    const uint32_t pq = p / 30, pc = valid ? tab.cls[p - pq * 30] : 0u;
    const bool early = valid && is_early(B0, Bc, p);
    if (early) cross_prime_early(tab, seg32, p, pq, pc, R, B0, L);
    __syncwarp();
    const uint32_t lw = (valid && !early) ? L >> 2 : 0u;  // fast path only for the others
    const uint32_t bits = tab.bits24[pc];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t off = class_off(tab, p, pq, pc, j, R, B0, false, L);
        const uint32_t bit = (bits >> (3 * j)) & 7u;
#pragma unroll
        for (uint32_t ph = 0; ph < 4; ++ph) {
            // p^-1 = p (mod 4), so off + k p = ph (mod 4) for k = (ph - off) p mod 4
            const uint32_t o = off + (((ph - off) * p) & 3u) * p;
            const uint32_t mask = ~(1u << (8u * ph + bit));
            for (uint32_t w = o >> 2; w < lw; w += p) atomicAnd(&seg32[w], mask);
        }
        __syncwarp();
    }
}

// Medium groups whose estimated costs are kept in shared memory for dealing
// them over the warps; the cost of a group is kMidSetup plus the hits of its
// smallest prime in a full segment, 8 S / p.
constexpr uint32_t kMidGroups = 256;
constexpr uint32_t kMidSetup = 224;

template <int MODE>
__global__ void __launch_bounds__(1024, 1) k_sieve(const SieveLaunch *__restrict__ Pg) {
    extern __shared__ uint4 smem4[];
    __shared__ SieveLaunch P;  // launch parameters, read from device memory (graph-replayable)
    if (threadIdx.x == 0) P = *Pg;
    uint8_t *seg = reinterpret_cast<uint8_t *>(smem4);
    uint32_t *seg32 = reinterpret_cast<uint32_t *>(smem4);
    __shared__ WheelTables tab;
    __shared__ unsigned long long s_item;
    __shared__ uint32_t s_range;
    __shared__ uint32_t s_small_next;
    __shared__ unsigned long long s_red[32];
    __shared__ uint32_t s_R[kSmallResidues];      // B0 mod p for the first small primes
    __shared__ uint32_t s_nseg;                     // base primes with p^2 below the segment end
    __shared__ uint32_t s_nbucket;                  // bucket primes with p^2 below the chunk end
    __shared__ uint32_t s_cnt[kMaxChunkSegments];  // bucket fill counts, one per segment of the chunk
    __shared__ __align__(8) uint64_t s_tile_bar;    // completes the pattern copy of each segment
    __shared__ uint32_t s_tile_fail;                // a wait for it hit kWaitLimit: the CTA stops
    __shared__ uint32_t s_xph[4];                   // B0 mod the periods of the further patterns
    __shared__ uint32_t s_midG;                     // medium groups dealt by cost (0: round-robin)
    __shared__ uint32_t s_midW[kMidGroups + 1];     // their cumulative costs
    uint32_t tile_phase = 0;
    if (threadIdx.x == 0) {
        s_tile_fail = 0;
        mbar_init(&s_tile_bar, 1);
        fence_proxy_async_smem();
    }

    init_tables(tab);
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t C = P.chunk_segs;
    if (tid < 32) {  // cumulative costs of the medium groups (read after the next barrier)
        const uint32_t ng = P.mid_end > P.small_end ? (P.mid_end - P.small_end + 31) / 32 : 0;
        const uint32_t G = ng <= kMidGroups ? ng : 0;
        uint32_t run = 0;
        for (uint32_t g0 = 0; g0 < G; g0 += 32) {
            const uint32_t g = g0 + lane;
            const uint32_t c =
                g < G ? kMidSetup + 8u * P.seg_bytes / __ldg(P.primes + P.small_end + 32u * g) : 0u;
            const uint32_t incl = warp_inclusive_scan(c, lane);
            if (g < G) s_midW[g + 1] = run + incl;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            s_midW[0] = 0;
            s_midG = G;
        }
    }
    uint32_t *const bucket_base = P.buckets ? P.buckets + (size_t)blockIdx.x * C * P.bucket_cap : nullptr;

    for (;;) {
        if (tid == 0) {
            unsigned long long item = atomicAdd(P.item_counter, 1ull);
            s_item = item;
            if (item < P.n_items) {
                uint32_t a = 0, b = P.n_ranges - 1;  // largest r with item_first <= item
                while (a < b) {
                    uint32_t mid = (a + b + 1) >> 1;
                    if (P.ranges[mid].item_first <= item) a = mid; else b = mid - 1;
                }
                s_range = a;
            }
        }
        if (tid < (int)C) s_cnt[tid] = 0;
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= P.n_items) break;
        const RangeDesc &rd = P.ranges[s_range];
        const uint32_t range_id = s_range;
        const uint32_t S = rd.seg_bytes;  // this range's segment size (<= P.seg_bytes)
        // this item: segments [s0, s0 + nchunk) of the range
        const uint64_t s0 = (item - rd.item_first) * C;
        const uint32_t nchunk = (uint32_t)(rd.nseg - s0 < C ? rd.nseg - s0 : C);
        const int64_t Bs = rd.Bbase + (int64_t)(s0 * S);
        const uint32_t n_range = rd.n_use;
        uint32_t chunk_bytes;
        {
            int64_t need = ((int64_t)rd.hi - 30 * Bs + 29) / 30;
            need = (need + 31) & ~(int64_t)31;
            const int64_t full = (int64_t)nchunk * S;
            chunk_bytes = (uint32_t)(need < full ? need : full);
        }

        // 0. bucket fill: every bucket prime with a multiple in this chunk
        //    appends its hits to the chunk's per-segment lists (in HBM)
        const bool use_buckets = rd.bucket_first < n_range;
        if (use_buckets) {
            if (tid < 32) {
                const uint64_t E = (uint64_t)(30 * (Bs + (int64_t)chunk_bytes));
                const uint64_t Eh = E < rd.hi ? E : rd.hi;
                const uint32_t n = primes_with_square_below(P.primes, n_range, Eh, lane);
                if (lane == 0) s_nbucket = n;
            }
            __syncthreads();
            // one lane per bucket prime, 32 primes per warp: for each segment of
            // the chunk the warp counts its lanes' hits, reserves room with one
            // shared-memory atomic, and each lane writes its hits contiguously
            const uint32_t nb = s_nbucket;
            for (uint32_t base = rd.bucket_first + (tid & ~31u); base < nb; base += blockDim.x) {
                const uint32_t i = base + lane;
                const bool valid = i < nb;
                const uint32_t p = valid ? __ldg(P.primes + i) : 1u;
                const uint64_t M = valid ? __ldg(P.magic + i) : ~0ull;
                const uint32_t pq = p / 30, pc = valid ? tab.cls[p - pq * 30] : 0u;
                WheelCursor wc = wheel_start(tab, p, M, pq, pc, Bs);
                uint32_t off = (valid && wc.off < (int64_t)chunk_bytes) ? (uint32_t)wc.off : chunk_bytes;
                uint32_t k = wc.k;
                const uint32_t bits = tab.bits24[pc], dadj = tab.dadj24[pc];
                for (uint32_t g = 0; g < nchunk; ++g) {
                    const uint32_t seg_lo = g * S, seg_end = seg_lo + S < chunk_bytes ? seg_lo + S : chunk_bytes;
                    uint32_t h = 0;
                    for (uint32_t o = off, kk = k; o < seg_end; o += wheel_step(pq, dadj, kk), kk = (kk + 1) & 7u) ++h;
                    __syncwarp();
                    const uint32_t incl = warp_inclusive_scan(h, lane);
                    uint32_t first = 0;
                    if (lane == 31 && incl) first = atomicAdd(s_cnt + g, incl);
                    first = __shfl_sync(0xffffffffu, first, 31) + incl - h;
                    uint32_t *list = bucket_base + (size_t)g * P.bucket_cap;
                    for (; off < seg_end; off += wheel_step(pq, dadj, k), k = (k + 1) & 7u, ++first) {
                        const uint32_t wo = off - seg_lo;
                        const uint32_t bit = (bits >> (3 * k)) & 7u;
                        if (first < P.bucket_cap)
                            list[first] = (wo >> 2) | ((((wo & 3u) << 3) | bit) << 16);
                        else
                            atomicOr(P.overflow, 1u);
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
        }

        // per-CTA wheel cursors of the large primes, carried from segment to
        // segment of this chunk; valid for primes [mid_end, n_prev)
        uint32_t *const cursors = P.cursors ? P.cursors + (size_t)blockIdx.x * P.cursor_stride : nullptr;
        uint32_t n_prev = 0;
        for (uint32_t g = 0; g < nchunk; ++g) {
            const uint64_t s = s0 + g;
            const int64_t B0 = Bs + (int64_t)g * S;
            const uint64_t Bc = B0 > 0 ? (uint64_t)B0 : 0;
            const int64_t base_int = 30 * B0;  // integer of bit 0 of byte 0
            const int64_t hi_rel = (int64_t)rd.hi - base_int, lo_rel = (int64_t)rd.lo - base_int;
            const uint32_t L = chunk_bytes - g * S < S ? chunk_bytes - g * S : S;

            // 1. pre-sieved pattern -> shared memory: one bulk (TMA) copy of the
            //    16-byte aligned shifted tile, overlapped with the prime-bound
            //    search below and waited for before the crossing starts
            {
                int64_t ph = B0 % (int64_t)kTilePeriod;
                if (ph < 0) ph += kTilePeriod;
                const uint32_t k = (uint32_t)ph & 15u;
                const uint4 *src = reinterpret_cast<const uint4 *>(P.tile + k * P.tile_stride + ((uint32_t)ph - k));
                // the previous segment's accesses are ordered before the copy by
                // the barrier that ended it and this fence
                if (tid == 0) {
                    fence_proxy_async_smem();
                    bulk_copy_g2s(smem4, src, L, &s_tile_bar);
                    if (P.xtile0) {
                        const int64_t x0 = B0 % (int64_t)kXTilePeriod0, x1 = B0 % (int64_t)kXTilePeriod1,
                                      x2 = B0 % (int64_t)kXTilePeriod2;
                        s_xph[0] = (uint32_t)(x0 < 0 ? x0 + kXTilePeriod0 : x0);
                        s_xph[1] = (uint32_t)(x1 < 0 ? x1 + kXTilePeriod1 : x1);
                        s_xph[2] = (uint32_t)(x2 < 0 ? x2 + kXTilePeriod2 : x2);
                        const int64_t x3 = B0 % (int64_t)kXTilePeriod3;
                        s_xph[3] = (uint32_t)(x3 < 0 ? x3 + kXTilePeriod3 : x3);
                    }
                }
            }
            // primes with p^2 >= the segment's end have no multiple to cross here
            if (tid < 32) {
                const int64_t seg_end = base_int + 30 * (int64_t)L;
                const uint64_t E = (uint64_t)(seg_end < (int64_t)rd.hi ? seg_end : (int64_t)rd.hi);
                const uint32_t n = primes_with_square_below(P.primes, n_range, E, lane);
                if (lane == 0) {
                    s_nseg = n;
                    s_small_next = 0;
                }
            }
            const uint32_t small_first = P.small_first;
            {
                const uint32_t se = P.small_end < n_range ? P.small_end : n_range;
                const uint32_t nr = se > small_first ? se - small_first : 0;
                for (uint32_t t = tid; t < nr && t < kSmallResidues; t += blockDim.x)
                    s_R[t] = mod_barrett(Bc, __ldg(P.primes + small_first + t), __ldg(P.magic + small_first + t));
            }
            {
                uint32_t tries = 0;
                while (!mbar_try_wait(&s_tile_bar, tile_phase) && ++tries < kWaitLimit) {
                }
                if (tries >= kWaitLimit) s_tile_fail = 1;
                tile_phase ^= 1u;
            }
            __syncthreads();
            // Every thread sees a failed wait after the barrier, and the CTA stops.  Its bulk
            // copy may then still be outstanding: the CTA exits without waiting for it (a
            // wait that already ran out for 2^24 polls would not end), which is only sound
            // because the copy is taken never to complete.  The host turns the flag into
            // SIEVE_EDEVICE and trusts no output of this launch; the condition has never
            // been seen in normal runs.
            if (s_tile_fail) break;
            // 1'. the further patterns (primes 23..59), ANDed in 16 bytes at a time
            //     from their L2-resident shifted copies.  In count mode the AND is
            //     fused into the popcount epilogue instead (step 4), which reads every
            //     word anyway -- except in the segment holding wheel bytes 0 and 1,
            //     whose fix-up (step 3) must come after the patterns.
            const bool fuse_x = MODE == kModeCount && P.xtile0 && !(B0 <= 2 && B0 + (int64_t)L > 0);
            if (P.xtile0 && !fuse_x) {
                const uint4 *x0 = reinterpret_cast<const uint4 *>(P.xtile0 + (s_xph[0] & 15u) * kXTileStride0 +
                                                                  (s_xph[0] & ~15u));
                const uint4 *x1 = reinterpret_cast<const uint4 *>(P.xtile1 + (s_xph[1] & 15u) * kXTileStride1 +
                                                                  (s_xph[1] & ~15u));
                const uint4 *x2 = reinterpret_cast<const uint4 *>(P.xtile2 + (s_xph[2] & 15u) * kXTileStride2 +
                                                                  (s_xph[2] & ~15u));
                const uint4 *x3 = P.xtile3 ? reinterpret_cast<const uint4 *>(P.xtile3 + (s_xph[3] & 15u) * kXTileStride3 +
                                                                             (s_xph[3] & ~15u))
                                           : nullptr;
                for (uint32_t q = tid; q < L / 16; q += blockDim.x) {
                    const uint4 a = __ldg(x0 + q), b = __ldg(x1 + q), c = __ldg(x2 + q);
                    uint4 v = smem4[q];
                    v.x &= a.x & b.x & c.x;
                    v.y &= a.y & b.y & c.y;
                    v.z &= a.z & b.z & c.z;
                    v.w &= a.w & b.w & c.w;
                    if (x3) {
                        const uint4 d = __ldg(x3 + q);
                        v.x &= d.x;
                        v.y &= d.y;
                        v.z &= d.z;
                        v.w &= d.w;
                    }
                    smem4[q] = v;
                }
                __syncthreads();
            }
            // a range on the Miller-Rabin path is sieved with the primes below 2^16 only
            const uint32_t n_seg = rd.mr && P.mr_end < s_nseg ? P.mr_end : s_nseg;
            // primes crossed here (not through the buckets): [8, n_use)
            const uint32_t n_use = use_buckets && rd.bucket_first < n_seg ? rd.bucket_first : n_seg;
            const uint32_t small_end = P.small_end < n_use ? P.small_end : n_use;
            const uint32_t n_small8 = (small_end > small_first ? small_end - small_first : 0) * 8;

            // 2a. medium primes [small_end, mid_end), 32 consecutive primes (a group)
            //     at a time.  The groups are dealt by estimated cost: warp w takes the
            //     w-th 1/32 of the cumulative cost, so a heavy group (small primes,
            //     many hits) is shared by several warps, each crossing it over its
            //     own part of the segment.
            const uint32_t mid_end = rd.mid_end < n_use ? rd.mid_end : n_use;
            const uint32_t Lw = L >> 2;
            {
                // G > 0: warp w takes the cost interval [x0, x1); G = 0 (too many
                // groups for the table): warp w takes groups w, w + 32, ... whole.
                // The cost is dealt over the groups this segment has (those below
                // mid_end, which this range's tier limit or p^2 may put before the
                // table's end), so no warp is dealt groups that are not crossed here.
                const uint32_t Gs = mid_end > P.small_end ? (mid_end - P.small_end + 31) / 32 : 0;
                const uint32_t G = s_midG < Gs ? s_midG : Gs, warp = tid >> 5, nwarps = blockDim.x >> 5;
                const uint32_t T = s_midW[G];
                const uint32_t x0 = (uint32_t)((uint64_t)T * warp / nwarps);
                const uint32_t x1 = (uint32_t)((uint64_t)T * (warp + 1) / nwarps);
                uint32_t g = warp;
                if (G) {
                    uint32_t hi = G - 1;  // the last group with W[g] <= x0
                    g = 0;
                    while (g < hi) {
                        const uint32_t mid = (g + hi + 1) >> 1;
                        if (s_midW[mid] <= x0) g = mid; else hi = mid - 1;
                    }
                }
                for (;; g += G ? 1u : nwarps) {
                    const uint32_t base = P.small_end + 32u * g;
                    if (base >= mid_end || (G && (g >= G || s_midW[g] >= x1))) break;
                    uint32_t a = 0, b = L;
                    if (G) {
                        // part [a, b) of the segment, cut at 32-byte boundaries that
                        // the neighbouring warp computes the same way
                        const uint32_t w0 = s_midW[g], wg = s_midW[g + 1] - w0;
                        const uint32_t u0 = (x0 > w0 ? x0 : w0) - w0, u1 = (x1 < w0 + wg ? x1 : w0 + wg) - w0;
                        a = (uint32_t)(((uint64_t)u0 * L / wg) & ~31ull);
                        b = (uint32_t)(((uint64_t)u1 * L / wg) & ~31ull);
                    }
                    if (a < b) cross_medium_group(tab, P.primes, P.magic, seg32 + a / 4, base, mid_end, lane, B0 + a, b - a);
                }
            }
            // 2a'. large primes below the bucket limit [mid_end, n_use): one lane
            //      per prime, walking its multiples in the segment with the wheel
            //      cursor (only the hits are visited, not all eight classes).  With
            //      per-CTA cursors the walk resumes where the previous segment of
            //      this chunk left it, so only primes new to the chunk pay for the
            //      start computation (Barrett reduction and wheel class).
            // Each lane takes kLargeUnroll primes per pass and issues all their
            // loads first: the loop is bound by load latency, not by arithmetic.
            for (uint32_t base = mid_end + (tid & ~31u) * kLargeUnroll; base < n_use;
                 base += blockDim.x * kLargeUnroll) {
                uint32_t pv[kLargeUnroll], sv[kLargeUnroll];
                uint64_t mv[kLargeUnroll];
#pragma unroll
                for (int u = 0; u < (int)kLargeUnroll; ++u) {
                    const uint32_t i = base + lane + 32u * u;
                    const bool valid = i < n_use;
                    pv[u] = valid ? __ldg(P.primes + i) : 1u;
                    const bool resume = valid && cursors && i < n_prev;
                    sv[u] = resume ? cursors[i - mid_end] : 0u;
                    mv[u] = (valid && !resume) ? __ldg(P.magic + i) : ~0ull;
                }
#pragma unroll
                for (int u = 0; u < (int)kLargeUnroll; ++u) {
                    const uint32_t i = base + lane + 32u * u;
                    const bool valid = i < n_use;
                    const uint32_t p = pv[u];
                    const uint32_t pq = p / 30, pc = valid ? tab.cls[p - pq * 30] : 0u;
                    uint32_t off, k;
                    if (valid && cursors && i < n_prev) {  // (offset from this segment's start) | class << 29
                        off = sv[u] & 0x1fffffffu;
                        k = sv[u] >> 29;
                    } else {
                        const WheelCursor wc = wheel_start(tab, p, mv[u], pq, pc, B0);
                        off = (valid && wc.off < (int64_t)0x7fffffff) ? (uint32_t)wc.off : 0x7fffffffu;
                        k = wc.k;
                    }
                    const uint32_t bits = tab.bits24[pc], dadj = tab.dadj24[pc];
                    const uint32_t l = valid ? L : 0u;
                    for (; off < l; off += wheel_step(pq, dadj, k), k = (k + 1) & 7u)
                        clear_bit(seg32, off, (bits >> (3 * k)) & 7u);
                    if (cursors && valid) cursors[i - mid_end] = (off - L) | (k << 29);
                }
                __syncwarp();
            }
            // 2c. drain this segment's bucket list
            if (use_buckets) {
                const uint32_t n = s_cnt[g] < P.bucket_cap ? s_cnt[g] : P.bucket_cap;
                const uint32_t *list = bucket_base + (size_t)g * P.bucket_cap;
                for (uint32_t e = tid; e < n; e += blockDim.x) {
                    const uint32_t v = list[e];
                    atomicAnd(&seg32[v & 0xffffu], ~(1u << (v >> 16)));
                }
            }
            // 2b. small primes [small_first, small_end): one (prime, class) progression per
            //     warp, taken dynamically in decreasing order of work.  The
            //     progression (stride p bytes) is split into 128 sub-progressions
            //     of stride 128 p: lane l takes the four whose bytes are 4 l + q
            //     (mod 128), q = 0..3.  Every lane then always writes bank l of
            //     the segment with one fixed bit mask, so a warp's 32 atomics
            //     never share a bank and need no per-hit mask arithmetic.
            for (;;) {
                uint32_t k = 0;
                if (lane == 0) k = atomicAdd(&s_small_next, 1u);
                k = __shfl_sync(0xffffffffu, k, 0);
                if (k >= n_small8) break;
                const uint32_t i = small_first + (k >> 3);
                const int j = (int)(k & 7);
                const uint32_t p = __ldg(P.primes + i);
                const uint32_t t = i - small_first;
                const uint32_t R = t < kSmallResidues ? s_R[t] : mod_barrett(Bc, p, __ldg(P.magic + i));
                const uint32_t pq = p / 30, pc = tab.cls[p - pq * 30];
                const uint32_t off = class_off(tab, p, pq, pc, j, R, B0, is_early(B0, Bc, p), L);
                if (off >= L) continue;
                const uint32_t bit = tab.bit[pc * 8 + j];
                const uint32_t pinv = inv_mod128(p);
                const uint32_t wstep = 32u * p;  // 128 p bytes = 32 p words
#pragma unroll
                for (uint32_t q = 0; q < 4; ++q) {
                    const uint32_t kappa = ((4u * (uint32_t)lane + q - off) * pinv) & 127u;
                    const uint32_t o = off + kappa * p;  // = 4 lane + q (mod 128)
                    const uint32_t mask = ~(1u << (8u * q + bit));
                    uint32_t w = o >> 2;
                    for (; w + 3u * wstep < Lw; w += 4u * wstep) {
                        atomicAnd(&seg32[w], mask);
                        atomicAnd(&seg32[w + wstep], mask);
                        atomicAnd(&seg32[w + 2u * wstep], mask);
                        atomicAnd(&seg32[w + 3u * wstep], mask);
                    }
                    for (; w < Lw; w += wstep) atomicAnd(&seg32[w], mask);
                }
            }
            __syncthreads();

            // 3. wheel bytes 0 and 1 (integers 1..59): 1 and 49 are not prime, the
            //    others are, though the patterns clear 7..19 and 23..59
            if (B0 <= 2 && B0 + (int64_t)L > 0) {  // the same for the whole CTA
                if (tid == 0) {
                    if (B0 <= 0) seg[-B0] = 0xFE;
                    if (B0 <= 1 && 1 - B0 < (int64_t)L) seg[1 - B0] = 0xDF;
                    // wheel byte 2 (61..89): 77 is the one composite; the fourth pattern clears 61, 67, 71
                    if (P.xtile3 && 2 - B0 < (int64_t)L) seg[2 - B0] = 0xEF;
                }
                __syncthreads();
            }

            unsigned long long cnt = 0;
            if (MODE == kModeCount) {
                // 4. popcount of the bits in [lo, hi); a range on the Miller-Rabin
                //    path also leaves its raw wheel words for k_mr_filter
                uint32_t *const raw = rd.mr ? rd.bitmap : nullptr;
                const uint4 *x0 = nullptr, *x1 = nullptr, *x2 = nullptr;
                if (fuse_x) {  // the further patterns' words for this segment (step 1')
                    x0 = reinterpret_cast<const uint4 *>(P.xtile0 + (s_xph[0] & 15u) * kXTileStride0 +
                                                         (s_xph[0] & ~15u));
                    x1 = reinterpret_cast<const uint4 *>(P.xtile1 + (s_xph[1] & 15u) * kXTileStride1 +
                                                         (s_xph[1] & ~15u));
                    x2 = reinterpret_cast<const uint4 *>(P.xtile2 + (s_xph[2] & 15u) * kXTileStride2 +
                                                         (s_xph[2] & ~15u));
                }
                if (!raw && lo_rel <= 0 && hi_rel >= 30 * (int64_t)L) {
                    // the whole segment lies in [lo, hi): no masks, 16-byte loads
                    if (fuse_x && P.xtile3) {
                        const uint4 *x3 = reinterpret_cast<const uint4 *>(P.xtile3 + (s_xph[3] & 15u) * kXTileStride3 +
                                                                          (s_xph[3] & ~15u));
                        for (uint32_t q = tid; q < L / 16; q += blockDim.x) {
                            const uint4 a = __ldg(x0 + q), b = __ldg(x1 + q), c = __ldg(x2 + q), d = __ldg(x3 + q);
                            const uint4 v = smem4[q];
                            cnt += __popc(v.x & a.x & b.x & c.x & d.x) + __popc(v.y & a.y & b.y & c.y & d.y) +
                                   __popc(v.z & a.z & b.z & c.z & d.z) + __popc(v.w & a.w & b.w & c.w & d.w);
                        }
                    } else if (fuse_x) {
                        for (uint32_t q = tid; q < L / 16; q += blockDim.x) {
                            const uint4 a = __ldg(x0 + q), b = __ldg(x1 + q), c = __ldg(x2 + q);
                            const uint4 v = smem4[q];
                            cnt += __popc(v.x & a.x & b.x & c.x) + __popc(v.y & a.y & b.y & c.y) +
                                   __popc(v.z & a.z & b.z & c.z) + __popc(v.w & a.w & b.w & c.w);
                        }
                    } else {
                        for (uint32_t q = tid; q < L / 16; q += blockDim.x) {
                            const uint4 v = smem4[q];
                            cnt += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
                        }
                    }
                } else {
                    const uint32_t *y0 = reinterpret_cast<const uint32_t *>(x0),
                                   *y1 = reinterpret_cast<const uint32_t *>(x1),
                                   *y2 = reinterpret_cast<const uint32_t *>(x2);
                    const uint32_t *y3 = fuse_x && P.xtile3
                                             ? reinterpret_cast<const uint32_t *>(P.xtile3 + (s_xph[3] & 15u) * kXTileStride3 +
                                                                                  (s_xph[3] & ~15u))
                                             : nullptr;
                    for (uint32_t w = tid; w < L / 4; w += blockDim.x) {
                        uint32_t v = seg32[w];
                        if (fuse_x) v &= __ldg(y0 + w) & __ldg(y1 + w) & __ldg(y2 + w);
                        if (y3) v &= __ldg(y3 + w);
                        if (raw) raw[w] = v;
                        const int64_t wb = 120 * (int64_t)w;
                        if (wb < lo_rel || wb + 120 > hi_rel) v &= range_mask(wb, lo_rel, hi_rel);
                        cnt += __popc(v);
                    }
                }
            } else {
                // 4'. each group of 32 wheel bytes (960 integers) is 15 words of the
                //     odd-only bitmap: bits [32 q, 32 q + 32) of the group's 480 odd
                //     positions, i.e. of the 15-bit expansions of its bytes
                //     floor(32 q / 15) .. + 3, shifted by 32 q mod 15.  One thread per
                //     output word, so a warp stores 32 consecutive words.
                const uint64_t nwords = rd.bitmap_words;
                const uint64_t o0 = rd.lo | 1;
                const uint64_t nbits = o0 < rd.hi ? (rd.hi - o0 + 1) / 2 : 0;
                uint32_t *out = rd.bitmap;
                const int64_t wbase = (base_int + 1 - (int64_t)o0) / 64;  // exact: the grid keeps n0 = o0 (mod 64)
                const uint32_t nout = (L / 32) * 15;
                for (uint32_t k = tid; k < nout; k += blockDim.x) {
                    const int64_t wq = wbase + k;
                    if (wq < 0 || wq >= (int64_t)nwords) continue;
                    const uint32_t gr = k / 15, q = k - 15 * gr;
                    const uint32_t b0 = 32 * gr + (32 * q) / 15, sh = (32 * q) % 15;
                    uint64_t e = (uint64_t)tab.expand[seg[b0]] | (uint64_t)tab.expand[seg[b0 + 1]] << 15 |
                                 (uint64_t)tab.expand[seg[b0 + 2]] << 30;
                    // sh = 14 (q = 7 only) reaches bit 45: bit 0 of byte b0 + 3 = 17 of the group
                    if (sh == 14) e |= (uint64_t)tab.expand[seg[b0 + 3]] << 45;
                    uint32_t v = (uint32_t)(e >> sh);
                    // 3 and 5 are prime but have no wheel bit
                    const int64_t n0 = base_int + 960 * (int64_t)gr + 1;  // first odd integer of the group
                    if (n0 <= 5 && n0 + 958 >= 3) {
#pragma unroll
                        for (int sp = 3; sp <= 5; sp += 2) {
                            const int64_t i = (sp - n0) / 2;  // odd position in the group
                            if (sp >= n0 && (i >> 5) == (int64_t)q) v |= 1u << (i & 31);
                        }
                    }
                    if (wq == (int64_t)nwords - 1 && (nbits & 31)) v &= (1u << (nbits & 31)) - 1u;
                    if (out) out[wq] = v;
                    cnt += __popc(v);
                }
            }
            cnt = warp_sum(cnt);
            if (lane == 0) s_red[tid >> 5] = cnt;
            __syncthreads();
            if (tid < 32) {
                unsigned long long v = tid < (int)(blockDim.x >> 5) ? s_red[tid] : 0ull;
                v = warp_sum(v);
                if (tid == 0) {
                    if (s == 0) v += rd.corr;
                    atomicAdd(P.counts + range_id, v);
                }
            }
            n_prev = n_use;
            __syncthreads();
        }
        if (s_tile_fail) {  // reported to the host as a device error; the CTA stops here
            if (tid == 0) atomicOr(P.overflow, 2u);
            break;
        }
    }
}

// ---------------------------------------------------------------- pattern tile

// Copy k (k = blockIdx.y) holds pattern bytes (i + k) mod period at offset i.
// Pattern byte b, bit j: 1 iff 30 b + r_j has no prime factor among the np
// primes of ps, whose product is the period.
struct TilePrimes {
    uint32_t p[5];
};

__global__ void k_build_tile(uint8_t *tile, uint64_t stride, uint32_t len, uint32_t period, TilePrimes ps, int np) {
    const uint32_t k = blockIdx.y;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        const uint32_t b = (uint32_t)(((uint64_t)i + k) % period);
        uint32_t v = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint64_t n = 30ull * b + c_res[j];
            bool keep = true;
            for (int t = 0; t < np; ++t) keep = keep && n % ps.p[t] != 0;
            if (keep) v |= 1u << j;
        }
        tile[k * stride + i] = (uint8_t)v;
    }
}

// Primes below 256 by trial division, ascending, one block of 256 threads.
__global__ void k_tiny_primes(uint32_t *out, uint32_t *n_out) {
    __shared__ uint32_t warp_cnt[8];
    const uint32_t n = threadIdx.x;
    bool prime = n >= 2;
    for (uint32_t d = 2; d * d <= n; ++d)
        if (n % d == 0) prime = false;
    const uint32_t ballot = __ballot_sync(0xffffffffu, prime);
    const int lane = n & 31, warp = n >> 5;
    if (lane == 0) warp_cnt[warp] = __popc(ballot);
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < warp; ++w) base += warp_cnt[w];
    if (prime) out[base + __popc(ballot & ((1u << lane) - 1u))] = n;
    if (n == 255) *n_out = base + __popc(ballot);
}

__global__ void k_magic(const uint32_t *primes, uint64_t *magic, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        magic[i] = ~0ull / primes[i];
}

// ---------------------------------------------------------------- compaction

template <typename T>
__global__ void k_put_two(T *out, T two) { out[0] = two; }

__global__ void k_finalize_count(const unsigned long long *count, const unsigned *overflow, uint64_t *out) {
    *out = *overflow ? ~0ull : *count;
}

}  // namespace

cudaError_t set_sieve_smem_limits() {
    const int bytes = (int)kMaxSegmentBytes;
    cudaError_t e = cudaFuncSetAttribute(k_sieve<kModeCount>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sieve<kModeBitmap>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_sieve(int mode, const SieveLaunch *d_launch, int grid, int threads, uint32_t seg_bytes,
                         cudaStream_t stream) {
    if (mode == kModeCount)
        k_sieve<kModeCount><<<grid, threads, seg_bytes, stream>>>(d_launch);
    else
        k_sieve<kModeBitmap><<<grid, threads, seg_bytes, stream>>>(d_launch);
    return cudaGetLastError();
}

cudaError_t launch_build_tile(uint8_t *tile, uint64_t stride, uint32_t len, uint32_t period, const uint32_t *ps,
                              int np, cudaStream_t stream) {
    if (np < 1 || np > 5) return cudaErrorInvalidValue;
    TilePrimes t{};
    for (int i = 0; i < np; ++i) t.p[i] = ps[i];
    dim3 grid((len + 255) / 256 < 4096 ? (len + 255) / 256 : 4096, kTileCopies);
    k_build_tile<<<grid, 256, 0, stream>>>(tile, stride, len, period, t, np);
    return cudaGetLastError();
}

cudaError_t launch_tiny_primes(uint32_t *out, uint32_t *n_out, cudaStream_t stream) {
    k_tiny_primes<<<1, 256, 0, stream>>>(out, n_out);
    return cudaGetLastError();
}

cudaError_t launch_magic(const uint32_t *primes, uint64_t *magic, uint64_t n, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    k_magic<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, stream>>>(primes, magic, n);
    return cudaGetLastError();
}


cudaError_t launch_finalize_count(const unsigned long long *count, const unsigned *overflow, uint64_t *out,
                                  cudaStream_t stream) {
    k_finalize_count<<<1, 1, 0, stream>>>(count, overflow, out);
    return cudaGetLastError();
}

namespace {
struct UploadBlock {
    uint64_t w[kUploadMaxBytes / 8];
};

// The launch block, passed by value, written to device memory, and the
// accumulators zeroed: one launch in place of a host-to-device copy and a memset.
__global__ void k_upload(const __grid_constant__ UploadBlock blk, uint32_t words, uint64_t *dst,
                         unsigned long long *acc, uint32_t acc_n) {
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = blk.w[i];
    for (uint32_t i = threadIdx.x; i < acc_n; i += blockDim.x) acc[i] = 0;
}
}  // namespace

cudaError_t launch_upload(void *dst, const void *src, size_t bytes, unsigned long long *acc, size_t acc_n,
                          cudaStream_t stream) {
    if (bytes > kUploadMaxBytes || bytes % 8 || acc_n > 0xffffffffu) return cudaErrorInvalidValue;
    UploadBlock blk;
    std::memcpy(blk.w, src, bytes);
    k_upload<<<1, 128, 0, stream>>>(blk, (uint32_t)(bytes / 8), static_cast<uint64_t *>(dst), acc, (uint32_t)acc_n);
    return cudaGetLastError();
}

cudaError_t launch_put_two(void *out, int out64, cudaStream_t stream, uint64_t sub) {
    if (out64)
        k_put_two<uint64_t><<<1, 1, 0, stream>>>(static_cast<uint64_t *>(out), 2 - sub);
    else
        k_put_two<uint32_t><<<1, 1, 0, stream>>>(static_cast<uint32_t *>(out), (uint32_t)(2 - sub));
    return cudaGetLastError();
}

}  // namespace gbs

namespace gbs {
cudaError_t launch_wait_selftest(const void *src, uint32_t bytes, int arm, uint32_t limit, int *status_dev,
                                 cudaStream_t stream) {
    k_wait_selftest<<<1, 256, bytes, stream>>>(static_cast<const uint4 *>(src), bytes, arm, limit, status_dev);
    return cudaGetLastError();
}
}  // namespace gbs
