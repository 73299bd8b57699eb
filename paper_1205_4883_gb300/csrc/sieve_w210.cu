// sieve_w210.cu -- the count-only segmented sieve on a mod-210 wheel.
//
// Layout: wheel group g holds the 48 integers 210 g + r, r running over the
// residues coprime to 210 in ascending order (r_0 = 1, r_1 = 11, ..., r_47 =
// 209); bit 48 g + i stands for 210 g + r_i.  Multiples of 2, 3, 5 and 7 have
// no bit, so a prime p is crossed at the multiples p m with m coprime to 210
// only: 48 / 210 of the integers instead of 8 / 30 on the mod-30 wheel, and
// 8 / 7 more integers per byte of shared memory.  Bits are packed LSB-first
// into 32-bit words, a group spans 1.5 words, and a segment of Sw words (Sw a
// multiple of 3) holds 2 Sw / 3 whole groups.  A pre-sieved pattern removes
// 11, 13, 17 and 19 (period 46189 groups).
//
// The multiples p m, m = 210 a + r_k, of a prime p = 210 pq + pr (class pc,
// r_pc = pr) lie in group p a + c_k, c_k = pq r_k + floor(pr r_k / 210), at bit
// index(pr r_k mod 210) of the group: for a fixed class k they form an
// arithmetic progression of stride 48 p bits (§3.1's crossing of the multiples
// of each prime, restricted to the wheel).
#include "internal.h"

namespace gbs {
namespace {

__device__ __forceinline__ uint32_t mod_barrett210(uint64_t x, uint32_t p, uint64_t M) {
    const uint64_t q = __umul64hi(x, M);
    const uint64_t r = x - q * (uint64_t)p;
    return (uint32_t)(r >= p ? r - p : r);
}

// floor(x / p) for x < 2^64 with M = floor((2^64 - 1) / p): umulhi(x, M) is the
// quotient or one less.
__device__ __forceinline__ uint64_t div_barrett210(uint64_t x, uint32_t p, uint64_t M) {
    uint64_t q = __umul64hi(x, M);
    if (x - q * (uint64_t)p >= p) ++q;
    return q;
}

__device__ __forceinline__ unsigned long long warp_sum210(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Number of base primes p (a prefix of length <= n) with p * p < E, by a
// 32-way search over the prefix; called by one full warp.
__device__ uint32_t primes_with_square_below210(const uint32_t *primes, uint32_t n, uint64_t E, int lane) {
    uint32_t a = 0, b = n;
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

// True when a segment starting at group G0 may begin before some class's first
// allowed multiple p m, m >= p: those lie below p^2 / 210 + 2 p groups.
__device__ __forceinline__ bool is_early210(uint64_t G0, uint32_t p) {
    return 210ull * G0 < (uint64_t)p * p + 420ull * p;
}

// Group offset (from the segment start G0) of the first multiple p m >= max(p^2,
// 210 G0) of class k, R = G0 mod p; values >= L mean no hit in the segment.
__device__ __forceinline__ uint32_t first_hit210(const W210Tables *__restrict__ T, uint32_t p, uint32_t pq,
                                                 uint32_t pc, uint32_t k, uint32_t R, uint64_t G0, bool early,
                                                 uint32_t L) {
    const uint32_t rk = __ldg(&T->r48[k]);
    const uint32_t ck = pq * rk + __ldg(&T->adj[pc * 48 + k]);
    uint32_t d = ck - R;
    if ((int32_t)d < 0) d += p;
    if (!early) return d;
    uint64_t start = G0 + d;
    const uint64_t q0 = p > rk ? (uint64_t)((p - rk + 209) / 210) : 0;  // m = 210 q + r_k >= p
    const uint64_t gmin = (uint64_t)p * q0 + ck;
    if (gmin > start) start = gmin;
    const uint64_t off = start - G0;
    return off < L ? (uint32_t)off : L;
}

// Bits of word w (relative to group G0 = integer 0) whose integers lie in
// [lo_rel, hi_rel).
__device__ uint32_t range_mask210(const W210Tables *__restrict__ T, uint32_t w, int64_t lo_rel, int64_t hi_rel) {
    uint32_t m = 0;
    for (uint32_t t = 0; t < 32; ++t) {
        const uint32_t b = 32 * w + t;
        const int64_t n = 210 * (int64_t)(b / 48) + __ldg(&T->r48[b % 48]);
        if (n >= lo_rel && n < hi_rel) m |= 1u << t;
    }
    return m;
}

__global__ void __launch_bounds__(1024, 1)
k_sieve210(const SieveLaunch *__restrict__ Pg, const W210Tables *__restrict__ T, const uint8_t *__restrict__ tile,
           uint64_t tile_stride) {
    extern __shared__ uint4 smem4[];
    uint32_t *seg32 = reinterpret_cast<uint32_t *>(smem4);
    __shared__ SieveLaunch P;  // launch parameters, read from device memory (graph-replayable)
    __shared__ unsigned long long s_item;
    __shared__ uint32_t s_range;
    __shared__ uint32_t s_small_next;
    __shared__ uint32_t s_nseg;
    __shared__ unsigned long long s_red[32];
    if (threadIdx.x == 0) P = *Pg;
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t C = P.chunk_segs;

    for (;;) {
        if (tid == 0) {
            const unsigned long long item = atomicAdd(P.item_counter, 1ull);
            s_item = item;
            if (item < P.n_items) {
                uint32_t a = 0, b = P.n_ranges - 1;  // largest r with item_first <= item
                while (a < b) {
                    const uint32_t mid = (a + b + 1) >> 1;
                    if (P.ranges[mid].item_first <= item) a = mid; else b = mid - 1;
                }
                s_range = a;
            }
        }
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= P.n_items) break;
        const uint32_t range_id = s_range;
        const RangeDesc &rd = P.ranges[range_id];
        const uint32_t Sw = rd.seg_bytes / 4, Sg = Sw / 3 * 2;  // this range's segment (<= the launch's)
        const uint64_t s0 = (item - rd.item_first) * C;
        const uint32_t nchunk = (uint32_t)(rd.nseg - s0 < C ? rd.nseg - s0 : C);
        const uint32_t n_range = rd.n_use;
        // per-CTA wheel cursors of the large primes, carried from segment to
        // segment of this chunk; valid for primes [mid_end, n_prev)
        uint32_t *const cursors = P.cursors ? P.cursors + (size_t)blockIdx.x * P.cursor_stride : nullptr;
        uint32_t n_prev = 0;
        for (uint32_t g = 0; g < nchunk; ++g) {
            const uint64_t s = s0 + g;
            const uint64_t G0 = (uint64_t)rd.Bbase + s * Sg;  // first group of the segment
            const uint64_t base_int = 210 * G0;
            const uint64_t need = (rd.hi - base_int + 209) / 210;  // groups up to hi
            const uint32_t L = need < Sg ? (uint32_t)need : Sg;
            const uint32_t Lw = (48 * L + 31) / 32;

            // 1. pre-sieved pattern (16-byte aligned copy of the shifted tile)
            {
                const uint64_t ph = (G0 % kW210Period) * 6;
                const uint32_t k = (uint32_t)ph & 15u;
                const uint4 *src = reinterpret_cast<const uint4 *>(tile + k * tile_stride + (ph - k));
                const uint32_t n16 = (Lw + 3) / 4;
                for (uint32_t i = tid; i < n16; i += blockDim.x) smem4[i] = __ldg(src + i);
            }
            if (tid < 32) {
                const uint64_t E0 = base_int + 210ull * L;
                const uint64_t E = E0 < rd.hi ? E0 : rd.hi;
                const uint32_t n = primes_with_square_below210(P.primes, n_range, E, lane);
                if (lane == 0) {
                    s_nseg = n;
                    s_small_next = 0;
                }
            }
            __syncthreads();
            const uint32_t n_use = s_nseg;
            const uint32_t small_end = P.small_end < n_use ? P.small_end : n_use;
            const uint32_t mid_end = rd.mid_end < n_use ? rd.mid_end : n_use;

            // 2a. medium primes [small_end, mid_end): one lane per prime, the
            //     warp taking 32 consecutive primes.  Each class progression
            //     (stride 48 p bits) is split into its even and odd hits: two
            //     sub-progressions of stride 96 p bits = 3 p words, each with
            //     one fixed mask (96 p = 0 mod 32).
            for (uint32_t base = P.small_end + (tid & ~31u); base < mid_end; base += blockDim.x) {
                const uint32_t i = base + lane;
                const bool valid = i < mid_end;
                const uint32_t p = valid ? __ldg(P.primes + i) : 1u;
                const uint64_t M = valid ? __ldg(P.magic + i) : ~0ull;
                const uint32_t R = mod_barrett210(G0, p, M);
                const uint32_t pq = p / 210, pc = valid ? __ldg(&T->idx[p - pq * 210]) : 0u;
                const bool early = is_early210(G0, p);
                const uint32_t lw = valid ? Lw : 0u, wstep = 3u * p;
                for (uint32_t k = 0; k < 48; ++k) {
                    const uint32_t d = first_hit210(T, p, pq, pc, k, R, G0, early, L);
                    const uint32_t b0 = 48u * d + __ldg(&T->bit[pc * 48 + k]);
#pragma unroll
                    for (uint32_t e = 0; e < 2; ++e) {
                        const uint32_t b = b0 + e * 48u * p;
                        const uint32_t mask = ~(1u << (b & 31u));
                        for (uint32_t w = d < L ? b >> 5 : lw; w < lw; w += wstep) atomicAnd(&seg32[w], mask);
                    }
                    __syncwarp();
                }
            }
            // 2b. large primes [mid_end, n_use): one lane per prime, walking its
            //     multiples class by class through the wheel (only the hits are
            //     visited).  The step from class k to k + 1 is pq gap_k +
            //     dadj_k groups; the packed step table holds the bit of class k,
            //     dadj_k and gap_k / 2.  With per-CTA cursors the walk resumes
            //     where the previous segment of the chunk left it.
            for (uint32_t base = mid_end + (tid & ~31u) * 4; base < n_use; base += blockDim.x * 4) {
                uint32_t pv[4], sv[4];
                uint64_t mv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t i = base + lane + 32u * u;
                    const bool valid = i < n_use;
                    pv[u] = valid ? __ldg(P.primes + i) : 1u;
                    const bool resume = valid && cursors && i < n_prev;
                    sv[u] = resume ? cursors[i - mid_end] : 0u;
                    mv[u] = (valid && !resume) ? __ldg(P.magic + i) : ~0ull;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t i = base + lane + 32u * u;
                    const bool valid = i < n_use;
                    const uint32_t p = pv[u];
                    const uint32_t pq = p / 210, pc = valid ? __ldg(&T->idx[p - pq * 210]) : 0u;
                    uint32_t off, k;
                    if (valid && cursors && i < n_prev) {  // (group offset from this segment) | class << 26
                        off = sv[u] & 0x3ffffffu;
                        k = sv[u] >> 26;
                    } else {
                        // first multiple at or after the segment start: a = floor(G0 / p),
                        // R = G0 mod p; class j lies before the start iff p r_j < 210 R,
                        // so k = #{ j : r_j <= floor((210 R - 1) / p) }
                        const uint64_t Q = div_barrett210(G0, p, mv[u]);
                        const uint32_t R = (uint32_t)(G0 - Q * p);
                        k = R ? __ldg(&T->cnt[(uint32_t)div_barrett210(210ull * R - 1, p, mv[u])]) : 0u;
                        uint64_t a = Q;
                        if (k == 48) {
                            k = 0;
                            ++a;
                        }
                        if (a < pq || (a == pq && k < pc)) {  // not before m = p
                            a = pq;
                            k = pc;
                        }
                        const uint64_t grp = (uint64_t)p * a + pq * __ldg(&T->r48[k]) + __ldg(&T->adj[pc * 48 + k]);
                        off = valid && grp - G0 < 0x7fffffffull ? (uint32_t)(grp - G0) : 0x7fffffffu;
                    }
                    const uint16_t *st = T->step + pc * 48;
                    const uint32_t l = valid ? L : 0u, pq2 = 2u * pq;
                    while (off < l) {
                        const uint32_t e = __ldg(st + k);
                        const uint32_t b = 48u * off + (e & 63u);
                        atomicAnd(&seg32[b >> 5], ~(1u << (b & 31u)));
                        off += pq2 * (e >> 10) + ((e >> 6) & 15u);
                        k = k == 47u ? 0u : k + 1u;
                    }
                    if (cursors && valid) cursors[i - mid_end] = (off - L) | (k << 26);
                }
                __syncwarp();
            }
            // 2c. small primes [8, small_end): one (prime, class) progression per
            //     warp, taken dynamically in decreasing order of work.  The
            //     progression (stride 48 p bits) is split into 64
            //     sub-progressions of stride 64 * 48 p bits = 96 p words; the
            //     hit t = s (mod 64) sits at bit b0 + 48 p s, whose value mod
            //     1024 is b0 + 16 (3 p s mod 64), so each 32-bit bank receives
            //     exactly two of them, at bits b0 mod 16 and b0 mod 16 + 16 of its
            //     words.  Lane l takes the two of bank l: a warp's 32 atomics
            //     never share a bank and each lane keeps two fixed masks.
            const uint32_t n_small = (small_end > kFirstCrossingPrime ? small_end - kFirstCrossingPrime : 0) * 48;
            for (;;) {
                uint32_t q = 0;
                if (lane == 0) q = atomicAdd(&s_small_next, 1u);
                q = __shfl_sync(0xffffffffu, q, 0);
                if (q >= n_small) break;
                const uint32_t i = kFirstCrossingPrime + q / 48, k = q % 48;
                const uint32_t p = __ldg(P.primes + i);
                const uint32_t R = mod_barrett210(G0, p, __ldg(P.magic + i));
                const uint32_t pq = p / 210, pc = __ldg(&T->idx[p - pq * 210]);
                const uint32_t d = first_hit210(T, p, pq, pc, k, R, G0, is_early210(G0, p), L);
                if (d >= L) continue;
                const uint32_t b0 = 48u * d + __ldg(&T->bit[pc * 48 + k]);
                const uint32_t a3 = 3u * p, inv = (a3 * (2u - a3 * a3)) & 63u;  // (3 p)^-1 mod 64
                const uint32_t uh = (b0 >> 4) & 63u, ul = b0 & 15u, wstep = 96u * p;
#pragma unroll
                for (uint32_t e = 0; e < 2; ++e) {
                    const uint32_t v = (2u * (uint32_t)lane + e - uh) & 63u;
                    const uint32_t sidx = (v * inv) & 63u;
                    uint32_t w = (b0 + 48u * p * sidx) >> 5;  // bank lane, bit 16 e + ul
                    const uint32_t mask = ~(1u << (16u * e + ul));
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

            // 3. group 0 (integers 0..209): 1 is not prime and 11, 13, 17, 19
            //    are, whatever the pattern says; no crossing reaches it
            if (tid == 0 && G0 == 0) {
                seg32[0] = kW210Group0Lo;
                seg32[1] = (seg32[1] & 0xffff0000u) | kW210Group0Hi;
            }
            __syncthreads();

            // 4. popcount of the bits in [lo, hi)
            unsigned long long cnt = 0;
            {
                const int64_t lo_rel = (int64_t)(rd.lo - base_int), hi_rel = (int64_t)(rd.hi - base_int);
                for (uint32_t w = tid; w < Lw; w += blockDim.x) {
                    uint32_t v = seg32[w];
                    const int64_t g_first = (32 * w) / 48, g_last = (32 * w + 31) / 48;
                    if (210 * g_first < lo_rel || 210 * (g_last + 1) > hi_rel) v &= range_mask210(T, w, lo_rel, hi_rel);
                    cnt += __popc(v);
                }
            }
            cnt = warp_sum210(cnt);
            if (lane == 0) s_red[tid >> 5] = cnt;
            __syncthreads();
            if (tid < 32) {
                unsigned long long v = tid < (int)(blockDim.x >> 5) ? s_red[tid] : 0ull;
                v = warp_sum210(v);
                if (tid == 0) {
                    if (s == 0) v += rd.corr;
                    atomicAdd(P.counts + range_id, v);
                }
            }
            n_prev = n_use;
            __syncthreads();
        }
    }
}

// Byte x of shifted copy k of the pattern: byte x + k of the periodic pattern,
// whose bit t stands for 210 g + r_i with 48 g + i = 8 (x + k) + t.
__global__ void k_build_tile210(const W210Tables *__restrict__ T, uint8_t *tile, uint64_t stride, uint32_t len) {
    const uint32_t k = blockIdx.y;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < len; x += gridDim.x * blockDim.x) {
        const uint32_t byte = (x + k) % kW210PeriodBytes;
        uint32_t v = 0;
#pragma unroll
        for (uint32_t t = 0; t < 8; ++t) {
            const uint32_t b = 8 * byte + t;
            const uint32_t n = 210 * (b / 48) + T->r48[b % 48];
            if (n % 11u && n % 13u && n % 17u && n % 19u) v |= 1u << t;
        }
        tile[k * stride + x] = (uint8_t)v;
    }
}

}  // namespace

void build_w210_tables(W210Tables *t) {
    uint32_t n = 0;
    for (uint32_t r = 0; r < 210; ++r) {
        t->idx[r] = 0xff;
        if (r % 2 && r % 3 && r % 5 && r % 7) {
            t->idx[r] = (uint8_t)n;
            t->r48[n++] = (uint8_t)r;
        }
    }
    for (uint32_t v = 0; v < 210; ++v) {
        uint32_t c = 0;
        for (uint32_t j = 0; j < 48; ++j) c += t->r48[j] <= v;
        t->cnt[v] = (uint8_t)c;
    }
    for (uint32_t c = 0; c < 48; ++c) {
        const uint32_t pr = t->r48[c];
        for (uint32_t k = 0; k < 48; ++k) {
            const uint32_t rk = t->r48[k], rk1 = k < 47 ? t->r48[k + 1] : 211u;
            t->adj[c * 48 + k] = (uint8_t)(pr * rk / 210);
            t->bit[c * 48 + k] = t->idx[pr * rk % 210];
            const uint32_t dadj = pr * rk1 / 210 - pr * rk / 210;  // <= 10
            const uint32_t gap2 = (rk1 - rk) / 2;                   // 1 .. 5
            t->step[c * 48 + k] = (uint16_t)(t->bit[c * 48 + k] | dadj << 6 | gap2 << 10);
        }
    }
}

cudaError_t set_sieve210_smem_limit() {
    return cudaFuncSetAttribute(k_sieve210, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kW210MaxSmemBytes);
}

cudaError_t launch_sieve210(const SieveLaunch *d_launch, const W210Tables *tab, const uint8_t *tile,
                            uint64_t tile_stride, int grid, int threads, uint32_t seg_bytes, cudaStream_t stream) {
    k_sieve210<<<grid, threads, seg_bytes, stream>>>(d_launch, tab, tile, tile_stride);
    return cudaGetLastError();
}

cudaError_t launch_build_tile210(const W210Tables *tab, uint8_t *tile, uint64_t stride, uint32_t len,
                                 cudaStream_t stream) {
    dim3 grid((len + 255) / 256 < 4096 ? (len + 255) / 256 : 4096, kTileCopies);
    k_build_tile210<<<grid, 256, 0, stream>>>(tab, tile, stride, len);
    return cudaGetLastError();
}

}  // namespace gbs
