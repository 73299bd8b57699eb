// sieve_mr.cu -- the Miller-Rabin path for narrow ranges high up.
//
// A range on this path is sieved by k_sieve with the base primes below 2^16
// only; the integers it leaves at or above 65537^2 may still have a prime
// factor between 2^16 and sqrt(hi).  Each of them is decided here by the
// deterministic Miller-Rabin test (the improved form of the Fermat test the
// paper names after Section 3.2's Algorithm 3), whose modular exponentiation
// is Algorithm 2 (square, multiply when the low bit of the exponent is set,
// shift), carried out on Montgomery residues.  A composite is subtracted from
// its range's count and, in bitmap mode, loses its bit.
//
// Work is flat: one thread per word of survivors, over the words of all the
// ranges on the path (their prefix sums, SieveLaunch::mr_words, map a word to
// its range), so narrow ranges do not leave threads idle.

#include "internal.h"

namespace gbs {
namespace {

__constant__ uint32_t c_res_mr[8] = {1, 7, 11, 13, 17, 19, 23, 29};

// Montgomery product a b R^-1 mod n (R = 2^64) for odd n < 2^62 and a, b < n,
// with nprime = -n^-1 mod 2^64: t = a b, m = (t mod R) nprime, and
// (t + m n) / R < 2 n, less n if needed.  The low word of t + m n is 0, so
// the carry out of it is 1 exactly when t's low word is not 0.
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t n, uint64_t nprime) {
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    const uint64_t m = lo * nprime;
    const uint64_t r = hi + __umul64hi(m, n) + (lo != 0);
    return r >= n ? r - n : r;
}

// How many of the first primes, as bases, decide every n below the bound: psi_k,
// the smallest strong pseudoprime to the first k prime bases, is 2152302898747
// for k = 5, 3474749660383 for k = 6 and 341550071728321 for k = 7 and 8
// (Jaeschke, Math. Comp. 61, 1993), 3825123056546413051 for k = 9 (Jiang and
// Deng, Math. Comp. 83, 2014); the first twelve decide every n < 3.18e23
// (Sorenson and Webster, Math. Comp. 86, 2017).
__device__ __forceinline__ int mr_bases_needed(uint64_t n) {
    if (n < 2152302898747ull) return 5;
    if (n < 3474749660383ull) return 6;
    if (n < 341550071728321ull) return 7;
    if (n < 3825123056546413051ull) return 9;
    return 12;
}

// Deterministic Miller-Rabin for odd n < 2^62 with no prime factor below 37.
__device__ __noinline__ bool mr_is_prime(uint64_t n) {
    uint64_t inv = n;  // n^-1 mod 2^64 by Newton steps (n is its own inverse mod 8)
#pragma unroll
    for (int i = 0; i < 5; ++i) inv *= 2 - n * inv;
    const uint64_t nprime = 0 - inv;
    const uint64_t one = (0 - n) % n;  // R mod n: Montgomery form of 1
    uint64_t r2 = one;                 // R^2 mod n by 64 doublings
    for (int i = 0; i < 64; ++i) {
        r2 <<= 1;
        if (r2 >= n) r2 -= n;
    }
    const uint64_t minus_one = n - one;
    uint64_t d = n - 1;
    const int s = __ffsll((long long)d) - 1;
    d >>= s;
    const uint32_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    const int nb = mr_bases_needed(n);
    for (int b = 0; b < nb; ++b) {
        uint64_t y = mont_mul(bases[b], r2, n, nprime);  // a R mod n
        uint64_t x = one;
        for (uint64_t e = d; e; e >>= 1) {  // Algorithm 2: x = a^d mod n
            if (e & 1) x = mont_mul(x, y, n, nprime);
            y = mont_mul(y, y, n, nprime);
        }
        if (x == one || x == minus_one) continue;
        bool witness = true;
        for (int r = 1; r < s && witness; ++r) {
            x = mont_mul(x, x, n, nprime);
            if (x == minus_one) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// Survivors of the sieve by the primes below 2^16 in the ranges on the
// Miller-Rabin path: thread f takes flat word f of those ranges' words (range
// q = P->mr_list[k] owns words [mr_words[k], mr_words[k + 1])), tests every
// set bit in [lo, hi) at or above P->mr_square, clears the composites' bits
// (bitmap mode) and subtracts them from the range's count.  Count mode reads
// the raw wheel words k_sieve left (ODD = false); bitmap mode the odd-only
// words of the output (ODD = true).
template <bool ODD>
__global__ void __launch_bounds__(256) k_mr_filter(const SieveLaunch *__restrict__ P) {
    const uint32_t n_mr = P->n_mr;
    if (n_mr == 0) return;
    const uint32_t *__restrict__ prefix = P->mr_words;
    const uint32_t total = prefix[n_mr];
    for (uint32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < total; f += gridDim.x * blockDim.x) {
        uint32_t a = 0, b = n_mr - 1;  // the last k with prefix[k] <= f
        while (a < b) {
            const uint32_t mid = (a + b + 1) >> 1;
            if (__ldg(prefix + mid) <= f) a = mid; else b = mid - 1;
        }
        const uint32_t r = P->mr_list[a];
        const RangeDesc &rd = P->ranges[r];
        const uint64_t w = f - __ldg(prefix + a);
        uint32_t *words = rd.bitmap;
        uint32_t v = words[w], keep = v;
        unsigned long long composites = 0;
        const uint64_t o0 = rd.lo | 1;
        const int64_t base_int = 30 * rd.Bbase;
        while (v) {
            const int bit = __ffs(v) - 1;
            v &= v - 1;
            const int64_t n = ODD ? (int64_t)(o0 + 64 * w + 2 * (uint64_t)bit)
                                  : base_int + 120 * (int64_t)w + 30 * (bit >> 3) + (int64_t)c_res_mr[bit & 7];
            if (n < (int64_t)rd.lo || n >= (int64_t)rd.hi || (uint64_t)n < P->mr_square) continue;
            if (!mr_is_prime((uint64_t)n)) {
                keep &= ~(1u << bit);
                ++composites;
            }
        }
        if (ODD && keep != words[w]) words[w] = keep;
        if (composites) atomicAdd(P->counts + r, 0ull - composites);
    }
}

}  // namespace

cudaError_t launch_mr_filter(int mode, const SieveLaunch *d_launch, int grid, cudaStream_t stream) {
    if (mode == kModeCount)
        k_mr_filter<false><<<grid, 256, 0, stream>>>(d_launch);
    else
        k_mr_filter<true><<<grid, 256, 0, stream>>>(d_launch);
    return cudaGetLastError();
}

}  // namespace gbs
