/*
 * oracle.c -- plain, slow, obviously correct CPU reference for the segmented
 * sieve of Eratosthenes.  TEST INFRASTRUCTURE ONLY: it is used by tests/, by
 * the smoke check and by the CPU baseline leg of bench.py, never by the
 * product path.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * What it computes (paper, Section 3.1, "Algorithm Design"): the sieve of
 * Eratosthenes marks as composite the multiples of each prime, starting from
 * the multiples of 2; what is left unmarked is prime.  Section 1 supplies the
 * bound that makes a range sieve possible: n is prime iff no prime <= sqrt(n)
 * divides it, so sieving [lo, hi) needs only the primes <= sqrt(hi - 1).
 * Eq. 3 splits the n integers into blocks of k; here a block ("segment") is a
 * fixed number of odd integers and the last one may be short (the reading of
 * Eq. 3 is N = ceil(n / k) blocks).
 *
 * Representation: one byte per ODD integer (no wheel, no bit packing inside
 * the sieve, no pre-sieved pattern).  2 is handled explicitly.  Packing into
 * the odd-only bitmap and the list is a separate, simple loop over the bytes.
 *
 * Result definitions (fixed readings, all exact integer):
 *   count(lo, hi)  = #{ p prime : lo <= p < hi }            (half-open range)
 *   bitmap(lo, hi) = o0 = lo | 1; bit i (word i >> 5, bit i & 31, LSB first)
 *                    is 1 iff o0 + 2 i is prime, 0 <= i < ceil((hi - o0) / 2);
 *                    bits past the range in the last word are 0.  2 has no bit.
 *   list(lo, hi)   = the primes in [lo, hi) ascending, 2 included.
 * 0 and 1 are not prime.
 *   crossings(lo, hi, pmin, w) = the bit-clears a wheel sieve of modulus w
 *                    performs on [lo, hi) for the primes >= pmin (defined at
 *                    oracle_crossings); the algorithmic work of the sieve.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

/* Odd integers per segment: 2^21 odd integers = 4 Mi integers, one byte each. */
#define ORACLE_SEG_ODDS (1u << 21)

/* floor(sqrt(n)) for any 64-bit n: the digit-by-digit (base 4) integer root. */
uint64_t oracle_isqrt(uint64_t n)
{
    uint64_t r = 0;
    /* bitwise integer square root: exact, no floating point */
    uint64_t bit = (uint64_t)1 << 62;
    while (bit > n) bit >>= 2;
    while (bit != 0) {
        if (n >= r + bit) {
            n -= r + bit;
            r = (r >> 1) + bit;
        } else {
            r >>= 1;
        }
        bit >>= 2;
    }
    return r;
}

/*
 * All primes <= limit, ascending, by the plain sieve of Eratosthenes over a
 * byte per integer (Section 3.1).  Writes at most cap of them to out (out may
 * be NULL) and returns how many there are.  Returns UINT64_MAX on allocation
 * failure.
 */
uint64_t oracle_base_primes(uint64_t limit, uint32_t *out, uint64_t cap)
{
    if (limit < 2) return 0;
    uint8_t *composite = (uint8_t *)calloc(limit + 1, 1);
    if (!composite) return UINT64_MAX;
    for (uint64_t p = 2; p * p <= limit; ++p) {
        if (composite[p]) continue;
        for (uint64_t m = p * p; m <= limit; m += p) composite[m] = 1;
    }
    uint64_t n = 0;
    for (uint64_t v = 2; v <= limit; ++v) {
        if (!composite[v]) {
            if (out && n < cap) out[n] = (uint32_t)v;
            ++n;
        }
    }
    free(composite);
    return n;
}

/*
 * Sieve one segment of odd integers.  mark[j] describes the odd integer
 * first_odd + 2 j for 0 <= j < nodds; on return mark[j] = 1 iff that integer
 * is composite or 1.  primes[0..np) are the odd primes <= sqrt(last integer).
 * For each prime p the crossing starts at max(p * p, the first odd multiple
 * of p >= first_odd) and steps by 2 p (the odd multiples), per Section 3.1.
 */
static void sieve_odd_segment(uint64_t first_odd, uint64_t nodds,
                              const uint32_t *primes, uint64_t np,
                              uint8_t *mark)
{
    memset(mark, 0, nodds);
    uint64_t last = first_odd + 2 * (nodds - 1);
    for (uint64_t k = 0; k < np; ++k) {
        uint64_t p = primes[k];
        if (p * p > last) break;
        uint64_t start = p * p;
        if (start < first_odd) {
            /* smallest multiple of p that is >= first_odd */
            uint64_t m = ((first_odd + p - 1) / p) * p;
            if ((m & 1) == 0) m += p; /* odd multiples only */
            start = m;
        }
        for (uint64_t m = start; m <= last; m += 2 * p)
            mark[(m - first_odd) / 2] = 1;
    }
    if (first_odd == 1) mark[0] = 1; /* 1 is not prime */
}

/* Bytes of mark[] needed for a range of nodds odd integers. */
static size_t seg_bytes(uint64_t nodds)
{
    return (size_t)(nodds < ORACLE_SEG_ODDS ? nodds : ORACLE_SEG_ODDS);
}

/* Odd primes <= sqrt(hi - 1), for sieving [lo, hi). */
static uint32_t *odd_base_primes(uint64_t hi, uint64_t *np)
{
    uint64_t lim = hi >= 2 ? oracle_isqrt(hi - 1) : 0;
    uint64_t n = oracle_base_primes(lim, NULL, 0);
    if (n == UINT64_MAX) return NULL;
    uint32_t *all = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!all) return NULL;
    oracle_base_primes(lim, all, n);
    /* drop 2: only odd integers are sieved */
    uint64_t j = 0;
    for (uint64_t i = 0; i < n; ++i)
        if (all[i] != 2) all[j++] = all[i];
    *np = j;
    return all;
}

/* ---------------------------------------------------------------- count */

typedef struct {
    uint64_t o0;      /* first odd integer of the whole range */
    uint64_t nodds;   /* odd integers in the whole range */
    uint64_t seg_begin, seg_end; /* segment indices handled by this thread */
    const uint32_t *primes;
    uint64_t np;
    uint64_t count;
    int failed;
} count_job;

static void *count_worker(void *arg)
{
    count_job *job = (count_job *)arg;
    uint8_t *mark = (uint8_t *)malloc(seg_bytes(job->nodds));
    if (!mark) { job->failed = 1; return NULL; }
    uint64_t c = 0;
    for (uint64_t s = job->seg_begin; s < job->seg_end; ++s) {
        uint64_t j0 = s * (uint64_t)ORACLE_SEG_ODDS;
        uint64_t n = job->nodds - j0;
        if (n > ORACLE_SEG_ODDS) n = ORACLE_SEG_ODDS;
        sieve_odd_segment(job->o0 + 2 * j0, n, job->primes, job->np, mark);
        for (uint64_t j = 0; j < n; ++j) c += (mark[j] == 0);
    }
    free(mark);
    job->count = c;
    return NULL;
}

static int pick_threads(int nthreads)
{
    if (nthreads > 0) return nthreads;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/*
 * Number of primes in [lo, hi) with nthreads threads (<= 0: one per online
 * core).  Returns UINT64_MAX on failure (bad range or no memory).
 */
uint64_t oracle_count(uint64_t lo, uint64_t hi, int nthreads)
{
    if (lo > hi) return UINT64_MAX;
    uint64_t c = (lo <= 2 && 2 < hi) ? 1 : 0;
    uint64_t o0 = lo | 1;
    if (o0 >= hi) return c;
    uint64_t nodds = (hi - o0 + 1) / 2;
    uint64_t np = 0;
    uint32_t *primes = odd_base_primes(hi, &np);
    if (!primes) return UINT64_MAX;
    uint64_t nseg = (nodds + ORACLE_SEG_ODDS - 1) / ORACLE_SEG_ODDS;
    int nt = pick_threads(nthreads);
    if ((uint64_t)nt > nseg) nt = (int)nseg;
    count_job *jobs = (count_job *)calloc((size_t)nt, sizeof(count_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
    if (!jobs || !tids) { free(jobs); free(tids); free(primes); return UINT64_MAX; }
    for (int t = 0; t < nt; ++t) {
        jobs[t].o0 = o0;
        jobs[t].nodds = nodds;
        jobs[t].seg_begin = nseg * (uint64_t)t / (uint64_t)nt;
        jobs[t].seg_end = nseg * (uint64_t)(t + 1) / (uint64_t)nt;
        jobs[t].primes = primes;
        jobs[t].np = np;
    }
    int failed = 0;
    for (int t = 1; t < nt; ++t)
        if (pthread_create(&tids[t], NULL, count_worker, &jobs[t]) != 0) {
            count_worker(&jobs[t]); /* run inline if no thread */
            tids[t] = 0;
        }
    count_worker(&jobs[0]);
    for (int t = 1; t < nt; ++t)
        if (tids[t]) pthread_join(tids[t], NULL);
    for (int t = 0; t < nt; ++t) {
        c += jobs[t].count;
        failed |= jobs[t].failed;
    }
    free(jobs); free(tids); free(primes);
    return failed ? UINT64_MAX : c;
}

/* ---------------------------------------------------------------- bitmap */

/*
 * The odd-only bitmap of [lo, hi) (layout in the header comment) into
 * out[0..nwords).  Words past the range are left untouched; bits past the
 * range inside the last word are written as 0.  Returns the number of
 * words the range needs, or UINT64_MAX on failure (out too small, bad range,
 * no memory).  Single-threaded: the packing loop is kept trivially simple.
 */
uint64_t oracle_bitmap(uint64_t lo, uint64_t hi, uint32_t *out, uint64_t nwords)
{
    if (lo > hi) return UINT64_MAX;
    uint64_t o0 = lo | 1;
    if (o0 >= hi) return 0;
    uint64_t nodds = (hi - o0 + 1) / 2;
    uint64_t need = (nodds + 31) / 32;
    if (nwords < need || !out) return UINT64_MAX;
    uint64_t np = 0;
    uint32_t *primes = odd_base_primes(hi, &np);
    uint8_t *mark = (uint8_t *)malloc(seg_bytes(nodds));
    if (!primes || !mark) { free(primes); free(mark); return UINT64_MAX; }
    memset(out, 0, need * sizeof(uint32_t));
    for (uint64_t j0 = 0; j0 < nodds; j0 += ORACLE_SEG_ODDS) {
        uint64_t n = nodds - j0;
        if (n > ORACLE_SEG_ODDS) n = ORACLE_SEG_ODDS;
        sieve_odd_segment(o0 + 2 * j0, n, primes, np, mark);
        for (uint64_t j = 0; j < n; ++j) {
            if (mark[j]) continue;
            uint64_t i = j0 + j; /* bit index: o0 + 2 i */
            out[i >> 5] |= (uint32_t)1 << (i & 31);
        }
    }
    free(primes); free(mark);
    return need;
}

/* ---------------------------------------------------------------- list */

/*
 * The primes of [lo, hi) ascending (2 included) into out[0..cap).  Returns
 * how many primes the range holds, even when that exceeds cap (only the
 * first cap are written), or UINT64_MAX on failure.
 */
uint64_t oracle_list(uint64_t lo, uint64_t hi, uint64_t *out, uint64_t cap)
{
    if (lo > hi) return UINT64_MAX;
    uint64_t n = 0;
    if (lo <= 2 && 2 < hi) {
        if (out && n < cap) out[n] = 2;
        ++n;
    }
    uint64_t o0 = lo | 1;
    if (o0 >= hi) return n;
    uint64_t nodds = (hi - o0 + 1) / 2;
    uint64_t np = 0;
    uint32_t *primes = odd_base_primes(hi, &np);
    uint8_t *mark = (uint8_t *)malloc(seg_bytes(nodds));
    if (!primes || !mark) { free(primes); free(mark); return UINT64_MAX; }
    for (uint64_t j0 = 0; j0 < nodds; j0 += ORACLE_SEG_ODDS) {
        uint64_t cnt = nodds - j0;
        if (cnt > ORACLE_SEG_ODDS) cnt = ORACLE_SEG_ODDS;
        sieve_odd_segment(o0 + 2 * j0, cnt, primes, np, mark);
        for (uint64_t j = 0; j < cnt; ++j) {
            if (mark[j]) continue;
            if (out && n < cap) out[n] = o0 + 2 * (j0 + j);
            ++n;
        }
    }
    free(primes); free(mark);
    return n;
}

/* ---------------------------------------------------------------- crossing work */

/* Greatest common divisor by Euclid's algorithm. */
static uint64_t gcd_u64(uint64_t a, uint64_t b)
{
    while (b != 0) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/*
 * #{ m : a <= m < b, gcd(m, w) = 1 }.  Every run of w consecutive integers
 * holds phi(w) of them (phi = that count over 1..w); the integers left after
 * the whole runs are tested one by one.
 */
static uint64_t coprime_between(uint64_t a, uint64_t b, uint64_t w, uint64_t phi)
{
    if (b <= a) return 0;
    uint64_t runs = (b - a) / w;
    uint64_t n = runs * phi;
    for (uint64_t m = a + runs * w; m < b; ++m)
        n += (gcd_u64(m, w) == 1);
    return n;
}

/*
 * The work of the crossing-off step on a wheel of modulus w.  Section 3.1
 * marks the multiples of each prime; Section 1 limits the primes to those
 * with p * p < hi; marking starts at p^2, i.e. at the multiple p * m with
 * m = p.  A wheel of modulus w (30, 210; w = 1 for no wheel) has no place for
 * integers sharing a factor with w, so only the multiples p * m with
 * gcd(m, w) = 1 are marked there.  The result is the number of pairs (p, m)
 * with p prime, pmin <= p, m >= p, gcd(m, w) = 1 and lo <= p * m < hi: one
 * bit-clear each (a composite with several such prime factors is cleared
 * once per factor).  Returns UINT64_MAX on failure (lo > hi, w = 0, no memory).
 */
uint64_t oracle_crossings(uint64_t lo, uint64_t hi, uint64_t pmin, uint64_t w)
{
    if (lo > hi || w == 0) return UINT64_MAX;
    if (hi < 2) return 0;
    uint64_t lim = oracle_isqrt(hi - 1); /* p * p < hi  <=>  p <= isqrt(hi - 1) */
    uint64_t np = oracle_base_primes(lim, NULL, 0);
    if (np == UINT64_MAX) return UINT64_MAX;
    uint32_t *primes = (uint32_t *)malloc((np ? np : 1) * sizeof(uint32_t));
    if (!primes) return UINT64_MAX;
    oracle_base_primes(lim, primes, np);
    uint64_t phi = 0;
    for (uint64_t m = 1; m <= w; ++m) phi += (gcd_u64(m, w) == 1);
    uint64_t total = 0;
    for (uint64_t k = 0; k < np; ++k) {
        uint64_t p = primes[k];
        if (p < pmin) continue;
        uint64_t m_lo = (lo + p - 1) / p;  /* smallest m with p * m >= lo */
        if (m_lo < p) m_lo = p;            /* marking starts at p * p */
        uint64_t m_hi = (hi - 1) / p + 1;  /* p * m < hi  <=>  m < m_hi */
        total += coprime_between(m_lo, m_hi, w, phi);
    }
    free(primes);
    return total;
}

/* Number of online cores the oracle uses when asked for "all of them". */
int oracle_default_threads(void) { return pick_threads(0); }
