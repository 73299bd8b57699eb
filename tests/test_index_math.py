"""CPU checks of the index arithmetic the CUDA kernels rely on, written out in
Python: each split of a progression of multiples must visit exactly the
multiples the plain definition gives (no GPU; no oracle involved)."""
import random

RES = [1, 7, 11, 13, 17, 19, 23, 29]
IDX = {r: i for i, r in enumerate(RES)}
GAPS = 0x26424246


def small_primes(n):
    return [p for p in range(23, n) if all(p % d for d in range(2, int(p ** 0.5) + 1))]


def inv_mod128(p):
    x = p
    x = (x * (2 - p * x)) & 0xFFFFFFFF
    x = (x * (2 - p * x)) & 0xFFFFFFFF
    return x & 127


def test_128_subprogressions_cover_the_progression_with_fixed_banks():
    # warp-cooperative small primes: lane l, q in 0..3 takes bytes = 4 l + q (mod 128)
    rng = random.Random(1)
    for _ in range(400):
        p = rng.choice([23, 29, 31, 37, 41, 101, 997, 1787, 1789])
        L = rng.choice([32, 64, 1024, 4128, 229376])
        off = rng.randrange(0, L)
        assert p * inv_mod128(p) % 128 == 1
        got = []
        for lane in range(32):
            for q in range(4):
                kappa = (((4 * lane + q - off) & 0xFFFFFFFF) * inv_mod128(p)) & 127
                o = off + kappa * p
                assert o % 128 == 4 * lane + q  # bank = lane, byte phase = q
                w = o >> 2
                while w < L >> 2:
                    got.append(4 * w + q)
                    w += 32 * p
        assert sorted(got) == list(range(off, L, p))


def test_four_phase_subprogressions_cover_the_progression():
    # medium primes: p^-1 = p (mod 4), so off + ((ph - off) p mod 4) p = ph (mod 4)
    rng = random.Random(2)
    mediums = small_primes(40000)[300:]
    for _ in range(1500):
        p = rng.choice(mediums)
        L = rng.choice([32, 1024, 4128, 229376])
        off = rng.randrange(0, L)
        got = []
        for ph in range(4):
            o = off + ((((ph - off) & 0xFFFFFFFF) * p) & 3) * p
            assert o % 4 == ph
            w = o >> 2
            while w < L >> 2:
                got.append(4 * w + ph)
                w += p
        assert sorted(got) == list(range(off, L, p))


def _wheel_walk(p, B0, span):
    """Multiples p m (m coprime to 30, m >= p) with wheel byte in [B0, B0 + span), in
    wheel order, as the kernel's wheel cursor produces them: (byte, bit)."""
    Bc = max(B0, 0)
    Q, R = divmod(Bc, p)
    pq, pr = divmod(p, 30)
    pc = IDX[pr]
    adj = [(pr * r) // 30 for r in RES]
    k = sum(1 for j in range(8) if pq * RES[j] + adj[j] < R)
    a = Q
    if k == 8:
        k, a = 0, a + 1
    if a < pq or (a == pq and k < pc):
        a, k = pq, pc
    off = p * a + pq * RES[k] + adj[k] - B0
    out = []
    while off < span:
        out.append((B0 + off, IDX[(pr * RES[k]) % 30]))
        rk1 = RES[k + 1] if k < 7 else 31
        off += pq * ((GAPS >> (4 * k)) & 15) + ((pr * rk1) // 30 - (pr * RES[k]) // 30)
        k = (k + 1) & 7
    return out


def _direct(p, B0, span):
    lo, hi = 30 * B0, 30 * (B0 + span)
    out = []
    m = max(p, -(-max(lo, 0) // p))
    while p * m < hi:
        if m % 2 and m % 3 and m % 5 and p * m >= lo:
            out.append((p * m // 30, IDX[p * m % 30]))
        m += 1
    return out


def test_wheel_cursor_walk_equals_the_definition():
    rng = random.Random(3)
    primes = small_primes(60000)
    for _ in range(400):
        p = rng.choice(primes)
        span = rng.choice([64, 1024, 8192, 65536])
        B0 = rng.choice([-32, -2, 0, 1, rng.randrange(0, 10**6), p * p // 30 - rng.randrange(0, 3 * p),
                         rng.randrange(0, p * p // 30 + 5 * p + 1)])
        B0 = max(B0, -32)
        assert _wheel_walk(p, B0, span) == _direct(p, B0, span), (p, B0, span)


def test_grid_origin_aligns_odd_words():
    # 30 Bbase <= lo, 30 Bbase = 0 (mod 30) and 30 Bbase + 1 = lo | 1 (mod 64), Bbase >= -32
    for lo in list(range(0, 4000)) + [10**12 + k for k in range(200)]:
        o0 = lo | 1
        a = ((o0 - 1) & 63) // 2
        t0_res = 30 * ((15 * a) & 31)
        t0 = lo - ((lo % 960 - t0_res) % 960)
        assert t0 <= lo < t0 + 960 and t0 % 30 == 0 and (t0 + 1 - o0) % 64 == 0
        assert t0 // 30 >= -32


def test_montgomery_miller_rabin_as_the_kernel_does_it():
    # mont_mul / mr_is_prime of the kernel, 64-bit wraparound written out,
    # against the Miller-Rabin the oracle tests are pinned with
    from numtheory import mr_is_prime as reference
    m64 = (1 << 64) - 1

    def mont_mul(a, b, n, nprime):
        lo, hi = (a * b) & m64, (a * b) >> 64
        m = (lo * nprime) & m64
        r = hi + ((m * n) >> 64) + (1 if lo else 0)
        return r - n if r >= n else r

    def kernel_mr(n):
        inv = n
        for _ in range(5):
            inv = (inv * (2 - n * inv)) & m64
        nprime = (-inv) & m64
        one = ((-n) & m64) % n
        r2 = one
        for _ in range(64):
            r2 <<= 1
            if r2 >= n:
                r2 -= n
        minus_one = n - one
        d = n - 1
        s = (d & -d).bit_length() - 1
        d >>= s
        for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
            y, x, e = mont_mul(a, r2, n, nprime), one, d
            while e:
                if e & 1:
                    x = mont_mul(x, y, n, nprime)
                y = mont_mul(y, y, n, nprime)
                e >>= 1
            if x in (one, minus_one):
                continue
            for _ in range(1, s):
                x = mont_mul(x, x, n, nprime)
                if x == minus_one:
                    break
            else:
                return False
        return True

    rng = random.Random(4)
    small = (3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    done = 0
    while done < 1500:
        n = rng.randrange(2**32, 2**62) | 1
        if any(n % p == 0 for p in small):
            continue
        assert kernel_mr(n) == reference(n), n
        done += 1
    for n in (2152302898747, 3474749660383, 341550071728321):  # strong pseudoprimes to small bases
        assert not kernel_mr(n)
