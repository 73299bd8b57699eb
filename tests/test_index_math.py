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


# ---------------------------------------------------------------- mod-210 wheel
R48 = [r for r in range(210) if r % 2 and r % 3 and r % 5 and r % 7]
IDX48 = {r: i for i, r in enumerate(R48)}


def _multiples210(p, G0, L):
    """(group offset, class bit) of the multiples p m, m >= p, gcd(m, 210) = 1, in
    groups [G0, G0 + L) -- the plain definition."""
    out = []
    m = max(p, (210 * G0 + p - 1) // p)
    while p * m < 210 * (G0 + L):
        if m % 2 and m % 3 and m % 5 and m % 7 and p * m >= 210 * G0:
            out.append((p * m // 210 - G0, IDX48[p * m % 210]))
        m += 1
    return out


def test_w210_tables_and_group0():
    assert len(R48) == 48 and R48[0] == 1 and R48[1] == 11 and R48[-1] == 209
    composite = [r for r in R48 if r == 1 or any(r % d == 0 for d in range(2, int(r ** 0.5) + 1))]
    assert composite == [1, 121, 143, 169, 187, 209]
    bits = sum(1 << i for i, r in enumerate(R48) if r not in composite)
    assert bits & 0xFFFFFFFF == 0xF7FFFFFE and bits >> 32 == 0x7BBE


def test_w210_first_class_closed_form():
    # class j's first multiple of turn a = floor(G0 / p) lies before G0 iff c_j < R,
    # c_j = floor(p r_j / 210), i.e. iff r_j <= floor((210 R - 1) / p)
    rng = random.Random(11)
    cnt = [sum(1 for r in R48 if r <= v) for v in range(210)]
    primes = small_primes(200000)[5:]
    for _ in range(3000):
        p = rng.choice(primes)
        R = rng.randrange(0, p)
        want = sum(1 for r in R48 if p * r // 210 < R)
        got = cnt[(210 * R - 1) // p] if R else 0
        assert got == want, (p, R)


def test_w210_step_table_walk_equals_the_definition():
    rng = random.Random(12)
    primes = small_primes(60000)[5:]
    for _ in range(300):
        p = rng.choice(primes)
        L = rng.choice([64, 1024, 8192])
        G0 = rng.choice([rng.randrange(0, 10**6), p * p // 210 - rng.randrange(0, 3 * p),
                         rng.randrange(p * p // 210, p * p // 210 + 10**6)])
        G0 = max(G0, 0)
        pq, pr = divmod(p, 210)
        pc = IDX48[pr]
        # start: turn a = G0 // p, class k by the closed form, not before m = p
        Q, R = divmod(G0, p)
        k = sum(1 for r in R48 if r <= (210 * R - 1) // p) if R else 0
        a = Q
        if k == 48:
            k, a = 0, a + 1
        if a < pq or (a == pq and k < pc):
            a, k = pq, pc
        off = p * a + pq * R48[k] + (pr * R48[k]) // 210 - G0
        got = []
        while off < L:
            rk, rk1 = R48[k], (R48[k + 1] if k < 47 else 211)
            got.append((off, IDX48[pr * rk % 210]))
            dadj = pr * rk1 // 210 - pr * rk // 210
            assert 0 <= dadj <= 10 and 1 <= (rk1 - rk) // 2 <= 5
            off += 2 * pq * ((rk1 - rk) // 2) + dadj
            k = 0 if k == 47 else k + 1
        assert got == _multiples210(p, G0, L), (p, G0, L)


def test_w210_small_split_is_conflict_free_and_complete():
    # class progression b0 + 48 p t (bits); lane l, e in {0, 1} takes t = s (mod 64) with
    # 3 p s = 2 l + e - floor(b0 / 16) (mod 64): its words are l (mod 32), its bit 16 e + b0 mod 16
    rng = random.Random(13)
    for _ in range(400):
        p = rng.choice([23, 29, 31, 97, 101, 127, 211, 509])
        Lw = rng.choice([96, 1536, 57342])
        b0 = rng.randrange(0, 32 * Lw)
        a3 = 3 * p
        inv = (a3 * (2 - a3 * a3)) & 63
        assert (a3 * inv) % 64 == 1
        uh, ul = (b0 >> 4) & 63, b0 & 15
        got = []
        for lane in range(32):
            for e in range(2):
                v = (2 * lane + e - uh) & 63
                s = (v * inv) & 63
                b = b0 + 48 * p * s
                assert (b >> 5) % 32 == lane and b & 31 == 16 * e + ul
                w = b >> 5
                while w < Lw:
                    got.append(32 * w + 16 * e + ul)
                    w += 96 * p
        assert sorted(got) == list(range(b0, 32 * Lw, 48 * p))


def test_w210_medium_even_odd_split():
    # the even and odd hits of a class progression (stride 96 p bits = 3 p words) keep
    # one bit position each: b0 mod 32 and (b0 + 48 p) mod 32
    rng = random.Random(14)
    primes = small_primes(20000)[30:]
    for _ in range(150):
        p = rng.choice(primes)
        Lw = rng.choice([96, 1536, 57342])
        b0 = rng.randrange(0, 32 * Lw)
        got = []
        for e in range(2):
            b = b0 + e * 48 * p
            w = b >> 5
            while w < Lw:
                got.append(32 * w + (b & 31))
                w += 3 * p
        assert sorted(got) == list(range(b0, 32 * Lw, 48 * p))


def test_bitmap_words_from_wheel_byte_expansions():
    # odd-only word q of a 32-byte wheel group = bits [32 q, 32 q + 32) of the bytes'
    # 15-bit expansions laid end to end: bytes floor(32 q / 15) .. + 2, and + 3 when
    # 32 q mod 15 = 14 (q = 7), never past the group's byte 31
    rng = random.Random(15)
    for _ in range(200):
        group = [rng.randrange(256) for _ in range(32)]
        stream = 0
        for b, byte in enumerate(group):  # 15-bit expansion: bit (r - 1) / 2 for each residue present
            e = sum(1 << ((RES[k] - 1) // 2) for k in range(8) if byte >> k & 1)
            stream |= e << (15 * b)
        for q in range(15):
            b0, sh = divmod(32 * q, 15)
            need = 4 if sh == 14 else 3
            assert b0 + need - 1 <= 31 and (sh + 31 < 15 * need)
            part = 0
            for j in range(need):
                byte = group[b0 + j]
                e = sum(1 << ((RES[k] - 1) // 2) for k in range(8) if byte >> k & 1)
                part |= e << (15 * j)
            assert (part >> sh) & 0xFFFFFFFF == (stream >> (32 * q)) & 0xFFFFFFFF, q


def test_first_class_closed_form_mod30():
    # class j's first multiple of turn a = floor(B / p) lies before wheel byte B iff
    # c_j = floor(p r_j / 30) < R = B mod p, iff r_j <= floor((30 R - 1) / p)
    cnt = [sum(1 for r in RES if r <= v) for v in range(30)]
    packed = [(0x4443322221111110 >> (4 * v)) & 15 if v < 16 else (0x87777776666554 >> (4 * (v - 16))) & 15
              for v in range(30)]
    assert packed == cnt
    rng = random.Random(16)
    primes = small_primes(200000)[3:]
    for _ in range(3000):
        p = rng.choice(primes)
        R = rng.randrange(0, p)
        want = sum(1 for r in RES if p * r // 30 < R)
        assert (cnt[(30 * R - 1) // p] if R else 0) == want, (p, R)


def deal_medium_parts(costs, nwarps, L):
    """The medium tier's dealing by cost, as the kernel does it: warp w takes the
    cost interval [T w / n, T (w + 1) / n) of the cumulative costs W, and of each
    group g it overlaps the segment part [a, b), cut at 32-byte boundaries."""
    W = [0]
    for c in costs:
        W.append(W[-1] + c)
    G, T = len(costs), W[-1]
    parts = []  # (warp, group, a, b)
    for warp in range(nwarps):
        x0, x1 = T * warp // nwarps, T * (warp + 1) // nwarps
        g, hi = 0, G - 1  # the last group with W[g] <= x0 (binary search)
        while g < hi:
            mid = (g + hi + 1) >> 1
            if W[mid] <= x0:
                g = mid
            else:
                hi = mid - 1
        while g < G and W[g] < x1:
            w0, wg = W[g], W[g + 1] - W[g]
            u0, u1 = max(x0, w0) - w0, min(x1, w0 + wg) - w0
            a, b = (u0 * L // wg) & ~31, (u1 * L // wg) & ~31
            if a < b:
                parts.append((warp, g, a, b))
            g += 1
    return parts


def test_medium_groups_dealt_by_cost_cover_each_segment_once():
    # every group's parts, over all warps, tile [0, L) exactly, at 32-byte boundaries,
    # and no warp's share of the estimated cost exceeds its 1/n by more than one part
    rng = random.Random(1205)
    primes = small_primes(90000)
    for trial in range(300):
        nwarps = rng.choice([8, 16, 32])
        L = 32 * rng.randrange(1, 229376 // 32 + 1)
        S = rng.choice([L, 229376])
        first = rng.randrange(0, 200)
        G = rng.randrange(1, 257)
        costs = [224 + 8 * S // primes[min(first + 32 * g, len(primes) - 1)] for g in range(G)]
        parts = deal_medium_parts(costs, nwarps, L)
        by_group = {}
        for warp, g, a, b in parts:
            assert a % 32 == 0 and b % 32 == 0 and 0 <= a < b <= L
            by_group.setdefault(g, []).append((a, b, warp))
        assert sorted(by_group) == list(range(G)), trial
        for g, ps in by_group.items():
            ps.sort()
            assert ps[0][0] == 0 and ps[-1][1] == L, (trial, g)
            for (a0, b0, w0), (a1, b1, w1) in zip(ps, ps[1:]):
                assert b0 == a1 and w0 < w1, (trial, g)
    # the default tier (primes from 449, 232 groups): the first group costs more than a
    # warp's share, so it is split, and every warp's estimated cost is within one
    # part's setup of its share
    costs = [224 + 8 * 229376 // primes[86 - 8 + 32 * g] for g in range(232)]
    parts = deal_medium_parts(costs, 32, 229376)
    share = sum(costs) / 32
    assert costs[0] > share and len({w for w, g, a, b in parts if g == 0}) >= 2
    for w in range(32):
        est = sum(224 + (costs[g] - 224) * (b - a) / 229376 for ww, g, a, b in parts if ww == w)
        n = sum(1 for ww, *_ in parts if ww == w)
        assert est <= share + 224 * n + 32, (w, est, share)


def test_fixup_of_wheel_bytes_0_and_1():
    # after the patterns (7..19 and 23..59) every prime below 60 is cleared, so the
    # kernel rewrites wheel bytes 0 (integers 1..29) and 1 (31..59) with their true value
    def is_prime(n):
        return n > 1 and all(n % d for d in range(2, int(n ** 0.5) + 1))
    for byte, want in ((0, 0xFE), (1, 0xDF)):
        v = sum(1 << k for k, r in enumerate(RES) if is_prime(30 * byte + r))
        assert v == want, (byte, hex(v))
    # no later wheel byte holds a pattern prime: byte 2 starts at 61
    assert all(30 * 2 + r > 59 for r in RES)


def test_pattern_constants_of_the_kernels():
    # the constants in csrc/internal.h against their definitions: each pattern's
    # period is the product of its primes (wheel bytes), each copy holds a period
    # plus the largest segment plus 32 bytes rounded up to 16, and the first prime
    # the small tier crosses is the base prime after the last pattern prime
    import pathlib
    import re
    src = (pathlib.Path(__file__).resolve().parents[1] / "paper_1205_4883_gb300" / "csrc" / "internal.h").read_text()
    const = {m.group(1): int(m.group(2)) for m in re.finditer(r"constexpr uint32_t (k\w+) = (\d+)u;", src)}
    assert const["kTilePeriod"] == 7 * 11 * 13 * 17 * 19
    assert const["kXTilePeriod0"] == 23 * 29 * 31
    assert const["kXTilePeriod1"] == 37 * 41 * 43
    assert const["kXTilePeriod2"] == 47 * 53 * 59
    base = [2, 3, 5] + [p for p in range(7, 100) if all(p % d for d in range(2, int(p ** 0.5) + 1))]
    assert base[const["kFirstCrossingPrime"]] == 23
    assert base[const["kFirstCrossingPrimeX"]] == 61
    seg = const["kMaxSegmentBytes"]
    assert seg % 32 == 0 and seg + 3072 <= 227 * 1024
    for per in (const["kXTilePeriod0"], const["kXTilePeriod1"], const["kXTilePeriod2"]):
        stride = (per + seg + 32 + 15) & ~15
        # the furthest 16-byte read of a segment starts below the period and stays in the copy
        assert stride % 16 == 0 and ((per - 1) & ~15) + seg <= stride
