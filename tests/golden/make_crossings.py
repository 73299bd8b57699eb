"""Writes crossings.txt: the crossing-off work of the wheel sieve on the
benchmarked ranges, computed by the CPU oracle alone (oracle.crossings).

The paper prints no such values.  Each line is the number of pairs (p, m),
p prime >= pmin with p^2 < hi, m >= p, gcd(m, wheel) = 1, lo <= p m < hi:
the bit-clears of Section 3.1's marking of multiples on a wheel of that
modulus.  pmin = 23 is the work of the mod-30 sieve after the pattern of
7..19 (every clear, however the kernel makes it); pmin = 61 and 73 the clears
left after the further patterns of 23..59 and 23..71; wheel 210 the mod-210
count path.

  python tests/golden/make_crossings.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

RANGES = [
    (0, 10**12, 23, 30), (0, 10**12, 61, 30), (0, 10**12, 73, 30), (0, 10**12, 23, 210),
    (0, 1 << 32, 23, 30), (0, 1 << 32, 61, 30),
    (0, 10**7, 23, 30), (0, 10**7, 61, 30),
    (10**14, 10**14 + 10**10, 23, 30), (10**14, 10**14 + 10**10, 61, 30),
    (0, 10**11, 23, 30),
]


def main():
    lines = ["# Crossing-off work (bit-clears) of the wheel sieve, from the CPU oracle",
             "# (oracle.crossings; written by make_crossings.py, no other source).",
             "# Format: lo hi pmin wheel clears"]
    for lo, hi, pmin, w in RANGES:
        lines.append(f"{lo} {hi} {pmin} {w} {oracle.crossings(lo, hi, pmin, w)}")
    with open(os.path.join(HERE, "crossings.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
