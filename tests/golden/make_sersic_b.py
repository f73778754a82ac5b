"""Write sersic_b.txt: nu_n with P(2n, nu_n) = 1/2 (Sec. 4.1, the half-light
definition below Eq. sersic-intensity), to 25 significant digits.

Computed with mpmath's arbitrary-precision regularised incomplete gamma and
root finder at 50 digits: a reference independent of both the oracle's C code
and scipy.  Run: python tests/golden/make_sersic_b.py
"""
import os

import mpmath as mp

mp.mp.dps = 50
NS = ["0.2", "0.36", "0.5", "0.75", "1", "1.5", "2", "2.5", "3", "4", "5", "6", "8", "10"]


def nu(n):
    a = 2 * mp.mpf(n)
    f = lambda x: mp.gammainc(a, 0, x, regularized=True) - mp.mpf(1) / 2
    return mp.findroot(f, a - mp.mpf(1) / 3)


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sersic_b.txt")
    with open(out, "w") as fh:
        fh.write("# n  nu_n  (P(2n, nu_n) = 1/2; Sec. 4.1, Eq. sersic-intensity; mpmath 50 digits)\n")
        for n in NS:
            fh.write(f"{n} {mp.nstr(nu(n), 25)}\n")
