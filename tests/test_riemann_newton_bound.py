"""The bound behind the kernels' Newton stopping rule for the star velocity (Sec. 2.1 flux;
the closed-form wave curves of reading c6).

The kernels solve phi(u) = p_1(u; u_L, p_L) - p_3(u; u_R, p_R) = 0 by safeguarded Newton.
They stop after a Newton step below 1e-9 c, because the error left is about K step^2 with
K = |phi''| / (2 |phi'|) at the root, and K stays below 0.5 / c. With two rarefactions
K = |u*| / (2 (u*^2 + c^2)) <= 1 / (4 c); shocks raise it to about 0.33 / c. This test checks
the bound in 40-digit arithmetic, with the wave curves restated from the PDE (Rankine-Hugoniot
shocks, closed-form rarefactions), on seeded states with |u_L|, |u_R| up to 100 c and
pressure jumps up to 2 * 10^4 c^2, for c = 1 and c = 0.1. The problem is invariant under
u -> u / c, p -> p / c^2, so K c does not depend on c.
"""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")


def wave1(u, uL, pL, c):
    c2 = c * c
    if u < uL:  # 1-shock: negative root s of s^2 - (uL + u) s - c^2 = 0, [p] = c^2 [u] / s
        sig = uL + u
        s = (sig - mp.sqrt(sig * sig + 4 * c2)) / 2
        return pL + c2 * (u - uL) / s
    G = lambda v: (v * v + v * mp.sqrt(v * v + c2) + c2 * mp.asinh(v / c)) / 2  # int (s + sqrt(s^2+c^2)) ds
    return pL - (G(u) - G(uL))


def wave3(u, uR, pR, c):
    c2 = c * c
    if u > uR:  # 3-shock: positive root
        sig = u + uR
        s = (sig + mp.sqrt(sig * sig + 4 * c2)) / 2
        return pR + c2 * (u - uR) / s
    H = lambda v: (v * mp.sqrt(v * v + c2) + c2 * mp.asinh(v / c) - v * v) / 2  # int (sqrt(s^2+c^2) - s) ds
    return pR - (H(uR) - H(u))


@pytest.mark.parametrize("c", [1.0, 0.1])
def test_newton_constant_below_bound(c):
    mp.mp.dps = 40
    rng = np.random.default_rng(97)
    cm = mp.mpf(c)
    worst = 0.0
    for R in (0.5, 4.0, 20.0, 100.0):
        for _ in range(40):
            ul, ur = [mp.mpf(x) * cm for x in rng.uniform(-R, R, 2)]
            pl, pr = [mp.mpf(x) * cm * cm for x in rng.uniform(-R * R, R * R, 2)]
            phi = lambda u: wave1(u, ul, pl, cm) - wave3(u, ur, pr, cm)
            # phi decreases strictly from +inf to -inf: bracket and bisect
            lo, hi = -cm * (10 * R * R + 10), cm * (10 * R * R + 10)
            assert phi(lo) > 0 > phi(hi)
            for _ in range(150):
                mid = (lo + hi) / 2
                if phi(mid) > 0:
                    lo = mid
                else:
                    hi = mid
            r = (lo + hi) / 2
            d1 = mp.diff(phi, r, 1)
            d2 = mp.diff(phi, r, 2)
            assert d1 < 0
            worst = max(worst, float(abs(d2) / (2 * abs(d1)) * cm))
    assert worst < 0.5, worst
