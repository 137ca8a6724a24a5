"""Pins of the oracle's exact artificial-compressibility Riemann flux (Sec. 2.1).

The 1D system along the face normal is
    p_t + c^2 (u_n)_x = 0,  (u_n)_t + (u_n^2 + p)_x = 0,  (u_t)_t + (u_n u_t)_x = 0.
Checks that do not reuse the oracle's formulas: the star state satisfies the
Rankine-Hugoniot relations across a shock and the characteristic ODEs across a
rarefaction (integrated here by RK4), and the flux is consistent and
mirror-symmetric.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

C = 1.0


def _rk4(f, y0, t0, t1, n=3000):
    y = np.array(y0, dtype=np.float64)
    h = (t1 - t0) / n
    t = t0
    for _ in range(n):
        k1 = f(t, y)
        k2 = f(t + h / 2, y + h / 2 * k1)
        k3 = f(t + h / 2, y + h / 2 * k2)
        k4 = f(t + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += h
    return y


def _flux1d(un, ut, p, c):
    """Physical flux of the 1D AC system for (p, u_n, u_t)."""
    return np.array([c * c * un, un * un + p, un * ut])


def _check_wave(side, u_from, ut_from, p_from, us, ut_star, ps, c):
    """Check the star-side state against the wave connecting it to (u_from, p_from)."""
    a = lambda u: np.sqrt(u * u + c * c)
    if side == 1:
        shock = us < u_from
    else:
        shock = us > u_from
    if shock:
        # Rankine-Hugoniot on all three equations with one speed s
        qa = np.array([p_from, u_from, ut_from])
        qb = np.array([ps, us, ut_star])
        Fa, Fb = _flux1d(u_from, ut_from, p_from, c), _flux1d(us, ut_star, ps, c)
        s = (Fb[0] - Fa[0]) / (qb[0] - qa[0])
        np.testing.assert_allclose(s * (qb - qa), Fb - Fa, atol=1e-12 * (1 + np.abs(Fb - Fa).max()))
        # Lax: 1-shock slower than both 1-characteristics' ordering, negative; 3-shock positive
        if side == 1:
            assert s < 0 and u_from - a(u_from) > s > us - a(us)
        else:
            assert s > 0 and us + a(us) > s > u_from + a(u_from)
    else:
        # rarefaction: integrate dp/du and du_t/du along the right eigenvector
        if side == 1:
            f = lambda u, y: np.array([-(u + a(u)), -y[1] / a(u)])
        else:
            f = lambda u, y: np.array([a(u) - u, y[1] / a(u)])
        y = _rk4(f, [p_from, ut_from], u_from, us)
        np.testing.assert_allclose([ps, ut_star], y, atol=1e-11)


@pytest.mark.parametrize("seed", range(3))
def test_star_state_satisfies_wave_relations(seed):
    uL, pL, uR, pR = S.face_states(8, seed)
    for i in range(8):
        for d in range(3):
            flux, us, ps, uf = O.riemann(uL[i], pL[i], uR[i], pR[i], d, C)
            t = [j for j in range(3) if j != d]
            # the star pressure seen from the left through the 1-wave and from the right through the 3-wave
            # agree (single star state); the tangential velocity is the upwind side's star value
            tL = uL[i][t[0]] * O.tang1(us, uL[i][d], C)
            tR = uR[i][t[0]] * O.tang3(us, uR[i][d], C)
            _check_wave(1, uL[i][d], uL[i][t[0]], pL[i], us, tL, ps, C)
            _check_wave(3, uR[i][d], uR[i][t[0]], pR[i], us, tR, ps, C)
            expect = tL if us > 0 else tR
            assert abs(uf[t[0]] - expect) < 1e-13
            # flux = n.(u (x) u + p I) at the interface state, continuity flux = u*
            assert abs(flux[3] - us) < 1e-15
            assert abs(flux[d] - (us * us + ps)) < 1e-13
            assert abs(flux[t[1]] - uf[t[1]] * us) < 1e-13


@pytest.mark.parametrize("seed", range(3))
def test_consistency_equal_states(seed):
    uL, pL, _, _ = S.face_states(10, seed)
    for i in range(10):
        for d in range(3):
            flux, us, ps, uf = O.riemann(uL[i], pL[i], uL[i], pL[i], d, C)
            exact = np.array([uL[i][j] * uL[i][d] + (pL[i] if j == d else 0.0) for j in range(3)] + [uL[i][d]])
            np.testing.assert_allclose(flux, exact, atol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_mirror_symmetry(seed):
    # reflecting x_d -> -x_d and swapping the sides reverses u*, keeps p* and the tangential velocity
    uL, pL, uR, pR = S.face_states(10, seed)
    for i in range(10):
        for d in range(3):
            f1, us1, ps1, uf1 = O.riemann(uL[i], pL[i], uR[i], pR[i], d, C)
            rl, rr = uR[i].copy(), uL[i].copy()
            rl[d] *= -1
            rr[d] *= -1
            f2, us2, ps2, uf2 = O.riemann(rl, pR[i], rr, pL[i], d, C)
            assert abs(us1 + us2) < 1e-13 and abs(ps1 - ps2) < 1e-12
            for j in range(3):
                if j != d:
                    assert abs(uf1[j] - uf2[j]) < 1e-12


def test_linear_acoustics_limit():
    # for small jumps around a rest state the star state is the linear acoustic one:
    # u* = (uL+uR)/2 + (pL-pR)/(2c), p* = (pL+pR)/2 + c (uL-uR)/2
    eps = 1e-6
    rng = np.random.default_rng(4)
    for _ in range(10):
        a, b, pa, pb = eps * rng.standard_normal(4)
        _, us, ps, _ = O.riemann([a, 0, 0], pa, [b, 0, 0], pb, 0, C)
        assert abs(us - (0.5 * (a + b) + (pa - pb) / (2 * C))) < 1e-11
        assert abs(ps - (0.5 * (pa + pb) + C * (a - b) / 2)) < 1e-11


@pytest.mark.parametrize("seed", range(3))
def test_flux_tangent_vs_central_differences(seed):
    uL, pL, uR, pR = S.face_states(10, seed)
    rng = np.random.default_rng(100 + seed)
    for i in range(10):
        d = i % 3
        du = rng.standard_normal(8)
        ex = O.riemann_tangent(uL[i], pL[i], uR[i], pR[i], du[:3], du[3], du[4:7], du[7], d, C)
        h = 1e-6
        fp = O.riemann(uL[i] + h * du[:3], pL[i] + h * du[3], uR[i] + h * du[4:7], pR[i] + h * du[7], d, C)[0]
        fm = O.riemann(uL[i] - h * du[:3], pL[i] - h * du[3], uR[i] - h * du[4:7], pR[i] - h * du[7], d, C)[0]
        np.testing.assert_allclose(ex, (fp - fm) / (2 * h), rtol=1e-6, atol=1e-7)
