"""Pins of the oracle's discrete equilibrium (Sec. III, Eqs. gx and gy) and of
its Shakhov relaxation target (Sec. II) against numerical integration and the
closed-form properties of the Shakhov model."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.oracle import Oracle

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40


def exact_sum(w, g, p, s):
    """sum_i w_i g_i p_i^s in 40-digit arithmetic (the float64 sum itself would
    cancel at high s), and sum_i |w_i g_i p_i^s|: the float64 rounding of the
    nodes and values moves the sum by ~1e-16 of the latter."""
    terms = [mpmath.mpf(a) * mpmath.mpf(b) * mpmath.mpf(c) ** s for a, b, c in zip(w, g, p)]
    return float(mpmath.fsum(terms)), float(mpmath.fsum(abs(t) for t in terms))

CASES = [(-0.4, 0.7), (0.0, 1.0), (0.25, 1.3), (0.9, 0.45)]


def gauss_half_moment(s, u, T, sign):
    """int over the half line sign*p > 0 of p^s N(p; u, T) dp, by adaptive quadrature."""
    f = lambda p: p ** s * math.exp(-(p - u) ** 2 / (2 * T)) / math.sqrt(2 * math.pi * T)
    lim = (0, np.inf) if sign > 0 else (-np.inf, 0)
    val, err = integrate.quad(f, *lim, epsabs=1e-14, epsrel=1e-13, limit=200)
    return val


@pytest.mark.parametrize("Qx,p0", [(4, 1.0), (7, 1.0), (7, 1.3), (12, 0.8), (16, 1.0), (24, 1.0)])
@pytest.mark.parametrize("u,T", CASES + [(0.1, 0.18), (-0.2, 1.82)])
def test_gx_recovers_half_range_moments(Qx, p0, u, T):
    """sum_{i in half} g_{x,i} p_i^s = int_half g p^s for s <= N_x (Sec. III)."""
    o = Oracle(dict(Qx=Qx, Qy=3, Nx=8, p0=p0))
    gx, _ = o.equilibrium_factors(u, 0.0, T)
    z, w = o.tab["zx"] * p0, o.tab["wx"]
    for s in range(min(o.Nxe, 12) + 1):
        plus, ap = exact_sum(w, gx[:Qx], z, s)
        minus, am = exact_sum(w, gx[Qx:], -z, s)
        rp, rm = gauss_half_moment(s, u, T, +1), gauss_half_moment(s, u, T, -1)
        assert abs(plus - rp) < 2e-12 * max(1.0, abs(rp)) + 1e-13 * ap, (s, plus, rp)
        assert abs(minus - rm) < 2e-12 * max(1.0, abs(rm)) + 1e-13 * am, (s, minus, rm)


@pytest.mark.parametrize("Qy,p0", [(4, 1.0), (7, 1.0), (9, 1.2), (20, 1.0), (24, 1.0)])
@pytest.mark.parametrize("u,T", CASES + [(0.1, 0.18), (-0.2, 1.82)])
def test_gy_recovers_full_range_moments(Qy, p0, u, T):
    """sum_j g_{y,j} p_j^l = E[(u + sqrt(T) Y)^l], l <= N_y (Sec. III, Eq. gy)."""
    o = Oracle(dict(Qx=2, Qy=Qy, Nx=8, p0=p0))
    _, gy = o.equilibrium_factors(0.0, u, T)
    y, w = o.tab["yy"] * p0, o.tab["wy"]
    for l in range(min(o.Nye, 12) + 1):
        # binomial expansion with Gaussian moments (k-1)!!
        ref = sum(math.comb(l, k) * u ** (l - k) * T ** (k / 2) * (math.prod(range(1, k, 2)) if k % 2 == 0 else 0)
                  for k in range(l + 1))
        got, absum = exact_sum(w, gy, y, l)
        assert abs(got - ref) < 1e-12 * max(1.0, abs(ref)) + 1e-13 * absum, (l, got, ref)


@pytest.mark.parametrize("Q", [4, 6, 8])
def test_discrete_maxwellian_moments(Q):
    """phi = n g_x g_y, chi = T phi has density n, velocity u, temperature T,
    pressure tensor n T delta_ij and zero heat flux (needs N >= 3)."""
    o = Oracle(dict(Qx=Q, Qy=Q, Nx=4))
    n, ux, uy, T = 1.3, 0.21, -0.33, 0.87
    gx, gy = o.equilibrium_factors(ux, uy, T)
    phi = n * np.outer(gx, gy).ravel()
    f = np.zeros((2, o.V, o.Nx))
    f[0] = phi[:, None]
    f[1] = T * phi[:, None]
    m = o.moments(f)[:, 0]
    ref = [n, ux, uy, T, n * T, n * T, n * T, 0.0, 0.0, 0.0]
    np.testing.assert_allclose(m, ref, rtol=1e-12, atol=1e-13)


def random_moments(rng):
    n = rng.uniform(0.7, 1.4)
    ux, uy = rng.uniform(-0.3, 0.3, 2)
    T = rng.uniform(0.7, 1.4)
    qx, qy = rng.uniform(-0.05, 0.05, 2)
    return np.array([n, ux, uy, T, 0, 0, 0, 0, qx, qy])


@pytest.mark.parametrize("N,conserved", [(3, 1), (4, 3), (5, 4), (6, 4), (9, 4)])
def test_shakhov_target_conservation(N, conserved):
    """The relaxation target keeps n (N >= 3), momentum (N >= 4) and energy
    (N >= 5) of the discrete distribution: degree counting of the integrals of
    g_x g_y (1 + S) (Sec. II, Shakhov terms)."""
    rng = np.random.default_rng(N)
    o = Oracle(dict(Qx=N + 1, Qy=N + 1, Nx=4, Pr=0.6))
    w, px, py = o.w, o.px, o.py
    for _ in range(3):
        m = random_moments(rng)
        tp, tc = o.target(m)
        n, ux, uy, T = m[:4]
        checks = [
            (np.sum(w * tp), n),
            (np.sum(w * px * tp), n * ux), (np.sum(w * py * tp), n * uy),
            (np.sum(w * ((px - ux) ** 2 + (py - uy) ** 2) * tp) + np.sum(w * tc), 3 * n * T),
        ]
        for k, (got, ref) in enumerate(checks[: [0, 1, 0, 3, 4][conserved]]):
            assert abs(got - ref) < 1e-12, (N, k, got, ref)


@pytest.mark.parametrize("N", [6, 8])
def test_shakhov_target_heat_flux(N):
    """With N >= 6 the target's heat flux is (1 - Pr) q: the Shakhov model sets
    the Prandtl number through the heat flux relaxation (Sec. II)."""
    rng = np.random.default_rng(7)
    Pr = 0.64
    o = Oracle(dict(Qx=N + 1, Qy=N + 1, Nx=4, Pr=Pr))
    w, px, py = o.w, o.px, o.py
    for _ in range(3):
        m = random_moments(rng)
        tp, tc = o.target(m)
        n, ux, uy, T = m[:4]
        xx, xy = px - ux, py - uy
        qx = np.sum(w * (0.5 * (xx ** 2 + xy ** 2) * xx * tp + 0.5 * xx * tc))
        qy = np.sum(w * (0.5 * (xx ** 2 + xy ** 2) * xy * tp + 0.5 * xy * tc))
        assert abs(qx - (1 - Pr) * m[8]) < 1e-12
        assert abs(qy - (1 - Pr) * m[9]) < 1e-12


def test_shakhov_reduces_to_bgk_at_unit_prandtl():
    """Pr = 1 switches the Shakhov factor off: the target is the Maxwellian."""
    o = Oracle(dict(Qx=5, Qy=5, Nx=4, Pr=1.0))
    m = np.array([1.1, 0.1, -0.2, 0.9, 0, 0, 0, 0, 0.03, -0.02])
    tp, tc = o.target(m)
    gx, gy = o.equilibrium_factors(0.1, -0.2, 0.9)
    feq = 1.1 * np.outer(gx, gy).ravel()
    np.testing.assert_allclose(tp, feq, rtol=1e-15)
    np.testing.assert_allclose(tc, 0.9 * feq, rtol=1e-15)
