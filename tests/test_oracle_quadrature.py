"""Pins of the oracle's quadrature tables (Sec. III: half-range and full-range
Gauss-Hermite rules) against closed forms and the paper's weight formulas."""
import math

import numpy as np
import pytest

from oracle import quadrature as q

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 60


def half_moment(k):
    # int_0^inf z^k exp(-z^2/2)/sqrt(2 pi) dz = 2^((k-1)/2) Gamma((k+1)/2) / sqrt(2 pi)
    return mpmath.mpf(2) ** (mpmath.mpf(k - 1) / 2) * mpmath.gamma(mpmath.mpf(k + 1) / 2) / mpmath.sqrt(2 * mpmath.pi)


def full_moment(k):
    return mpmath.mpf(0) if k % 2 else 2 * half_moment(k)


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 7, 16, 24])
def test_half_range_exact_below_2Q(Q):
    r = q.HalfRangeRule(Q)
    z = [mpmath.mpf(str(v)) for v in r.z]
    w = [mpmath.mpf(str(v)) for v in r.w]
    for k in range(2 * Q):
        quad = mpmath.fsum(wi * zi ** k for wi, zi in zip(w, z))
        assert abs(quad / half_moment(k) - 1) < mpmath.mpf(10) ** -40, (Q, k)
    # degree 2Q is no longer integrated exactly
    quad = mpmath.fsum(wi * zi ** (2 * Q) for wi, zi in zip(w, z))
    assert abs(quad / half_moment(2 * Q) - 1) > mpmath.mpf(10) ** -30
    assert abs(sum(float(x) for x in r.w) - 0.5) < 1e-15
    assert all(float(x) > 0 for x in r.z)


@pytest.mark.parametrize("Q", [2, 4, 7, 16, 24])
def test_half_range_weight_formula_of_paper(Q):
    """Sec. III prints w_i = p_i a_{Q-1}^2 / (h_{Q-1}^2(p_i)[p_i + h_Q^2(0)/sqrt(2 pi)])."""
    r = q.HalfRangeRule(Q)
    paper = np.array(q.paper_half_range_weight(r))
    ours = np.array([float(x) for x in r.w])
    np.testing.assert_allclose(paper, ours, rtol=1e-14)


@pytest.mark.parametrize("Q", [1, 2, 4, 7, 20, 24])
def test_full_range_rule(Q):
    r = q.FullRangeRule(Q)
    y = [mpmath.mpf(str(v)) for v in r.y]
    w = [mpmath.mpf(str(v)) for v in r.w]
    for k in range(2 * Q):
        quad = mpmath.fsum(wi * yi ** k for wi, yi in zip(w, y))
        ref = full_moment(k)
        assert abs(quad - ref) < mpmath.mpf(10) ** -40 * max(1, abs(ref)), (Q, k)
    # textbook rule (numpy's probabilists' Gauss-Hermite), normalised by sqrt(2 pi)
    yn, wn = np.polynomial.hermite_e.hermegauss(Q)
    np.testing.assert_allclose([float(v) for v in r.y], yn, atol=1e-13)
    np.testing.assert_allclose([float(v) for v in r.w], wn / math.sqrt(2 * math.pi), rtol=1e-12, atol=1e-300)
    # Sec. III prints w_j = Q! / H_{Q+1}^2(y_j) (read: probabilists' He)
    np.testing.assert_allclose(q.paper_full_range_weight(r), [float(v) for v in r.w], rtol=1e-13)


@pytest.mark.parametrize("Q", [3, 7, 16])
def test_half_range_orthonormal(Q):
    """h_l orthonormal on [0, inf) with exp(-z^2/2)/sqrt(2 pi): checked by the
    rule itself (exact for degree <= 2Q-1) and by mpmath.quad."""
    r = q.HalfRangeRule(Q)
    c = [[mpmath.mpf(str(x)) for x in row] for row in r.coeff]

    def h(l, z):
        return mpmath.fsum(c[l][s] * z ** s for s in range(l + 1))

    for l, k in [(0, 0), (1, 1), (Q - 1, Q - 1), (1, Q - 1), (2, 3)]:
        val = mpmath.quad(lambda z: h(l, z) * h(k, z) * mpmath.exp(-z * z / 2) / mpmath.sqrt(2 * mpmath.pi),
                          [0, 5, 10, mpmath.inf])
        assert abs(val - (1 if l == k else 0)) < 1e-25, (l, k, val)


@pytest.mark.parametrize("N", [0, 1, 3, 6, 15, 23])
@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.37, 0.8), (-0.6, 1.5), (0.1, 0.18)])
def test_gx_bracket_is_twice_the_half_range_moment(N, u, T):
    """The bracket of Eq. gx, (T/2)^{s/2}[(1+erf z)P_s^+ + 2e^{-z^2}/sqrt(pi) P_s^*],
    with zeta = u/sqrt(2T), equals 2 int_0^inf p^s N(p; u, T) dp (p0 = 1)."""
    from oracle.oracle import gx_bracket
    B = gx_bracket(N, u / math.sqrt(2 * T), T / 2)
    for s in range(N + 1):
        ref = 2 * mpmath.quad(lambda p: p ** s * mpmath.exp(-(p - u) ** 2 / (2 * T)) / mpmath.sqrt(2 * mpmath.pi * T),
                              [0, mpmath.inf])
        assert abs(B[s] - float(ref)) <= 1e-14 * max(1.0, abs(float(ref))), (s, B[s], ref)
