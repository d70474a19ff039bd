"""Pins of the oracle's WENO-5 reconstruction and TVD RK-3 integrator (Sec. III:
WENO-5 of Jiang & Shu, RK-3 of Shu & Osher) against their textbook properties."""
import math

import numpy as np
import pytest

from oracle.oracle import ssprk3, weno5


def test_weno_constant_and_linear():
    assert weno5(2.5, 2.5, 2.5, 2.5, 2.5) == pytest.approx(2.5, abs=1e-15)
    # point values of a linear function: every candidate stencil is exact
    v = [0.1 * k - 0.3 for k in range(5)]
    assert weno5(*v) == pytest.approx(0.1 * 2.5 - 0.3, abs=1e-15)


def _fd_derivative(f, h):
    """d/dx of periodic point values f by WENO-5 fluxes (upwind, positive speed)."""
    n = len(f)
    ext = np.concatenate([f[-3:], f, f[:3]])
    # face k sits left of cell k; its upwind cell is k-1 (stencil k-3..k+1)
    face = np.array([weno5(*ext[k:k + 5]) for k in range(n + 1)])
    return (face[1:] - face[:-1]) / h


@pytest.mark.parametrize("shift", [0.0, 0.37])
def test_weno_fifth_order_on_smooth_data(shift):
    """Finite-difference WENO-5 is fifth-order accurate on smooth data away
    from critical points (Jiang & Shu 1996): f = exp(sin(2 pi x) + shift)
    restricted to where f' is bounded away from zero."""
    errs = []
    sizes = [40, 80, 160]
    for n in sizes:
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        f = np.exp(0.3 * np.sin(2 * np.pi * x) + shift)
        d = _fd_derivative(f, h)
        exact = f * 0.3 * 2 * np.pi * np.cos(2 * np.pi * x)
        mask = np.abs(np.cos(2 * np.pi * x)) > 0.3
        errs.append(np.max(np.abs(d - exact)[mask]))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > 4.5, (errs, rates)


def test_weno_is_essentially_non_oscillatory():
    """At a jump the reconstruction stays within the data range (to O(eps))."""
    for v in ([0, 0, 0, 1, 1], [0, 0, 1, 1, 1], [1, 1, 1, 0, 0]):
        r = weno5(*map(float, v))
        assert -1e-3 < r < 1 + 1e-3


def test_weno_shift_and_sign_covariance():
    """Smoothness indicators use differences only: adding a constant shifts
    the face value by it, and negating the data negates it."""
    rng = np.random.default_rng(0)
    for _ in range(10):
        v = rng.normal(size=5)
        r = weno5(*v)
        assert weno5(*(v + 3.0)) == pytest.approx(r + 3.0, abs=1e-13)
        assert weno5(*(-v)) == pytest.approx(-r, abs=1e-15)


@pytest.mark.parametrize("z", [-0.1, -0.8, -2.0, -2.5])
def test_rk3_amplification_real(z):
    """SSP RK-3 on y' = lam y multiplies by 1 + z + z^2/2 + z^3/6, z = lam dt."""
    y = ssprk3(np.array([1.0]), 1.0, lambda y: z * y)
    assert y[0] == pytest.approx(1 + z + z * z / 2 + z ** 3 / 6, rel=1e-14)


@pytest.mark.parametrize("a,b", [(-0.3, 1.1), (0.0, 1.5), (-1.0, 0.2)])
def test_rk3_amplification_complex(a, b):
    """Same on the rotation y' = [[a, -b], [b, a]] y, i.e. z = a + i b."""
    A = np.array([[a, -b], [b, a]])
    y = ssprk3(np.array([1.0, 0.0]), 1.0, lambda y: A @ y)
    z = complex(a, b)
    R = 1 + z + z * z / 2 + z ** 3 / 6
    assert y[0] == pytest.approx(R.real, abs=1e-14)
    assert y[1] == pytest.approx(R.imag, abs=1e-14)
