"""Pins of the oracle's two accelerations of steady solves: local (per-node)
pseudo-time steps with mass renormalisation, and the half channel with a
symmetry plane at x = 0 (Sec. II: phi(-x, -p_x, -p_y) = phi(x, p_x, p_y) for
walls of equal temperature moving at -u_w and +u_w).

What fixes them, independently of their own code: the plain RK-3 and
amplification factor of the node-wise step; the full-channel solution, whose
right half the half channel must reproduce step by step; and the steady state
of the global time step, which the local-step iteration must reach (the fixed
point of a pseudo-time iteration does not depend on its step sizes once the
mass is held)."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, grid, local_time_steps, ssprk3, ssprk3_nodal
from tests.helpers import moment_errors

SQ2 = math.sqrt(2.0)


# ---- node-wise RK-3 -------------------------------------------------------------------

def test_nodal_rk3_with_equal_steps_is_the_plain_rk3():
    rng = np.random.default_rng(1)
    A = rng.normal(size=(12, 12)) * 0.3
    y0 = rng.normal(size=(3, 4))
    fn = lambda y: (A @ y.ravel()).reshape(y.shape)   # noqa: E731
    a = ssprk3(y0.ravel(), 0.07, lambda y: A @ y)
    b = ssprk3_nodal(y0, np.full(4, 0.07), fn)
    assert np.array_equal(a, b.ravel())


def test_nodal_rk3_amplification_per_node():
    """y' = lambda y per component: node s is multiplied by 1 + z + z^2/2 + z^3/6, z = lambda dt_s."""
    lam = np.array([-1.0, -3.0, 0.5, -0.2, 2.0])
    dtn = np.array([0.01, 0.2, 0.05, 0.3, 0.11])
    y0 = np.array([[1.0, 2.0, -1.0, 0.5, 3.0], [0.3, -0.7, 1.1, 2.0, -1.5]])
    y = ssprk3_nodal(y0, dtn, lambda y: lam[None, :] * y).reshape(y0.shape)
    z = lam * dtn
    assert np.allclose(y, y0 * (1 + z + z * z / 2 + z ** 3 / 6), rtol=1e-15, atol=1e-15)


# ---- local time steps -------------------------------------------------------------------

@pytest.mark.parametrize("delta", [0.1, 5.0])
def test_local_steps_bound_and_minimum(delta):
    """dt_s respects the CFL bound of its own node and half the smallest relaxation time,
    equals the CFL bound where that is the smaller, and its minimum is the global step."""
    p = dict(Nx=20, Qx=5, Qy=4, stretch_A=0.95, delta=delta, T_left=0.7, T_right=1.3)
    o = Oracle(dict(p, local_dt=1))
    zmax = float(np.max(o.tab["zx"]))
    cfl_s = 0.5 * o.J * o.deta / zmax
    tau_min = min(T ** 0.5 / (T * delta * SQ2) for T in (1.0, 0.7, 1.3))   # omega = 0.5
    assert np.all(o.dtn <= cfl_s * (1 + 1e-15)) and np.all(o.dtn <= 0.5 * tau_min * (1 + 1e-15))
    assert np.all((np.abs(o.dtn - cfl_s) < 1e-16) | (np.abs(o.dtn - 0.5 * tau_min) < 1e-16))
    assert o.dtn.min() == pytest.approx(Oracle(p).dt, rel=1e-15)
    with pytest.raises(ValueError):
        local_time_steps(dict(p, dt=1e-3, cfl=0.5, p0=1.0, omega=0.5, delta=delta, T_left=0.7, T_right=1.3),
                         o.J, o.deta, zmax)


def test_local_steps_on_a_uniform_grid_are_the_global_step():
    """A = 0: every node has the same step and the fluxes telescope, so the mass
    ratio is 1 to round-off and the iteration is the time-accurate scheme."""
    p = dict(Nx=24, Qx=4, Qy=5, delta=0.8, T_left=0.7, T_right=1.3, u_left=-0.2, u_right=0.1)
    a, b = Oracle(p), Oracle(dict(p, local_dt=1))
    assert np.all(b.dtn == a.dt)
    a.run(60)
    b.run(60)
    assert np.max(np.abs(a.f - b.f)) < 1e-13


def test_rest_state_stays_a_fixed_point_with_local_steps():
    o = Oracle(dict(Nx=16, Qx=5, Qy=5, stretch_A=math.sqrt(0.9), delta=2.0, local_dt=1))
    f0 = o.f.copy()
    assert np.max(o.run(40)) < 1e-15
    assert np.max(np.abs(o.f - f0)) < 1e-13


def test_local_steps_hold_the_mass():
    """Without renormalisation the local steps change the mass (the fluxes do not
    telescope). A step of the iteration is that plain node-wise RK-3 step times
    M_ref / M(f^n), and the mass then differs from M_ref by one step's drift only."""
    p = dict(Nx=20, Qx=4, Qy=4, stretch_A=0.95, delta=0.3, T_left=0.6, T_right=1.5, u_left=-0.2,
             u_right=0.2, local_dt=1)
    o = Oracle(p)
    m0 = o.total_mass()
    f = o.f.copy()
    for _ in range(150):                       # the same iteration without renormalisation
        f = ssprk3_nodal(f, o.dtn, lambda y: o.rhs(y)[0]).reshape(f.shape)
    assert abs(o.total_mass(f) - m0) > 1e-6 * m0
    o.run(149)
    fn = o.f.copy()
    plain = ssprk3_nodal(fn, o.dtn, lambda y: o.rhs(y)[0]).reshape(fn.shape)
    o.run(1)
    assert np.max(np.abs(o.f - plain * (m0 / o.total_mass(fn)))) < 1e-15 * np.max(np.abs(plain))
    drift = o.total_mass(plain) - o.total_mass(fn)       # this step's own change of mass
    assert abs((o.total_mass() - m0) - m0 * drift / o.total_mass(fn)) < 1e-14


def test_local_steps_reach_the_global_steady_state():
    """The steady state does not depend on the pseudo-time steps: the local-step
    iteration stops at the global-step solution, in fewer steps on a stretched grid."""
    p = dict(Nx=16, Qx=4, Qy=4, stretch_A=0.9, delta=0.5, u_left=-0.1, u_right=0.15, T_left=0.8,
             T_right=1.2)
    g, l = Oracle(p), Oracle(dict(p, local_dt=1))
    m0 = g.total_mass()
    kg, rg = g.run_to_steady(1e-13, 100000)
    kl, rl = l.run_to_steady(1e-13, 100000)
    assert rg < 1e-13 and rl < 1e-13
    assert kl < kg / 2, (kl, kg)
    e = moment_errors(l.moments(), g.moments())   # both within their distance to the limit
    assert np.all(e < 1e-8), e
    assert abs(l.total_mass() - m0) < 1e-12


# ---- half channel -------------------------------------------------------------------------

def test_half_grid_is_the_right_half_of_the_full_grid():
    for A in (0.0, 0.98):
        x, J, d = grid(32, A)
        xh, Jh, dh = grid(16, A, half=True)
        assert np.array_equal(x[16:], xh) and np.array_equal(J[16:], Jh) and d == dh
        assert xh[0] > 0 and xh[-1] < 0.5


@pytest.mark.parametrize("A,delta", [(0.0, 1.0), (0.9, 0.2), (0.98, 8.0)])
def test_half_channel_follows_the_full_channel(A, delta):
    """From the rest state, each step of the half channel equals the right half of
    the full channel of twice the nodes (same grid, same time step)."""
    S, Qx, Qy = 12, 5, 6
    p = dict(Nx=2 * S, Qx=Qx, Qy=Qy, stretch_A=A, delta=delta, u_left=-0.3, u_right=0.3, T_left=1.3,
             T_right=1.3, omega=0.7)
    full, half = Oracle(p), Oracle(dict(p, Nx=S, half_channel=1))
    assert half.dt == full.dt
    for _ in range(3):
        full.run(40)
        half.run(40)
        scale = np.max(np.abs(full.f))
        assert np.max(np.abs(full.f[:, :, S:] - half.f)) < 1e-12 * scale
    e = moment_errors(half.moments(), full.moments()[:, S:])
    assert np.all(e < 1e-11), e


def test_half_channel_conserves_mass():
    """The symmetry plane carries no mass flux (each face value of a velocity equals
    that of its mirror, with the opposite p_x): mass is conserved to round-off."""
    o = Oracle(dict(Nx=20, Qx=4, Qy=5, stretch_A=0.9, delta=0.7, u_left=-0.25, u_right=0.25, T_left=1.4,
                    T_right=1.4, half_channel=1))
    m0 = o.total_mass()
    o.run(150)
    assert abs(o.total_mass() - m0) < 1e-14
    _, nw = o.rhs()
    assert nw[0] == 0.0 and nw[1] > 0


def test_half_channel_with_local_steps_reaches_the_full_steady_state():
    S = 8
    p = dict(Nx=2 * S, Qx=4, Qy=4, stretch_A=0.9, delta=0.5, u_left=-0.12, u_right=0.12)
    full, half = Oracle(p), Oracle(dict(p, Nx=S, half_channel=1, local_dt=1))
    full.run_to_steady(1e-13, 100000)
    _, r = half.run_to_steady(1e-13, 100000)
    assert r < 1e-13
    e = moment_errors(half.moments(), full.moments()[:, S:])
    assert np.all(e < 1e-8), e


def test_half_channel_needs_symmetric_walls():
    for bad in (dict(T_left=1.1), dict(u_left=0.1, u_right=0.2)):
        with pytest.raises(ValueError):
            Oracle(dict(dict(Nx=8, Qx=4, Qy=4, u_left=-0.1, u_right=0.1, half_channel=1), **bad))
