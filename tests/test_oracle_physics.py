"""Pins of the oracle's whole time step against what the physics of planar
Couette flow fixes: equilibrium fixed point, exact mass conservation with
diffuse walls (Eqs. diffuse, diffuse_nw), the mirror symmetry of Sec. II, the
free-molecular closed form (delta -> 0) and the Navier-Stokes limit
(P_xy = -mu du_y/dx with mu from Eq. tau, delta large)."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle

SQ2 = math.sqrt(2.0)


@pytest.mark.parametrize("Q,A,p0", [(4, 0.0, 1.0), (5, math.sqrt(0.9), 1.0), (6, 0.5, 1.2)])
def test_rest_maxwellian_is_a_fixed_point(Q, A, p0):
    o = Oracle(dict(Nx=16, Qx=Q, Qy=Q, stretch_A=A, p0=p0, delta=2.0))
    f0 = o.f.copy()
    res = o.run(40)
    assert np.max(res) < 1e-15
    assert np.max(np.abs(o.f - f0)) < 1e-13


@pytest.mark.parametrize("delta", [0.0, 0.7, 20.0])
@pytest.mark.parametrize("A", [0.0, math.sqrt(0.9)])
def test_mass_is_conserved(delta, A):
    """Telescoping fluxes, zero wall mass flux and a collision that keeps n
    (N >= 3) conserve sum_s J_s deta n_s to round-off."""
    o = Oracle(dict(Nx=24, Qx=4, Qy=5, stretch_A=A, delta=delta, T_left=0.6, T_right=1.4,
                    u_left=-0.2, u_right=0.3, omega=0.7))
    m0 = o.total_mass()
    o.run(150)
    assert abs(o.total_mass() - m0) < 2e-14


def test_wall_density_balances_the_mass_flux():
    """With an outgoing flux the wall density n_w of Eq. diffuse_nw is such
    that the rate of change of mass vanishes: d/dt sum J deta n = 0."""
    o = Oracle(dict(Nx=16, Qx=5, Qy=4, delta=1.0, T_left=0.8, T_right=1.3, u_left=0.1, u_right=-0.2))
    o.run(30)
    L, nw = o.rhs()
    dndt = np.sum(o.w[:, None] * L[0], axis=0)
    assert abs(np.sum(o.J * o.deta * dndt)) < 1e-13
    assert np.all(nw > 0)


def test_mirror_symmetry():
    """phi(-x, -p_x, -p_y) = phi(x, p_x, p_y) for walls moving at -u_w, +u_w
    with equal temperatures (Sec. II)."""
    Qx, Qy, Nx = 5, 6, 20
    o = Oracle(dict(Nx=Nx, Qx=Qx, Qy=Qy, stretch_A=0.8, delta=1.5, u_left=-0.25, u_right=0.25))
    o.run(200)
    f = o.f.reshape(2, 2, Qx, Qy, Nx)
    mirrored = f[:, ::-1, :, ::-1, ::-1]          # -p_x swaps halves, -p_y reverses j, -x reverses s
    assert np.max(np.abs(f - mirrored)) < 1e-12 * np.max(np.abs(f))


@pytest.mark.parametrize("TL,TR,uL,uR", [(1.0, 1.0, -0.1, 0.1), (0.8, 1.2, -0.1, 0.15), (0.5, 2.0, 0.05, 0.3)])
def test_free_molecular_closed_form(TL, TR, uL, uR):
    """delta = 0: each half of the velocity set carries its wall's Maxwellian,
    n_L sqrt(T_L) = n_R sqrt(T_R) (zero mass flux) and (n_L + n_R)/2 = 1, so
    P_xy = -(u_R - u_L) 2 sqrt(T_L T_R) / ((sqrt T_L + sqrt T_R) sqrt(2 pi))."""
    o = Oracle(dict(Nx=12, Qx=4, Qy=4, delta=0.0, T_left=TL, T_right=TR, u_left=uL, u_right=uR))
    k, r = o.run_to_steady(1e-14, 400000)
    assert r < 1e-14
    m = o.moments()
    sL, sR = math.sqrt(TL), math.sqrt(TR)
    pxy = -(uR - uL) * 2 * sL * sR / ((sL + sR) * math.sqrt(2 * math.pi))
    np.testing.assert_allclose(m[0], 1.0, atol=1e-10)
    np.testing.assert_allclose(m[7], pxy, atol=1e-10)
    _, nw = o.rhs()
    np.testing.assert_allclose(nw, [2 * sR / (sL + sR), 2 * sL / (sL + sR)], atol=1e-10)
    # mean wall-parallel velocity (n_L u_L + n_R u_R)/2
    uy = (uL * 2 * sR / (sL + sR) + uR * 2 * sL / (sL + sR)) / 2
    np.testing.assert_allclose(m[2], uy, atol=1e-10)


def test_shear_number_free_molecular():
    """Eq. Pi with equal walls at u_w = sqrt(2) v_ref: Pi = -T_xy/(2 P_ref) -> 1/sqrt(pi) as delta -> 0."""
    uw = SQ2
    o = Oracle(dict(Nx=8, Qx=4, Qy=7, delta=0.0, u_left=-uw, u_right=uw))
    o.run_to_steady(1e-14, 400000)
    pi_num = -o.moments()[7] / (2.0 * 1.0)
    np.testing.assert_allclose(pi_num, 1 / math.sqrt(math.pi), rtol=1e-10)


def test_navier_stokes_limit():
    """delta = 100: the bulk shear stress follows Newton's law with the
    viscosity of Eq. tau, mu = T^omega / (delta sqrt 2) (L = v_ref = 1)."""
    uw, delta, omega = 0.05, 100.0, 0.5
    o = Oracle(dict(Nx=32, Qx=5, Qy=5, delta=delta, u_left=-uw, u_right=uw, omega=omega))
    f = np.zeros((2, o.V, o.Nx))
    for s in range(o.Nx):   # start near the answer: local Maxwellian with a linear profile
        gx, gy = o.equilibrium_factors(0.0, 1.8 * uw * o.x[s], 1.0)
        g = np.outer(gx, gy).ravel()
        f[0, :, s] = g
        f[1, :, s] = g
    o.set_state(f)
    k, r = o.run_to_steady(1e-11, 60000)
    assert r < 1e-11
    m = o.moments()
    dudx = np.gradient(m[2], o.x)
    mu = m[3] ** omega / (delta * SQ2)
    bulk = slice(8, 24)
    np.testing.assert_allclose(m[7][bulk], (-mu * dudx)[bulk], rtol=2e-4)
    # and Pi -> 1/delta (Eq. Pi with u_w -> the slip-free velocity jump) to O(1/delta)
    assert abs(-m[7][16] / (2 * uw) * delta * SQ2 - 1) < 0.05


@pytest.mark.parametrize("delta,Q", [(1.0, 5), (10.0, 6)])
def test_steady_momentum_flux_and_shear_stress_uniform(delta, Q):
    """Steady state at finite delta (Sec. II, Eq. boltz_red): with a collision term
    that conserves y-momentum (N >= 4), the y-momentum balance of the reduced
    equation makes the p_y-momentum flux through every interface the same. The
    interface fluxes are recovered from L = dphi/dt by the flux-form telescoping
    G_{s+1/2} - G_{1/2} = -sum_{k <= s} J_k deta sum_v w_v p_y L_v,k; they are uniform
    to the residual. The nodal P_xy is the same flux seen through the nodes: in the
    central half of the channel (away from the walls' kinetic layers) it is uniform to
    the WENO-5 truncation error, which falls at the scheme's order under refinement;
    the mass flux n u_x vanishes to the same truncation."""
    spreads = []
    for Nx in (16, 32):
        o = Oracle(dict(Nx=Nx, Qx=Q, Qy=Q, delta=delta, u_left=-0.1, u_right=0.1, omega=0.5))
        k, r = o.run_to_steady(1e-12, 400000)
        assert r < 1e-12
        L, _ = o.rhs()
        dmom = (o.w * o.py) @ L[0]                       # d/dt (n u_y) per node
        G = np.cumsum(o.J * o.deta * dmom)               # G_{s+1/2} - G_{1/2}, up to sign
        m = o.moments()
        pxy = m[7]
        assert np.max(np.abs(G)) < 1e-9 * abs(pxy.mean()) + 100 * r
        bulk = slice(Nx // 4, 3 * Nx // 4)
        spreads.append((pxy[bulk].max() - pxy[bulk].min()) / abs(pxy.mean()))
        assert np.max(np.abs(m[0] * m[1])) < 1e-5 * 16 / Nx
    # WENO-5 is fifth order on smooth profiles: at least a factor 2^4 per halving of the spacing
    assert spreads[1] < spreads[0] / 16, spreads
    assert spreads[1] < 1e-6, spreads


def test_outgoing_ghosts_extrapolate_cubics_exactly():
    """The outgoing ghost nodes beyond each wall extrapolate the last four nodes by the
    cubic through them (reading R6 of the wall treatment; the paper's discrete form is
    silent): on rows that are cubics in the node index, the advection of the outgoing
    populations at the two nodes next to a wall equals that of the same cubic on a grid
    where the ghost positions are real nodes. A lower-order extrapolation differs by a
    multiple of the rows' third difference."""
    Nx, ext, Q = 12, 4, 4
    small = Oracle(dict(Nx=Nx, Qx=Q, Qy=Q, delta=0.0))
    big = Oracle(dict(Nx=Nx + 2 * ext, Qx=Q, Qy=Q, delta=0.0))
    rng = np.random.default_rng(7)
    c = rng.uniform(-1, 1, size=(2, small.V, 4)) * np.array([1.0, 0.3, 0.05, 0.004])
    s_big = np.arange(Nx + 2 * ext) - ext - (Nx - 1) / 2          # node index, centred
    rows = np.einsum("fvk,ks->fvs", c, np.vstack([s_big ** k for k in range(4)])) + 2.0
    big.set_state(rows)
    small.set_state(rows[:, :, ext:ext + Nx].copy())
    L_small, _ = small.rhs()
    L_big, _ = big.rhs()
    # uniform grids (J = 1): L deta is the flux difference, independent of the spacing
    a = L_small * small.deta
    b = L_big[:, :, ext:ext + Nx] * big.deta
    right, left = small.px > 0, small.px < 0
    scale = np.max(np.abs(b))
    for nodes, rows_sel in (([Nx - 1, Nx - 2], right), ([0, 1], left)):
        d = np.abs(a[:, rows_sel][:, :, nodes] - b[:, rows_sel][:, :, nodes])
        assert np.max(d) < 1e-12 * scale, np.max(d) / scale
