"""The oracle's table viscosity law (Eqs. mun, interp) against what the paper
fixes: on each interval [T_n, T_{n+1}] mu is the power law through both table
points, the end intervals extend beyond the table, Pr is piecewise constant
(Pr_1 below T_2, Pr_n from T_n, Pr_N above T_N), and delta refers to mu(T_ref).
A table sampled from mu = T^omega must therefore reproduce the power-law solver."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07803_gb300 import workloads

BASE = dict(Nx=24, Qx=4, Qy=5, delta=2.0, u_left=-0.2, u_right=0.15, T_left=0.6, T_right=1.7, Pr=0.7,
            stretch_A=0.8)


def table_from_power_law(omega, T, scale=3.7, Pr=0.7):
    T = np.asarray(T, dtype=float)
    return dict(mu_law="table", tab_T=T, tab_mu=scale * T ** omega, tab_Pr=np.full(len(T), Pr))


@pytest.mark.parametrize("T", [[0.9, 1.2], [0.3, 0.8, 1.1, 2.5], [1.5, 2.0, 4.0]])
def test_table_sampled_from_a_power_law_reproduces_it(T):
    """Any table of mu = c T^omega (here also not containing T_ref = 1, so the end
    segments extrapolate) gives the power-law step to rounding."""
    o1 = Oracle(dict(BASE, omega=0.72))
    o2 = Oracle(dict(BASE, omega=0.0, **table_from_power_law(0.72, T)))
    assert o2.dt == pytest.approx(o1.dt, rel=1e-14)
    f = workloads.perturbed_state(o1.V, o1.Nx, o1.f, seed=3, amplitude=0.2)
    o1.set_state(f)
    o2.set_state(f)
    o1.run(15)
    o2.run(15)
    assert np.max(np.abs(o2.f - o1.f)) <= 1e-13 * np.max(np.abs(o1.f))


def test_mu_is_the_segment_power_law_and_continuous():
    tab = workloads.synthetic_viscosity_table(seed=11, n=9)
    o = Oracle(dict(BASE, **tab))
    T, mu = tab["tab_T"], tab["tab_mu"]
    mu_ref = None
    for k in range(len(T) - 1):   # the segment holding T = 1 defines mu(T_ref)
        if T[k] <= 1.0 < T[k + 1] or (k == 0 and 1.0 < T[0]) or (k == len(T) - 2 and 1.0 >= T[-1]):
            w = math.log(mu[k + 1] / mu[k]) / math.log(T[k + 1] / T[k])
            mu_ref = mu[k] * (1.0 / T[k]) ** w
    assert mu_ref is not None
    for k in range(len(T)):       # table points: the table value (continuity at the joints)
        assert o.mu_ratio(T[k]) * mu_ref == pytest.approx(mu[k], rel=1e-13)
    for k in range(len(T) - 1):   # interior points: the power law of their own segment
        w = math.log(mu[k + 1] / mu[k]) / math.log(T[k + 1] / T[k])
        t = math.sqrt(T[k] * T[k + 1])
        assert o.mu_ratio(t) * mu_ref == pytest.approx(mu[k] * (t / T[k]) ** w, rel=1e-13)
    w0 = math.log(mu[1] / mu[0]) / math.log(T[1] / T[0])
    wN = math.log(mu[-1] / mu[-2]) / math.log(T[-1] / T[-2])
    assert o.mu_ratio(0.5 * T[0]) * mu_ref == pytest.approx(mu[0] * 0.5 ** w0, rel=1e-13)
    assert o.mu_ratio(3.0 * T[-1]) * mu_ref == pytest.approx(mu[-1] * 3.0 ** wN, rel=1e-13)
    assert o.mu_ratio(1.0) == pytest.approx(1.0, rel=1e-15)


def test_prandtl_is_piecewise_constant_as_printed():
    tab = dict(mu_law="table", tab_T=np.array([0.5, 1.0, 2.0, 4.0]), tab_mu=np.array([1.0, 1.6, 2.6, 4.1]),
               tab_Pr=np.array([0.60, 0.62, 0.64, 0.66]))
    o = Oracle(dict(BASE, **tab))
    assert o.prandtl(0.1) == 0.60 and o.prandtl(0.99) == 0.60      # Pr_1 below T_2
    assert o.prandtl(1.0) == 0.62 and o.prandtl(1.99) == 0.62      # Pr_2 on [T_2, T_3)
    assert o.prandtl(2.0) == 0.64 and o.prandtl(3.9) == 0.64
    assert o.prandtl(4.0) == 0.66 and o.prandtl(50.0) == 0.66      # Pr_N from T_N on


def test_delta_refers_to_mu_at_the_reference_temperature():
    """Scaling every tabulated mu by a constant changes nothing: the relaxation
    time uses mu(T)/mu(T_ref) with delta defined at T_ref."""
    tab = workloads.synthetic_viscosity_table(seed=5, n=12)
    o1 = Oracle(dict(BASE, **tab))
    o2 = Oracle(dict(BASE, **dict(tab, tab_mu=tab["tab_mu"] * 123.0)))
    o1.run(10)
    o2.run(10)
    assert np.max(np.abs(o2.f - o1.f)) <= 1e-14 * np.max(np.abs(o1.f))


def test_variable_prandtl_changes_the_heat_flux_relaxation():
    """With Pr(T) taken per node, a table whose Pr differs from the constant one
    changes the solution (the law is actually used), mass stays conserved."""
    tab = table_from_power_law(0.72, [0.3, 0.8, 1.1, 2.5], Pr=0.7)
    tab2 = dict(tab, tab_Pr=np.array([0.55, 0.6, 0.75, 0.8]))
    o1 = Oracle(dict(BASE, **tab))
    o2 = Oracle(dict(BASE, **tab2))
    f = workloads.perturbed_state(o1.V, o1.Nx, o1.f, seed=8, amplitude=0.2)
    o1.set_state(f)
    o2.set_state(f)
    m0 = o2.total_mass()
    o1.run(20)
    o2.run(20)
    assert np.max(np.abs(o2.f - o1.f)) > 1e-6
    assert o2.total_mass() == pytest.approx(m0, rel=1e-13)
