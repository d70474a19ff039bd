"""The table viscosity law (Eqs. mun, interp: mu piecewise power law, Pr
piecewise constant) on the GPU against the FP64 oracle, with a seeded synthetic
table spanning the temperatures of non-isothermal walls."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07803_gb300 import build, lbc, workloads
from tests.helpers import gpu_available, moment_errors

pytestmark = pytest.mark.gpu

CASE = dict(Nx=70, Qx=6, Qy=7, stretch_A=math.sqrt(0.9), delta=3.0, u_left=-0.2, u_right=0.25, T_left=0.45,
            T_right=2.3, **workloads.synthetic_viscosity_table(seed=7, n=24))


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


@pytest.mark.parametrize("precision,tol,nsteps", [("fp64", 1e-12, 10), ("fp64", 1e-12, 80), ("fp32", 1e-5, 30)])
def test_table_law_parity(precision, tol, nsteps):
    p = dict(CASE, precision=precision)
    o = Oracle(p)
    s = lbc.Solver(p)
    assert s.dt == pytest.approx(o.dt, rel=1e-14)
    f = workloads.perturbed_state(o.V, o.Nx, o.f, seed=19, amplitude=0.15)
    s.set_state(f)
    o.set_state(f)
    s.step(nsteps)
    o.run(nsteps)
    e = moment_errors(s.moments(), o.moments())
    assert np.all(e < tol), dict(zip(lbc.MOMENT_NAMES, e))
    s.close()


def test_power_law_table_equals_power_law_on_gpu():
    T = np.array([0.3, 0.7, 1.2, 2.8])
    p1 = dict(CASE, mu_law="power", omega=0.66, Pr=0.68)
    p2 = dict(CASE, omega=0.0, tab_T=T, tab_mu=5.0 * T ** 0.66, tab_Pr=np.full(4, 0.68))
    a, b = lbc.Solver(p1), lbc.Solver(p2)
    a.step(40)
    b.step(40)
    fa, fb = a.get_state(), b.get_state()
    assert np.max(np.abs(fa - fb)) <= 1e-12 * np.max(np.abs(fa))
    a.close()
    b.close()


def test_table_and_power_law_instances_in_one_batch():
    ps = [dict(CASE, precision="fp32"), dict(CASE, mu_law="power", omega=0.7, precision="fp32")]
    b = lbc.Batch(ps)
    b.step(20)
    for i, p in enumerate(ps):
        o = Oracle(p)
        o.run(20)
        e = moment_errors(b.moments(i), o.moments())
        assert np.all(e < 1e-5), (i, dict(zip(lbc.MOMENT_NAMES, e)))
    b.close()
