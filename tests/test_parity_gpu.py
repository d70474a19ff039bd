"""GPU parity: the CUDA path through the C ABI against the FP64 oracle,
element by element on the same seeded inputs.

Tolerances: FP64 state 1e-12 on every moment (normalised as in
helpers.moment_errors); FP32 state 1e-5. Sizes span several 32-node tiles,
ragged last tiles (Nx = 65, 66, 72), more than one velocity chunk (V >= 128),
stretched grids, non-isothermal walls, p0 != 1 and delta = 0.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07803_gb300 import build, lbc, workloads
from tests.helpers import gpu_available, moment_errors, weighted_state_error

pytestmark = pytest.mark.gpu

SQ2 = math.sqrt(2.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


CASES = {
    "c1": workloads.c1(),
    "ragged65_stretched": dict(Nx=65, Qx=5, Qy=6, stretch_A=math.sqrt(0.9), delta=2.0, u_left=-0.1, u_right=0.2,
                               T_left=0.8, T_right=1.25, omega=0.7, Pr=0.68),
    "ragged66_p0": dict(Nx=66, Qx=6, Qy=5, p0=1.2, delta=0.4, u_left=0.05, u_right=-0.15, T_left=1.1, T_right=0.9),
    "chunks_V160": dict(Nx=72, Qx=8, Qy=10, stretch_A=0.7, delta=5.0, u_left=-0.3, u_right=0.3, T_left=0.6,
                        T_right=1.4, omega=0.6),
    "collisionless": dict(Nx=40, Qx=4, Qy=5, delta=0.0, u_left=-0.2, u_right=0.1, T_left=1.2, T_right=0.7),
    "low_order": dict(Nx=48, Qx=7, Qy=7, Nexp_x=3, Nexp_y=4, delta=1.0, u_left=-0.1, u_right=0.1),
}


def run_pair(params, nsteps, precision="fp64", state=None):
    p = dict(params)
    p["precision"] = precision
    s = lbc.Solver(p)
    o = Oracle(p)
    assert s.dt == pytest.approx(o.dt, rel=1e-14)
    if state is not None:
        s.set_state(state)
        o.set_state(state)
    s.step(nsteps)
    o.run(nsteps)
    return s, o


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nsteps", [1, 10, 100])
def test_fp64_parity_fixed_steps(name, nsteps):
    s, o = run_pair(CASES[name], nsteps)
    e = moment_errors(s.moments(), o.moments())
    assert np.all(e < 1e-12), dict(zip(lbc.MOMENT_NAMES, e))
    assert weighted_state_error(s.get_state(), o.f, o.w) < 1e-12
    s.close()


def test_fp64_parity_1000_steps_c1():
    s, o = run_pair(CASES["c1"], 1000)
    e = moment_errors(s.moments(), o.moments())
    assert np.all(e < 1e-12), dict(zip(lbc.MOMENT_NAMES, e))
    s.close()


@pytest.mark.parametrize("name", ["c1", "ragged65_stretched", "chunks_V160"])
def test_fp64_parity_from_perturbed_state(name):
    """A seeded smooth perturbation exercises the nonlinear WENO weights, the
    Shakhov heat-flux factor and non-trivial wall fluxes from the first step."""
    p = CASES[name]
    o = Oracle(p)
    f = workloads.perturbed_state(o.V, o.Nx, o.f, seed=11, amplitude=0.2)
    s, o = run_pair(p, 20, state=f)
    e = moment_errors(s.moments(), o.moments())
    assert np.all(e < 1e-12), dict(zip(lbc.MOMENT_NAMES, e))
    s.close()


@pytest.mark.parametrize("name", ["c1", "ragged65_stretched", "chunks_V160", "collisionless"])
@pytest.mark.parametrize("nsteps", [1, 50])
def test_fp32_parity_fixed_steps(name, nsteps):
    s, o = run_pair(CASES[name], nsteps, precision="fp32")
    e = moment_errors(s.moments(), o.moments())
    assert np.all(e < 1e-5), dict(zip(lbc.MOMENT_NAMES, e))
    s.close()


def test_run_to_steady_c1():
    """Config 1 to max|df| < 1e-10: same stopping step (+-1) and steady moments."""
    p = CASES["c1"]
    s = lbc.Solver(p)
    o = Oracle(p)
    ks, rs = s.run_to_steady(1e-10, 100000)
    ko, ro = o.run_to_steady(1e-10, 100000)
    assert abs(ks - ko) <= 1
    assert rs < 1e-10
    e = moment_errors(s.moments(), o.moments())
    assert np.all(e < 1e-11), dict(zip(lbc.MOMENT_NAMES, e))
    assert s.steps == ks
    s.close()


def test_run_to_steady_reports_not_converged():
    s = lbc.Solver(CASES["c1"])
    with pytest.raises(lbc.LbcError) as e:
        s.run_to_steady(1e-14, 70)
    assert e.value.status == lbc.ENOTCONV
    assert s.steps == 70
    s.close()


def test_graph_and_eager_steps_agree():
    """lbc_step uses CUDA graphs for groups of 64 steps: 130 steps in one call
    equal 130 single-step calls bit for bit."""
    p = CASES["ragged65_stretched"]
    a = lbc.Solver(p)
    b = lbc.Solver(p)
    a.step(130)
    for _ in range(130):
        b.step(1)
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.steps == b.steps == 130
    a.close()
    b.close()


def test_mass_conservation_on_gpu():
    p = dict(CASES["chunks_V160"])
    s = lbc.Solver(p)
    o = Oracle(p)
    m0 = np.sum(o.J * o.deta * s.moments()[0])
    s.step(300)
    m1 = np.sum(o.J * o.deta * s.moments()[0])
    assert abs(m1 - m0) < 1e-13
    s.close()


def test_rest_state_is_fixed_point_on_gpu():
    for prec in ("fp64", "fp32"):
        s = lbc.Solver(dict(Nx=70, Qx=6, Qy=6, stretch_A=0.8, delta=3.0, precision=prec))
        f0 = s.get_state()
        s.step(25)
        tol = 1e-13 if prec == "fp64" else 1e-6
        assert np.max(np.abs(s.get_state() - f0)) < tol
        s.close()


def test_set_state_roundtrip_and_nonfinite_rejected():
    s = lbc.Solver(dict(Nx=33, Qx=4, Qy=4))
    f = workloads.perturbed_state(s.V, s.Nx, s.get_state(), seed=5)
    s.set_state(f)
    assert np.array_equal(s.get_state(), f)
    f[0, 3, 7] = np.nan
    with pytest.raises(lbc.LbcError) as e:
        s.set_state(f)
    assert e.value.status == lbc.EINVAL
    s.close()


def perturbed(o, seed, amplitude=0.1):
    """A seeded non-equilibrium state of problem o: every velocity row of the rest
    state modulated by its own low Fourier modes in x, so that from the first step
    every node has non-trivial n, u, T, q, the nonlinear WENO weights and the wall
    fluxes are in play, and the moment sums cancel across velocities."""
    return workloads.perturbed_state(o.V, o.Nx, o.f, seed=seed, amplitude=amplitude)


@pytest.mark.parametrize("delta", workloads.C2_DELTAS)
def test_full_size_c2_perturbed(delta):
    """Config 2 at full size (Nx = 2048, 32 x 20 velocities), FP32 state, from a seeded
    perturbed state: 3 steps against the oracle (1e-5)."""
    p = workloads.c2(delta)
    o = Oracle(p)
    s, o = run_pair(p, 3, precision="fp32", state=perturbed(o, seed=20 + int(10 * delta)))
    e = moment_errors(s.moments(), o.moments())
    assert np.all(e < 1e-5), dict(zip(lbc.MOMENT_NAMES, e))
    s.close()


def test_full_size_c2_fp64_perturbed():
    """Config 2 at full size in FP64 from a perturbed state: 3 steps, 1e-12."""
    p = workloads.c2(1.0, precision="fp64")
    o = Oracle(p)
    s, o = run_pair(p, 3, precision="fp64", state=perturbed(o, seed=31))
    e = moment_errors(s.moments(), o.moments())
    assert np.all(e < 1e-12), dict(zip(lbc.MOMENT_NAMES, e))
    assert weighted_state_error(s.get_state(), o.f, o.w) < 1e-12
    s.close()


def test_benchmark_launch_configuration_matches_oracle():
    """The benchmark's exact configuration: the four delta solves of the single-large-solve
    workload as one FP32 batch with the autotuned cluster size, stepped the way the
    benchmark steps them, from seeded perturbed states installed in one call; 3 steps,
    each solve against the oracle (1e-5)."""
    ps = [workloads.c2(d, precision="fp32") for d in workloads.C2_DELTAS]
    b = lbc.Batch(ps)
    b.autotune(2)
    orcs = [Oracle(p) for p in ps]
    states = [perturbed(o, seed=40 + i) for i, o in enumerate(orcs)]
    b.set_states(states)
    b.step(2)
    b.step_timed(1)
    for i, (p, o) in enumerate(zip(ps, orcs)):
        o.set_state(states[i])
        o.run(3)
        e = moment_errors(b.moments(i), o.moments())
        assert np.all(e < 1e-5), (p["delta"], dict(zip(lbc.MOMENT_NAMES, e)))
    b.close()
