"""GPU parity of the two accelerations of steady solves against the FP64 oracle:
local pseudo-time steps with mass renormalisation (local_dt) and the half
channel with a symmetry plane at x = 0 (half_channel), alone, together, in
mixed batches and in the pool; and the steady state of the local steps against
that of the global step."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07803_gb300 import build, lbc, workloads
from tests.helpers import gpu_available, moment_errors, weighted_state_error

pytestmark = pytest.mark.gpu

SQ2 = math.sqrt(2.0)

LTS = dict(Nx=70, Qx=5, Qy=6, stretch_A=0.95, delta=0.4, u_left=-0.2, u_right=0.25, T_left=0.7, T_right=1.4,
           omega=0.7, local_dt=1)
HALF = dict(Nx=45, Qx=6, Qy=5, stretch_A=0.98, delta=1.5, u_left=-0.3 * SQ2, u_right=0.3 * SQ2, T_left=1.2,
            T_right=1.2, half_channel=1)
HALF_ONE_TILE = dict(Nx=16, Qx=7, Qy=7, Nexp_x=6, Nexp_y=6, stretch_A=0.98, delta=10.0, u_left=-SQ2,
                     u_right=SQ2, omega=0.66, half_channel=1)
BOTH = dict(HALF, Nx=38, delta=0.3, local_dt=1)
PLAIN = dict(Nx=50, Qx=4, Qy=5, stretch_A=0.9, delta=1.0, u_left=-0.1, u_right=0.2, T_left=0.9, T_right=1.1)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


def check(moments, o, tol, tag):
    e = moment_errors(moments, o.moments())
    assert np.all(e < tol), (tag, dict(zip(lbc.MOMENT_NAMES, e)))


@pytest.mark.parametrize("case", ["lts", "half", "half_one_tile", "both"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_single_solver_matches_oracle(case, precision, tol):
    p = dict(dict(lts=LTS, half=HALF, half_one_tile=HALF_ONE_TILE, both=BOTH)[case], precision=precision)
    s, o = lbc.Solver(p), Oracle(p)
    assert s.dt == pytest.approx(o.dt, rel=1e-14)
    for k in (1, 30):
        s.step(k)
        o.run(k)
        check(s.moments(), o, tol, (case, k))
    assert weighted_state_error(s.get_state(), o.f, o.w) < tol
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_local_steps_from_an_installed_state(precision, tol):
    """set_state makes the installed state's mass the one the iteration keeps."""
    p = dict(LTS, precision=precision)
    s, o = lbc.Solver(p), Oracle(p)
    f = workloads.perturbed_state(s.V, s.Nx, s.get_state(), seed=3, amplitude=0.05)
    s.set_state(f)
    o.set_state(f)
    s.step(40)
    o.run(40)
    check(s.moments(), o, tol, "installed")
    m = s.moments()[0]
    assert abs(np.sum(o.J * o.deta * m) - o.total_mass()) < 1e-6
    s.close()


def test_mixed_batch_matches_oracle():
    """Plain, local-step, half-channel and both kinds of instances in one batch (FP64)."""
    ps = [PLAIN, LTS, HALF, BOTH, HALF_ONE_TILE]
    b = lbc.Batch(ps)
    b.step(20)
    for i, p in enumerate(ps):
        o = Oracle(p)
        o.run(20)
        check(b.moments(i), o, 1e-12, i)
    b.close()


@pytest.mark.parametrize("cluster", [2, 8])
def test_same_result_alone_and_in_the_mix(cluster):
    ps = [dict(p, precision="fp32") for p in (LTS, HALF, BOTH, PLAIN)]
    b = lbc.Batch(ps, cluster=cluster)
    states = []
    for i in range(len(ps)):
        f = workloads.perturbed_state(b.V[i], b.Nx[i], b.get_state(i), seed=40 + i, amplitude=0.05)
        b.set_state(i, f)
        states.append(f)
    b.step(70)
    for i, p in enumerate(ps[:3]):
        a = lbc.Batch([p, PLAIN | dict(precision="fp32")], cluster=cluster)
        a.set_state(0, states[i])
        a.step(70)
        assert np.array_equal(a.get_state(0), b.get_state(i)), i
        a.close()
    b.close()


def test_local_steps_reach_the_global_steady_state():
    """FP64: the local-step iteration stops at the global step's steady state, in
    fewer steps, and at the oracle's stopping step."""
    p = dict(Nx=40, Qx=4, Qy=4, stretch_A=0.95, delta=0.3, u_left=-0.1, u_right=0.15, T_left=0.8, T_right=1.2)
    g, l = lbc.Solver(p), lbc.Solver(dict(p, local_dt=1))
    kg, _ = g.run_to_steady(1e-12, 400000)
    kl, _ = l.run_to_steady(1e-12, 400000)
    assert kl < kg / 2, (kl, kg)
    e = moment_errors(l.moments(), g.moments())   # both within their distance to the limit
    assert np.all(e < 2e-7), dict(zip(lbc.MOMENT_NAMES, e))
    o = Oracle(dict(p, local_dt=1))
    ko, _ = o.run_to_steady(1e-12, 400000)
    assert abs(ko - kl) <= 1, (ko, kl)
    check(l.moments(), o, 1e-10, "steady")
    g.close()
    l.close()


def test_pooled_local_step_and_half_channel_instances():
    pool = lbc.Pool(cluster=4, precision="fp64", budget_bytes=1 << 30)
    ps = [LTS, HALF, PLAIN]
    slots = [pool.try_add(p) for p in ps]
    assert pool.run(1e-30, 25) == []
    for slot, p in zip(slots, ps):
        o = Oracle(p)
        o.run(25)
        check(pool.moments(slot), o, 1e-12, slot)
    pool.close()
