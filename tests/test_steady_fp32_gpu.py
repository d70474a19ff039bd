"""FP32 steady states against the FP64 oracle's steady state.

The stated tolerance for reduced-precision runs is 1e-5 on every moment
(normalised as in helpers.moment_errors). A steady state is the fixed point of
the step, so each run is compared with the limit, not with another run that
stopped at the same residual: the oracle and a GPU FP64 run go to r < 1e-14
(these problems contract by ~0.4 % per step, so a run stopped at r is about
r / 0.004 from the limit in the state), and the FP32 runs to r < 1e-10 or,
where the FP32 evaluation of the right-hand side keeps the residual above that,
for a fixed number of steps past the point where the state stops changing.

The compensated FP32 state (each value carries its rounding remainder) is the
form whose steady state meets the tolerance; the plain FP32 state stalls once
the step's increments fall below half an ulp of the values, at a steady state
biased by about eps_32 |f| tau / dt, and its error is measured and bounded here
so that a regression shows.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07803_gb300 import build, lbc, workloads
from tests.helpers import gpu_available, moment_errors

pytestmark = pytest.mark.gpu

CASES = {
    "c1": workloads.c1(),
    # stretched grid, unequal wall temperatures and speeds, local pseudo-time steps
    "stretched_nonisothermal": dict(Nx=48, Qx=6, Qy=6, stretch_A=0.9, delta=2.0, u_left=-0.2, u_right=0.15,
                                    T_left=0.7, T_right=1.4, omega=0.7, Pr=0.68, local_dt=1),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


_refs = {}


def oracle_steady(name):
    if name not in _refs:
        o = Oracle(CASES[name])
        k, r = o.run_to_steady(1e-14, 400000)
        assert r < 1e-14
        _refs[name] = (k, o.moments())
    return _refs[name]


def run_fp32(params, compensated, k_ref):
    """FP32 run to r < 1e-10, or 3 k_ref steps if the residual stays above it."""
    s = lbc.Solver(dict(params, precision="fp32", compensated=int(compensated)))
    try:
        s.run_to_steady(1e-10, 3 * k_ref)
    except lbc.LbcError as e:
        assert e.status == lbc.ENOTCONV
    return s


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_steady_state_matches_oracle(name):
    k, ref = oracle_steady(name)
    s = lbc.Solver(dict(CASES[name], precision="fp64"))
    s.run_to_steady(1e-14, 4 * k)
    e = moment_errors(s.moments(), ref)
    assert np.all(e < 1e-9), dict(zip(lbc.MOMENT_NAMES, e))
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_compensated_steady_state_matches_oracle(name):
    k, ref = oracle_steady(name)
    s = run_fp32(CASES[name], True, k)
    m = s.moments()
    e = moment_errors(m, ref)
    assert np.all(e < 1e-5), dict(zip(lbc.MOMENT_NAMES, e))
    s64 = lbc.Solver(dict(CASES[name], precision="fp64"))
    s64.run_to_steady(1e-14, 4 * k)
    e64 = moment_errors(m, s64.moments())
    assert np.all(e64 < 1e-5), dict(zip(lbc.MOMENT_NAMES, e64))
    s.close()
    s64.close()


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_plain_steady_state_error_bounded(name):
    """The plain FP32 state's stalled steady state: within 1e-3 of the limit (a bound
    on the measured bias, not the reduced-precision tolerance)."""
    k, ref = oracle_steady(name)
    s = run_fp32(CASES[name], False, k)
    e = moment_errors(s.moments(), ref)
    assert np.all(e < 1e-3), dict(zip(lbc.MOMENT_NAMES, e))
    s.close()


# ---- the stall rule (lbc_set_stall_window) ----

STALL_WINDOW = 2048   # residual samples every 64 steps: 32 samples per window


@pytest.mark.parametrize("name", list(CASES))
def test_stall_rule_ends_compensated_fp32_within_tolerance(name):
    """Run to an unreachable threshold with the stall rule: the run ends with ESTALLED long
    before max_steps, at a state still within 1e-5 of the limit."""
    k, ref = oracle_steady(name)
    s = lbc.Solver(dict(CASES[name], precision="fp32", compensated=1))
    s.set_stall_window(STALL_WINDOW)
    with pytest.raises(lbc.LbcError) as e:
        s.run_to_steady(1e-14, 3 * k)
    assert e.value.status == lbc.ESTALLED
    taken = s.steps
    assert 0 < taken < 3 * k and taken % 64 == 0, taken
    err = moment_errors(s.moments(), ref)
    assert np.all(err < 1e-5), dict(zip(lbc.MOMENT_NAMES, err))
    s.close()


def test_stall_rule_leaves_converging_fp64_run_alone():
    """A contracting FP64 run stops where it stops without the rule (same step, same residual)."""
    p = dict(CASES["stretched_nonisothermal"], precision="fp64")
    plain = lbc.Solver(p)
    k0, r0 = plain.run_to_steady(1e-12, 200_000)
    ruled = lbc.Solver(p)
    ruled.set_stall_window(STALL_WINDOW)
    k1, r1 = ruled.run_to_steady(1e-12, 200_000)
    assert (k1, r1) == (k0, r0)
    assert np.array_equal(ruled.get_state(), plain.get_state())
    plain.close()
    ruled.close()


def test_stall_rule_in_a_batch_stops_each_instance_at_its_sample():
    """FP32 batch: each instance stalls at its own step; its stalled state is bit for bit the
    same batch's after the reported number of plain steps, its reported residual is at or
    above the threshold; with a threshold above the FP32 noise every instance converges,
    sooner, and nothing stalls."""
    params = [dict(workloads.c1(), precision="fp32"),
              dict(CASES["stretched_nonisothermal"], precision="fp32"),
              dict(workloads.c1(), precision="fp32", delta=3.0, Nx=40)]
    b = lbc.Batch(params, cluster=1)
    b.set_stall_window(STALL_WINDOW)
    ks, rs = b.run_to_steady(1e-14, 150_000, raise_notconv=False)
    ref = lbc.Batch(params, cluster=1)
    done = 0
    for i in sorted(range(len(params)), key=lambda j: ks[j]):
        assert 0 < ks[i] < 150_000 and ks[i] % 64 == 0, ks
        assert rs[i] >= 1e-14
        ref.step(ks[i] - done)
        done = ks[i]
        assert np.array_equal(b.get_state(i), ref.get_state(i)), (i, ks)
    ref.close()
    with pytest.raises(lbc.LbcError) as e:
        b.run_to_steady(1e-14, 150_000)
    assert e.value.status == lbc.ESTALLED
    # a threshold above the FP32 noise floor: every instance converges, no stall
    b2 = lbc.Batch(params, cluster=1)
    b2.set_stall_window(STALL_WINDOW)
    ks2, rs2 = b2.run_to_steady(1e-7, 150_000)
    assert all(r < 1e-7 for r in rs2) and all(k2 < k for k2, k in zip(ks2, ks))
    b.close()
    b2.close()


def test_stall_window_argument_checked():
    with lbc.Solver(dict(workloads.c1(), precision="fp32")) as s:
        with pytest.raises(lbc.LbcError) as e:
            s.set_stall_window(-1)
        assert e.value.status == lbc.EINVAL
        s.set_stall_window(0)
