"""Batches of uneven instances in one stage launch (lbc_batch_*): every
instance against the FP64 oracle, and the same result alone and in the mix.

"Alone" is a batch of one instance with the mix's cluster size forced, so its
velocity chunks (and with them the order of every floating-point sum) are those
the instance has in the mix: results must then agree bit for bit. Against the
oracle the tolerances are those of the single-solver parity tests.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07803_gb300 import build, lbc, workloads
from tests.helpers import gpu_available, moment_errors

pytestmark = pytest.mark.gpu

MIX = [
    dict(Nx=64, Qx=4, Qy=4, delta=1.0, u_left=-0.05 * math.sqrt(2), u_right=0.05 * math.sqrt(2)),
    dict(Nx=65, Qx=5, Qy=6, stretch_A=math.sqrt(0.9), delta=2.0, u_left=-0.1, u_right=0.2, T_left=0.8,
         T_right=1.25, omega=0.7, Pr=0.68),
    dict(Nx=72, Qx=8, Qy=10, stretch_A=0.7, delta=5.0, u_left=-0.3, u_right=0.3, T_left=0.6, T_right=1.4,
         omega=0.6),
    dict(Nx=40, Qx=4, Qy=5, delta=0.0, u_left=-0.2, u_right=0.1, T_left=1.2, T_right=0.7),
    dict(Nx=48, Qx=7, Qy=7, Nexp_x=3, Nexp_y=4, delta=1.0, u_left=-0.1, u_right=0.1),
    dict(Nx=130, Qx=12, Qy=9, stretch_A=0.9, delta=0.3, u_left=0.1, u_right=-0.25, T_left=1.0, T_right=2.0,
         p0=1.1),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


def with_precision(ps, precision):
    return [dict(p, precision=precision) for p in ps]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_mixed_batch_matches_oracle(precision, tol):
    ps = with_precision(MIX, precision)
    b = lbc.Batch(ps)
    b.step(12)
    for i, p in enumerate(ps):
        o = Oracle(p)
        assert b.dt[i] == pytest.approx(o.dt, rel=1e-14)
        o.run(12)
        e = moment_errors(b.moments(i), o.moments())
        assert np.all(e < tol), (i, dict(zip(lbc.MOMENT_NAMES, e)))
        assert b.steps(i) == 12
    b.close()


@pytest.mark.parametrize("cluster", [3, 8, 16])
def test_same_result_alone_and_in_the_mix(cluster):
    """Every instance of a mixed batch equals, bit for bit, its own batch of one
    with the same cluster size; from perturbed states, FP32."""
    ps = with_precision(MIX, "fp32")
    b = lbc.Batch(ps, cluster=cluster)
    assert b.shape()[0] == cluster
    states = []
    for i in range(len(ps)):
        f = workloads.perturbed_state(b.V[i], b.Nx[i], b.get_state(i), seed=100 + i, amplitude=0.1)
        b.set_state(i, f)
        states.append(f)
    b.step(70)   # one graph of 64 steps and 6 eager steps
    for i, p in enumerate(ps):
        a = lbc.Batch([p], cluster=cluster)
        a.set_state(0, states[i])
        a.step(70)
        assert np.array_equal(a.get_state(0), b.get_state(i)), i
        a.close()
    b.close()


def test_small_instance_in_a_wide_cluster():
    """V = 32 velocities in 16 chunk CTAs: most chunks of each tile are empty."""
    p = dict(Nx=95, Qx=4, Qy=4, delta=0.7, u_left=0.1, u_right=-0.1, T_left=1.3, T_right=0.9)
    b = lbc.Batch([p, dict(p, delta=4.0)], cluster=16)
    b.step(10)
    for i, d in enumerate((0.7, 4.0)):
        o = Oracle(dict(p, delta=d))
        o.run(10)
        e = moment_errors(b.moments(i), o.moments())
        assert np.all(e < 1e-12), dict(zip(lbc.MOMENT_NAMES, e))
    b.close()


def test_batch_run_to_steady_per_instance():
    """Each instance stops at its own step; each equals a single solver's run."""
    base = workloads.c1()
    ps = [dict(base, delta=d) for d in (0.5, 1.0, 3.0)]
    b = lbc.Batch(ps)
    ks, rs = b.run_to_steady(1e-9, 100000)
    for i, p in enumerate(ps):
        s = lbc.Solver(p)
        k1, r1 = s.run_to_steady(1e-9, 100000)
        assert abs(ks[i] - k1) <= 1, (i, ks[i], k1)
        assert rs[i] < 1e-9
        assert b.steps(i) == ks[i]
        e = moment_errors(b.moments(i), s.moments())
        assert np.all(e < 1e-9), dict(zip(lbc.MOMENT_NAMES, e))
        s.close()
    assert len(set(ks)) > 1   # different rarefaction, different stopping steps
    b.step(3)                 # plain stepping after a run-to-steady call
    assert [b.steps(i) for i in range(3)] == [k + 3 for k in ks]
    b.close()


def test_batch_not_converged_reports_each_instance():
    ps = [workloads.c1(), dict(workloads.c1(), delta=2.0)]
    b = lbc.Batch(ps)
    ks, rs = b.run_to_steady(1e-15, 80, raise_notconv=False)
    assert ks == [80, 80]
    assert all(r > 1e-15 for r in rs)
    b.close()


def test_set_state_touches_one_instance():
    ps = MIX[:3]
    b = lbc.Batch(ps)
    before = [b.get_state(i) for i in range(3)]
    f = workloads.perturbed_state(b.V[1], b.Nx[1], before[1], seed=9)
    b.set_state(1, f)
    assert np.array_equal(b.get_state(1), f)
    assert np.array_equal(b.get_state(0), before[0])
    assert np.array_equal(b.get_state(2), before[2])
    b.close()


def test_autotune_picks_a_shape_and_restores_rest():
    ps = with_precision(MIX, "fp32")
    b = lbc.Batch(ps)
    rest = [b.get_state(i) for i in range(len(ps))]
    c = b.autotune(2)
    assert 1 <= c <= 16 and b.shape()[0] == c
    for i in range(len(ps)):
        assert np.array_equal(b.get_state(i), rest[i])
        assert b.steps(i) == 0
    b.step(5)
    o = Oracle(ps[2])
    o.run(5)
    e = moment_errors(b.moments(2), o.moments())
    assert np.all(e < 1e-5), dict(zip(lbc.MOMENT_NAMES, e))
    b.close()


def test_batch_rejects_mixed_precision_and_names_bad_instance():
    with pytest.raises(lbc.LbcError) as e:
        lbc.Batch([dict(MIX[0], precision="fp32"), dict(MIX[1], precision="fp64")])
    assert e.value.status == lbc.EINVAL
    with pytest.raises(lbc.LbcError) as e:
        lbc.Batch([MIX[0], dict(MIX[1], Qx=0)])
    assert "instance 1" in str(e.value)


def test_set_states_and_moments_all_match_the_single_calls():
    """lbc_batch_set_states / lbc_batch_moments_all do what n single calls do; a
    state with a NaN leaves every instance unchanged."""
    ps = with_precision(MIX[:4], "fp32")
    a, b = lbc.Batch(ps), lbc.Batch(ps)
    fs = [workloads.perturbed_state(a.V[i], a.Nx[i], a.get_state(i), seed=30 + i) for i in range(len(ps))]
    fs[2] = None                                   # instance 2 keeps its state
    for i, f in enumerate(fs):
        if f is not None:
            a.set_state(i, f)
    b.set_states(fs)
    for i in range(len(ps)):
        assert np.array_equal(a.get_state(i), b.get_state(i)), i
    a.step(7)
    b.step(7)
    mall = b.moments_all()
    for i in range(len(ps)):
        assert np.array_equal(mall[i], b.moments(i)), i
        assert np.array_equal(mall[i], a.moments(i)), i
    before = [b.get_state(i) for i in range(len(ps))]
    bad = [f.copy() if f is not None else None for f in fs]
    bad[1][0, 3, 5] = np.nan
    with pytest.raises(lbc.LbcError) as e:
        b.set_states(bad)
    assert e.value.status == lbc.EINVAL
    for i in range(len(ps)):
        assert np.array_equal(b.get_state(i), before[i]), i
    a.close()
    b.close()


def test_set_states_with_local_steps_and_compensated_instances():
    """The batched upload builds most instances' stage data while later copies land;
    local-step instances rebuild theirs (with the mass reference) after the check. Either
    way the instances then step exactly as after single uploads."""
    base = with_precision(MIX[:3], "fp32")
    ps = [dict(base[0], local_dt=1, stretch_A=0.9), dict(base[1], compensated=1), base[2],
          dict(base[0], compensated=1, local_dt=1, stretch_A=0.9)]
    a, b = lbc.Batch(ps), lbc.Batch(ps)
    fs = [workloads.perturbed_state(a.V[i], a.Nx[i], a.get_state(i), seed=50 + i) for i in range(len(ps))]
    for i, f in enumerate(fs):
        a.set_state(i, f)
    b.set_states(fs)
    a.step(9)
    b.step(9)
    for i in range(len(ps)):
        assert np.array_equal(a.get_state(i), b.get_state(i)), i
        assert np.array_equal(a.moments(i), b.moments(i)), i
    a.close()
    b.close()


SQ2 = math.sqrt(2.0)


def extended_mix(precision):
    """The mix plus instances of the extended kernel form (local steps, half channel, compensated)."""
    ps = with_precision(MIX, precision) + [
        dict(Nx=40, Qx=5, Qy=5, stretch_A=0.95, delta=0.3, u_left=-0.1, u_right=0.1, local_dt=1, precision=precision),
        dict(Nx=24, Qx=6, Qy=7, stretch_A=0.98, delta=1.0, u_left=-SQ2, u_right=SQ2, half_channel=1, local_dt=1,
             precision=precision)]
    if precision == "fp32":
        ps.append(dict(workloads.c1(), precision="fp32", compensated=1))
    return ps


def assert_same_states(a, b, precision):
    for i in range(a.n):
        x, y = a.get_state(i), b.get_state(i)
        if precision == "fp64":
            assert np.max(np.abs(x - y)) <= 1e-14 * np.max(np.abs(x)), i
        else:
            assert np.array_equal(x, y), i
        assert a.steps(i) == b.steps(i)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("cluster", [1, 3, 5])
@pytest.mark.parametrize("form", [1, 3])
def test_solo_and_split_forms_equal_cluster_form(precision, cluster, form):
    """The solo form (independent chunk CTAs; the tile's last CTA sums the chunk partials from
    device memory and builds the node data) and the split form (a second launch builds every
    tile's node data) compute the cluster form's sums in the same order: bit for bit in FP32;
    the FP64 node arithmetic is compiled separately in each form (the compiler may fuse its
    multiply-adds differently), compared to 1e-14 relative."""
    for ps in (with_precision(MIX, precision), extended_mix(precision)):
        a = lbc.Batch(ps, cluster=cluster)
        a.set_form(False)
        b = lbc.Batch(ps, cluster=cluster)
        b.set_form(form)
        assert not a.solo and b.form == form
        for n in (1, 2, 64, 5):   # eager launches and a captured group of 64 steps
            a.step(n)
            b.step(n)
        assert_same_states(a, b, precision)
        a.close()
        b.close()


@pytest.mark.parametrize("form", [1, 3])
def test_solo_and_split_forms_run_to_steady_match_cluster_form(form):
    ps = [dict(workloads.c1(), delta=d) for d in (0.5, 3.0)] + with_precision(MIX[:2], "fp64")
    a = lbc.Batch(ps, cluster=2)
    a.set_form(False)
    b = lbc.Batch(ps, cluster=2)
    b.set_form(form)
    ka, ra = a.run_to_steady(1e-9, 20000, raise_notconv=False)
    kb, rb = b.run_to_steady(1e-9, 20000, raise_notconv=False)
    assert list(ka) == list(kb)
    np.testing.assert_allclose(np.asarray(rb), np.asarray(ra), rtol=1e-9)
    assert_same_states(a, b, "fp64")
    a.close()
    b.close()


def test_forms_at_the_benchmark_size():
    """Four C2 solves (the benchmark's batch, which fills the device: the default is the solo
    form) from a perturbed state, three steps in the solo, split and cluster forms: bit for bit."""
    ps = [workloads.c2(d, precision="fp32") for d in workloads.C2_DELTAS]
    a = lbc.Batch(ps, cluster=3)
    assert a.solo
    states = [workloads.perturbed_state(a.V[i], a.Nx[i], a.get_state(i), seed=7 + i) for i in range(a.n)]
    a.set_states(states)
    a.step(3)
    for form in (0, 3):
        b = lbc.Batch(ps, cluster=3)
        b.set_form(form)
        b.set_states(states)
        b.step(3)
        assert_same_states(a, b, "fp32")
        b.close()
    a.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("form", [2, 4])
def test_full_chunk_forms_match_oracle(precision, tol, form):
    """The solo form with 256-row chunks (form 2: each instance's last chunk shorter, empty
    chunk CTAs where an instance has fewer chunks than the batch): every instance against the
    oracle, including one whose velocity set spans two chunks (320 rows: 256 + 64)."""
    ps = with_precision(MIX, precision) + [
        dict(Nx=80, Qx=16, Qy=10, stretch_A=0.9, delta=1.5, u_left=-0.2, u_right=0.1, T_left=0.9, T_right=1.2,
             precision=precision)]
    b = lbc.Batch(ps)
    b.set_form(form)
    assert b.form == form and b.shape()[0] == 2
    b.step(12)
    for i, p in enumerate(ps):
        o = Oracle(p)
        o.run(12)
        e = moment_errors(b.moments(i), o.moments())
        assert np.all(e < tol), (i, dict(zip(lbc.MOMENT_NAMES, e)))
    b.close()
