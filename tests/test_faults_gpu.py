"""Failure paths, made on the host or by a bounded device wait; nothing here
faults, traps or hangs the GPU.

LBC_FAULT (read by the library at each use) makes the allocation, launch and
admission wrappers report failure without calling CUDA, and "wait:N" makes every
stage CTA wait at most N polls on an mbarrier that nothing arrives at: the
kernel's bounded-wait path records the timeout, waits for the copies it issued
and returns, and the host reports LBC_ETIMEOUT. Each test checks the status,
that the failed call changed nothing it should not, and that the context stays
usable afterwards."""
import numpy as np
import pytest

from paper_1810_07803_gb300 import build, lbc, workloads
from tests.helpers import gpu_available

pytestmark = pytest.mark.gpu

SMALL = dict(workloads.c1(), Nx=40)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bounded_wait_gives_up_and_reports(monkeypatch, precision):
    p = dict(SMALL, precision=precision)
    ref = lbc.Solver(p)
    ref.step(5)
    s = lbc.Solver(p)
    rest = s.get_state()
    monkeypatch.setenv("LBC_FAULT", "wait:64")
    with pytest.raises(lbc.LbcError) as e:
        s.run_to_steady(1e-10, 10)
    assert e.value.status == lbc.ETIMEOUT
    monkeypatch.delenv("LBC_FAULT")
    with pytest.raises(lbc.LbcError) as e:   # refused until a state is installed
        s.step(1)
    assert e.value.status == lbc.ETIMEOUT
    s.set_state(rest)
    s.step(5)
    assert np.array_equal(s.get_state(), ref.get_state())
    s.close()
    ref.close()


def test_bounded_wait_in_a_batch(monkeypatch):
    ps = [dict(SMALL, delta=d, precision="fp32") for d in (0.5, 2.0)]
    b = lbc.Batch(ps)
    rest = [b.get_state(i) for i in range(len(ps))]
    monkeypatch.setenv("LBC_FAULT", "wait:16")
    with pytest.raises(lbc.LbcError) as e:
        b.run_to_steady(1e-10, 5)
    assert e.value.status == lbc.ETIMEOUT
    monkeypatch.delenv("LBC_FAULT")
    b.set_states(rest)
    b.step(3)
    ref = lbc.Batch(ps)
    ref.step(3)
    for i in range(len(ps)):
        assert np.array_equal(b.get_state(i), ref.get_state(i))
    b.close()
    ref.close()


@pytest.mark.parametrize("kind", ["solver", "batch"])
def test_injected_bounds_flag_reports_and_halts(monkeypatch, kind):
    """LBC_FAULT=bounds:S uploads control blocks that carry a failed-check site, as a range
    check of the checked build records it: the next read reports LBC_EBOUNDS naming the
    site, stepping is refused until a state is installed, and the results then continue
    bit for bit."""
    ps = [dict(SMALL, precision="fp32"), dict(SMALL, delta=2.0, precision="fp32")]
    make = (lambda: lbc.Solver(ps[0])) if kind == "solver" else (lambda: lbc.Batch(ps))
    ref = make()
    ref.step(4)
    b = make()
    rest = b.get_state() if kind == "solver" else [b.get_state(i) for i in range(2)]
    monkeypatch.setenv("LBC_FAULT", "bounds:5")
    with pytest.raises(lbc.LbcError) as e:
        b.run_to_steady(1e-10, 5)
    assert e.value.status == lbc.EBOUNDS
    assert "state store" in str(e.value)
    monkeypatch.delenv("LBC_FAULT")
    with pytest.raises(lbc.LbcError) as e:   # refused until a state is installed
        b.step(1)
    assert e.value.status == lbc.EBOUNDS
    if kind == "solver":
        b.set_state(rest)
        b.step(4)
        assert np.array_equal(b.get_state(), ref.get_state())
    else:
        b.set_states(rest)
        b.step(4)
        for i in range(2):
            assert np.array_equal(b.get_state(i), ref.get_state(i))
    b.close()
    ref.close()


def test_injected_allocation_failure(monkeypatch):
    monkeypatch.setenv("LBC_FAULT", "alloc")
    with pytest.raises(lbc.LbcError) as e:
        lbc.Solver(SMALL)
    assert e.value.status == lbc.ENOMEM
    monkeypatch.delenv("LBC_FAULT")
    with lbc.Solver(SMALL) as s:
        s.step(2)
        assert np.all(np.isfinite(s.moments()))


def test_injected_launch_failure_leaves_the_solver_unchanged(monkeypatch):
    ref = lbc.Solver(SMALL)
    ref.step(70)
    s = lbc.Solver(SMALL)
    monkeypatch.setenv("LBC_FAULT", "launch")
    for n in (3, 70):   # eager launches and a captured group
        with pytest.raises(lbc.LbcError) as e:
            s.step(n)
        assert e.value.status == lbc.ECUDA
    assert s.steps == 0
    monkeypatch.delenv("LBC_FAULT")
    s.step(70)
    assert s.steps == 70
    assert np.array_equal(s.get_state(), ref.get_state())
    s.close()
    ref.close()


def test_injected_admission_refusal_queues(monkeypatch):
    pool = lbc.Pool(cluster=1, precision="fp32", budget_bytes=1 << 30, max_instances=4, max_tiles=64)
    monkeypatch.setenv("LBC_FAULT", "admit")
    assert pool.try_add(SMALL) is None
    assert pool.usage()[1] == 0
    monkeypatch.delenv("LBC_FAULT")
    slot = pool.try_add(SMALL)
    assert slot is not None
    monkeypatch.setenv("LBC_FAULT", "launch")
    with pytest.raises(lbc.LbcError) as e:
        pool.run(1e-8, 4)
    assert e.value.status == lbc.ECUDA
    monkeypatch.delenv("LBC_FAULT")
    pool.run(1e-8, 4)
    assert pool.info(slot)[3] == 4
    pool.close()


@pytest.mark.parametrize("form", [1, 3])
def test_bounded_wait_in_the_solo_and_split_forms(monkeypatch, form):
    """A timed-out stage in the solo form still counts its CTAs in, so the tiles' counts stay
    consistent; in the split form the node-step launch runs on whatever the stage left. Either
    way, after a state is installed the batch continues bit for bit."""
    ps = [dict(SMALL, delta=d, precision="fp32") for d in (0.5, 2.0)]
    b = lbc.Batch(ps, cluster=2)
    b.set_form(form)
    rest = [b.get_state(i) for i in range(len(ps))]
    monkeypatch.setenv("LBC_FAULT", "wait:16")
    with pytest.raises(lbc.LbcError) as e:
        b.run_to_steady(1e-10, 5)
    assert e.value.status == lbc.ETIMEOUT
    monkeypatch.delenv("LBC_FAULT")
    b.set_states(rest)
    b.step(3)
    ref = lbc.Batch(ps, cluster=2)
    ref.set_form(form)
    ref.step(3)
    for i in range(len(ps)):
        assert np.array_equal(b.get_state(i), ref.get_state(i))
    b.close()
    ref.close()
