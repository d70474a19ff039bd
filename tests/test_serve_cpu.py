"""Host logic of the serving loop with a fake pool (no GPU): Poisson arrivals,
FIFO admission limited by memory, requests that arrive while others run join
the next chunk, each leaves at its own convergence, latency bookkeeping."""
import numpy as np
import pytest

from paper_1810_07803_gb300 import serve


class FakePool:
    """Instances converge after a fixed number of steps (their 'work'); the budget
    counts instances."""

    def __init__(self, capacity):
        self.capacity, self.slots, self.log = capacity, {}, []

    def try_add(self, params):
        if len(self.slots) >= self.capacity:
            return None
        slot = min(set(range(self.capacity)) - set(self.slots))
        self.slots[slot] = dict(need=params["work"], steps=0, reported=False, rid=params["rid"])
        self.log.append(("add", params["rid"]))
        return slot

    def run(self, residual, nsteps):
        done = []
        for slot, s in self.slots.items():
            s["steps"] = min(s["need"], s["steps"] + nsteps)
            if s["steps"] >= s["need"] and not s["reported"]:
                s["reported"] = True
                done.append(slot)
        self.log.append(("run", sorted(self.slots[k]["rid"] for k in self.slots)))
        return done

    def info(self, slot):
        s = self.slots[slot]
        return 8, 16, 0.1, s["steps"], 0.0 if s["reported"] else 1.0

    def moments(self, slot):
        return np.zeros((10, 8))

    def remove(self, slot):
        self.log.append(("remove", self.slots.pop(slot)["rid"]))


def test_poisson_arrivals_have_the_rate():
    t = serve.poisson_arrivals(200.0, 50.0, seed=1)
    assert np.all(np.diff(t) > 0) and t[-1] < 50.0
    assert len(t) / 50.0 == pytest.approx(200.0, rel=0.05)
    gaps = np.diff(t)
    assert np.mean(gaps) == pytest.approx(1 / 200.0, rel=0.05)
    assert np.std(gaps) == pytest.approx(np.mean(gaps), rel=0.1)   # exponential: std = mean


def test_trace_is_seeded():
    a, b = serve.make_trace(50.0, 2.0, seed=3), serve.make_trace(50.0, 2.0, seed=3)
    assert [r.params for r in a] == [r.params for r in b]
    assert [r.arrival for r in a] == [r.arrival for r in b]


def test_continuous_batching_admits_fifo_and_retires_each_at_its_step():
    reqs = [serve.Request(k, arr, dict(rid=k, work=w))
            for k, (arr, w) in enumerate([(0, 64), (0, 32), (0, 96), (1.5, 32), (2.5, 32)])]
    pool = FakePool(capacity=2)
    srv = serve.Server(residual=1e-8, chunk=32, pool=pool)
    out = srv.serve(reqs, clock="steps")
    # only two fit: 0 and 1 start; 2 waits for a slot; 3 and 4 join as slots free up
    assert pool.log[:3] == [("add", 0), ("add", 1), ("run", [0, 1])]
    order = [rid for kind, rid in pool.log if kind == "remove"]
    assert order.index(1) < order.index(0)                  # the shorter one leaves first
    adds = [rid for kind, rid in pool.log if kind == "add"]
    assert adds == [0, 1, 2, 3, 4]                          # FIFO admission
    for r in out:
        assert r.converged and r.finished >= r.admitted >= r.arrival
        assert r.steps == dict(enumerate([64, 32, 96, 32, 32]))[r.rid]
    assert max(len(run) for kind, run in pool.log if kind == "run") == 2   # never above capacity


def test_summary_percentiles():
    reqs = [serve.Request(k, 0.0, {}, admitted=0.0, finished=float(k + 1), converged=True) for k in range(100)]
    s = serve.summary(reqs, "x", 1.0, 1.0)
    assert s["latency_p50_s"] == pytest.approx(50.5)
    assert s["latency_p99_s"] == pytest.approx(99.01)
    assert s["solves_per_s"] == pytest.approx(1.0)


def test_request_stopped_at_the_step_cap():
    """A request that does not converge leaves at max_steps, unconverged, with the pool's own
    step count; the others are unaffected (the loop counts running requests' steps itself)."""
    reqs = [serve.Request(0, 0.0, dict(rid=0, work=1000)), serve.Request(1, 0.0, dict(rid=1, work=64))]
    pool = FakePool(capacity=2)
    srv = serve.Server(residual=1e-8, chunk=32, max_steps=128, pool=pool)
    out = {r.rid: r for r in srv.serve(reqs, clock="steps")}
    assert not out[0].converged and out[0].steps == 128
    assert out[1].converged and out[1].steps == 64
    assert [rid for kind, rid in pool.log if kind == "remove"] == [1, 0]
