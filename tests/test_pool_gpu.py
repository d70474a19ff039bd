"""The instance pool and the serving loop on the GPU: admission by device
budget, parity of pooled instances with the FP64 oracle, and the same result
for every request alone and in a continuously batched mix."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07803_gb300 import build, lbc, serve, workloads
from tests.helpers import gpu_available, moment_errors

pytestmark = pytest.mark.gpu

MIX = [
    dict(Nx=40, Qx=4, Qy=4, delta=1.0, u_left=-0.07, u_right=0.07),
    dict(Nx=65, Qx=5, Qy=6, stretch_A=math.sqrt(0.9), delta=2.0, u_left=-0.1, u_right=0.2, T_left=0.8,
         T_right=1.25, omega=0.7, Pr=0.68),
    dict(Nx=72, Qx=8, Qy=6, stretch_A=0.7, delta=0.6, u_left=-0.3, u_right=0.3, T_left=0.7, T_right=1.3),
    dict(Nx=33, Qx=6, Qy=5, delta=3.0, u_left=0.05, u_right=-0.15, T_left=1.1, T_right=0.9, p0=1.2),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


def test_pooled_instances_match_the_oracle_fp64():
    pool = lbc.Pool(cluster=4, precision="fp64", budget_bytes=1 << 30)
    slots = [pool.try_add(p) for p in MIX]
    assert None not in slots
    assert pool.run(1e-30, 25) == []          # nothing converges to 1e-30
    for slot, p in zip(slots, MIX):
        assert pool.info(slot)[3] == 25
        o = Oracle(p)
        o.run(25)
        e = moment_errors(pool.moments(slot), o.moments())
        assert np.all(e < 1e-12), (slot, dict(zip(lbc.MOMENT_NAMES, e)))
    pool.close()


def test_admission_by_device_budget():
    fp = [lbc.Pool.footprint(dict(p, precision="fp32"), 4) for p in MIX[:3]]
    assert fp[2] // 2 < fp[1]                               # freeing instance 1 makes room for 2
    pool = lbc.Pool(cluster=4, precision="fp32", budget_bytes=fp[0] + fp[1] + fp[2] // 2)
    a, b = pool.try_add(MIX[0]), pool.try_add(MIX[1])
    assert a is not None and b is not None
    assert pool.try_add(MIX[2]) is None                     # does not fit: the caller queues it
    used, n, _ = pool.usage()
    assert n == 2 and used == fp[0] + fp[1]
    pool.remove(b)
    assert pool.usage()[0] == fp[0]
    assert pool.try_add(MIX[2]) is not None                 # fits once memory is freed
    assert pool.usage()[0] == fp[0] + fp[2]
    pool.close()


def test_instance_leaves_at_its_own_converged_step():
    """Three copies of one problem at different rarefaction converge at different
    steps; each equals the single-instance solver's run-to-steady (FP64)."""
    base = dict(Nx=40, Qx=4, Qy=4, u_left=-0.07, u_right=0.07)
    ps = [dict(base, delta=d) for d in (0.5, 1.5, 4.0)]
    pool = lbc.Pool(cluster=2, precision="fp64", budget_bytes=1 << 30)
    slots = [pool.try_add(p) for p in ps]
    finished = {}
    for _ in range(2000):
        for s in pool.run(1e-9, 64):
            finished[s] = pool.info(s)[3]
        if len(finished) == 3:
            break
    assert len(finished) == 3
    for slot, p in zip(slots, ps):
        s = lbc.Solver(p)
        k, r = s.run_to_steady(1e-9, 200000)
        assert abs(finished[slot] - k) <= 1, (finished[slot], k)
        e = moment_errors(pool.moments(slot), s.moments())
        assert np.all(e < 1e-10), dict(zip(lbc.MOMENT_NAMES, e))
        s.close()
    assert len(set(finished.values())) == 3
    pool.close()


def _small(rng):
    p = serve.small_solve(rng)
    p.update(Nx=int(rng.integers(32, 65)), Qx=int(rng.integers(4, 7)), Qy=int(rng.integers(4, 7)),
             delta=float(rng.uniform(0.5, 2.0)))
    return p


def test_same_result_alone_and_in_the_served_mix():
    """Requests that arrive while others run join the next chunk of steps. Each
    request's steps and moments equal, bit for bit, serving it alone (converged
    or stopped at the step cap alike)."""
    rng = np.random.default_rng(12)
    reqs = [serve.Request(k, float(arr), _small(rng)) for k, arr in enumerate([0, 0, 1, 1, 2, 4, 5, 5])]
    kw = dict(cluster=3, residual=1e-6, chunk=48, budget_bytes=1 << 30, max_steps=12000)
    srv = serve.Server(**kw)
    mixed = srv.serve([serve.Request(r.rid, r.arrival, r.params) for r in reqs], clock="steps")
    srv.close()
    assert sum(r.converged for r in mixed) >= len(mixed) // 2
    assert len({r.steps for r in mixed}) > 1
    for r in mixed:
        alone = serve.Server(**kw)
        a = alone.serve([serve.Request(r.rid, 0.0, r.params)], clock="steps")[0]
        alone.close()
        assert (a.steps, a.converged) == (r.steps, r.converged), (r.rid, a.steps, r.steps)
        assert np.array_equal(a.moments, r.moments), r.rid


def test_pool_rejects_instances_too_large_for_its_cluster():
    pool = lbc.Pool(cluster=1, precision="fp32", budget_bytes=1 << 30)
    with pytest.raises(lbc.LbcError) as e:   # 2 x 24 x 24 = 1152 velocities need more than one chunk CTA
        pool.try_add(dict(Nx=64, Qx=24, Qy=24))
    assert e.value.status == lbc.EINVAL
    pool.close()
