"""Full-size parity of the non-isothermal grid (Nx = 1024, 48 x 24 velocities,
T_R/T_L in {1, 3, 10} x delta in {0.5, 5, 50}) and of a sample of the 512-solve
uneven batch, each in the launch configuration a user gets (one batch of all
instances), against the FP64 oracle after a few steps.

The oracle steps one solve of the non-isothermal grid in about a second, so the
full grid is compared whole; from the uneven batch, whose oracle cost would be
minutes, the smallest, the largest and a seeded sample of instances are
compared, and every instance is checked for finite moments and conserved mass."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07803_gb300 import build, lbc, workloads
from tests.helpers import gpu_available, moment_errors

pytestmark = pytest.mark.gpu

REPORTED = ("n", "T", "q_x", "P_xy")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


def test_nonisothermal_grid_matches_oracle():
    """Both precisions, one batch of the nine solves each, from seeded perturbed states
    installed in one call (every node and velocity off equilibrium, so the bulk WENO,
    the per-node equilibrium at non-trivial (u, T, q) and the moment sums are in play),
    3 steps; the oracle runs once per solve."""
    ref, states = [], []
    for i, p in enumerate(workloads.c3(precision="fp64")):
        o = Oracle(p)
        f = workloads.perturbed_state(o.V, o.Nx, o.f, seed=60 + i, amplitude=0.1)
        states.append(f)
        o.set_state(f)
        o.run(3)
        ref.append(o.moments())
    for precision, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        ps = workloads.c3(precision=precision)
        b = lbc.Batch(ps)
        b.set_states(states)
        b.step(3)
        worst = {}
        for i, p in enumerate(ps):
            e = moment_errors(b.moments(i), ref[i])
            for k in REPORTED:
                worst[k] = max(worst.get(k, 0.0), float(e[lbc.MOMENT_NAMES.index(k)]))
            assert np.all(e < tol), (precision, p["T_right"] / p["T_left"], p["delta"],
                                     dict(zip(lbc.MOMENT_NAMES, e)))
        print(precision, {k: f"{v:.1e}" for k, v in worst.items()})
        b.close()


def test_uneven_batch_sampled():
    ps = workloads.c4()
    b = lbc.Batch(ps)
    sizes = [p["Nx"] * 2 * p["Qx"] * p["Qy"] for p in ps]
    rng = np.random.default_rng(44)
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), *rng.choice(len(ps), 3, replace=False).tolist()})
    m0 = {i: b.moments(i)[0].copy() for i in range(len(ps))}
    b.step(2)
    for i in range(len(ps)):
        m = b.moments(i)
        assert np.all(np.isfinite(m)), i
    for i in sample:
        o = Oracle(ps[i])
        o.run(2)
        e = moment_errors(b.moments(i), o.moments())
        assert np.all(e < 1e-5), (i, dict(zip(lbc.MOMENT_NAMES, e)))
        mass0 = float(np.sum(o.J * o.deta * m0[i]))
        mass = float(np.sum(o.J * o.deta * b.moments(i)[0]))
        assert abs(mass - mass0) < 1e-5 * mass0, i
    b.close()
