"""The convergence study's models (Sec. V, last paragraph) on the GPU against the
oracle, step by step: the reference model HHLB(10;50) x HLB(6;7) on S = 48 nodes
and the production models HHLB(6;7) x HLB(6;7), HHLB(10;16) x HLB(6;7) on S = 16,
all on the stretched grid A = 0.98 with u_w = sqrt(2), the half channel and local
pseudo-time steps, as the study runs them. Qx = 50 reaches half-range weights
near 1e-50 and weight-divided equilibria far outside the other parity cases.
FP64 within 1e-12, the compensated FP32 state within 1e-5."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07803_gb300 import build, lbc, studies
from tests.helpers import gpu_available, moment_errors

pytestmark = pytest.mark.gpu

OMEGA, PR = 0.66, 2.0 / 3.0


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


MODELS = [("reference", d) for d in (0.1, 1.0, 10.0)] + [("production", d) for d in (0.1, 10.0)]


@pytest.mark.parametrize("kind,delta", MODELS)
def test_study_model_matches_oracle(kind, delta):
    make = studies.reference if kind == "reference" else studies.production
    nsteps = 20
    o = Oracle(make(delta, OMEGA, PR))
    o.run(nsteps)
    ref = o.moments()
    for precision, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        p = make(delta, OMEGA, PR, precision=precision, compensated=precision == "fp32")
        s = lbc.Solver(p)
        s.step(nsteps)
        e = moment_errors(s.moments(), ref)
        assert np.all(e < tol), (precision, dict(zip(lbc.MOMENT_NAMES, e)))
        s.close()
