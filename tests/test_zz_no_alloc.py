"""The allocation-free entry point (lbc_step_noalloc) against the regular
solver (lbc_create + lbc_step): same problem, same initial state, compared on
two calls in a row, each continuing from the previous call's output.

lbc_step_noalloc serves callers that cannot allocate device memory (an
application whose allocator owns the GPU memory, or a latency-critical loop):
it keeps its working memory in a static device array inside the library and
steps a state buffer that the caller owns. Here the caller's buffer is a torch
CUDA tensor. This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

from paper_1810_07803_gb300 import build, lbc, workloads
from tests.helpers import gpu_available, weighted_state_error

pytestmark = pytest.mark.gpu

PROBLEM = dict(Nx=65, Qx=5, Qy=6, stretch_A=math.sqrt(0.9), delta=2.0, u_left=-0.1, u_right=0.2,
               T_left=0.8, T_right=1.25, omega=0.7, Pr=0.68)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build()


def weights(p):
    _, wx = lbc.quadrature(p["Qx"], True)
    _, wy = lbc.quadrature(p["Qy"], False)
    return np.outer(np.concatenate([wx, wx]), wy).ravel()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_matches_regular_solver_on_two_calls(precision, tol):
    import torch
    p = dict(PROBLEM, precision=precision)
    s = lbc.Solver(p)
    f0 = workloads.perturbed_state(s.V, s.Nx, s.get_state(), seed=21, amplitude=0.1)
    s.set_state(f0)
    state = torch.tensor(f0, dtype=torch.float64, device="cuda")   # caller-owned device buffer
    w = weights(p)
    for _ in range(2):
        s.step(12)
        lbc.step_noalloc(p, state.data_ptr(), 12)
        torch.cuda.synchronize()
        err = weighted_state_error(state.cpu().numpy(), s.get_state(), w)
        assert err < tol, err
    s.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    p = dict(workloads.c2(1.0, precision="fp64"))
    state = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lbc.LbcError) as e:
        lbc.step_noalloc(p, state.data_ptr(), 1)
    assert e.value.status == lbc.EINVAL
    assert "allocation-free path has" in str(e.value)


def test_noalloc_call_allocates_no_device_memory():
    """After a first call (which resolves the static array's address and sets kernel
    attributes), a call leaves the device's free memory as it was: it allocates nothing."""
    import torch
    p = dict(PROBLEM, precision="fp32")
    with lbc.Solver(p) as s:
        f0 = s.get_state()
    state = torch.tensor(f0, dtype=torch.float64, device="cuda")
    lbc.step_noalloc(p, state.data_ptr(), 3)     # warm-up: first call on this device
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    lbc.step_noalloc(p, state.data_ptr(), 3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # a released pool block could only raise the free figure; an allocation would lower it
    assert free1 >= free0, (free0, free1)
