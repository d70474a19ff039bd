"""The range-checked build (liblbc_checked.so: the kernels compiled with
LBC_CHECKED). Every computed index of the stage, node-equilibrium and
persistent kernels is checked before its access: TMA box alignment, bulk-copy
extents, stencil, ghost and RK-base columns, equilibrium factor indices,
state and compensation stores, symmetry-plane partners, cluster exchange
slots and persistent work neighbours. A failed check skips the access and is
reported as LBC_EBOUNDS; nothing traps.

The binding picks the library when it loads (LBC_CHECKED=1), so the parity,
batch, configuration, compensated-state, persistent and allocation-free test
files run again in a child process against the checked library: every kernel
form (FP64 and FP32, plain and extended, single and batched launches, cluster
sizes 1 to 4, the persistent form) must pass its oracle comparisons with no
check failing."""
import os
import subprocess
import sys

import pytest

from paper_1810_07803_gb300 import build
from tests.helpers import gpu_available

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ["tests/test_parity_gpu.py", "tests/test_batch_gpu.py", "tests/test_configs_gpu.py",
         "tests/test_compensated_gpu.py", "tests/test_persistent_gpu.py", "tests/test_zz_no_alloc.py"]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not gpu_available():
        pytest.skip("no GPU")
    build.build(checked=True)


def child_env():
    return dict(os.environ, LBC_CHECKED="1")


def test_binding_loads_the_checked_library():
    code = "from paper_1810_07803_gb300 import lbc; assert lbc.checked_build(), lbc.LIB_PATH"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=child_env(), capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr


def test_parity_files_pass_with_every_index_checked():
    r = subprocess.run([sys.executable, "-m", "pytest", *FILES, "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=child_env(), capture_output=True, text=True, timeout=1800)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-30:])
    assert r.returncode == 0, tail
    assert "passed" in tail and "failed" not in tail, tail
