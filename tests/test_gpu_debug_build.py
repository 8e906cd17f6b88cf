"""The checked build (liblc_debug.so, -DLC_DEBUG=1): its index checks are
wired to the host, and it runs the GPU parity suites to the same results as
the release build with no check failing.

The checked build tests every neighbour id, cluster label, destination and
coarse id the kernels follow against the array it addresses; a failed check
is recorded (never a fault) and turns the call into LC_ERR_DEVICE.  The
self-test fails one check on purpose without addressing memory.  The suites
run in a child process with LC_DEBUG=1, which makes the binding load the
checked build, so any recorded failure fails the test that made the call."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2608_01503_gb300 import _build  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_families.py", "tests/test_gpu_leiden.py",
          "tests/test_gpu_constrained.py", "tests/test_gpu_batch.py", "tests/test_gpu_tables.py",
          "tests/test_gpu_ablations.py", "tests/test_gpu_server.py"]


@pytest.fixture(scope="module")
def checked_env():
    _build.build(debug=True)
    env = dict(os.environ)
    env["LC_DEBUG"] = "1"
    return env


def test_selftest_reports_the_planted_failure(checked_env):
    code = ("import paper_2608_01503_gb300 as lc\n"
            "assert lc.library_path().endswith('liblc_debug.so')\n"
            "assert lc.lc_debug_enabled()\n"
            "d = lc.lc_debug_selftest()\n"
            "assert d == (15 << 56) | 7, hex(d)\n"
            "print('selftest ok')\n")
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=checked_env, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "selftest ok" in p.stdout


def test_parity_suites_pass_under_the_checked_build(checked_env):
    p = subprocess.run([sys.executable, "-m", "pytest", *SUITES, "-m", "gpu and not slow", "-x", "-q",
                        "-p", "no:cacheprovider"],
                       cwd=ROOT, env=checked_env, capture_output=True, text=True, timeout=1800)
    assert p.returncode == 0, (p.stdout[-4000:] + p.stderr[-2000:])
