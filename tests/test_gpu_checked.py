"""The checked build (libamgd_checked.so, compiled with AMGD_CHECKS): every
gather index the sweep and distance kernels read from the matrix -- a column
index, a renumbered column or a row map -- is tested against the vector block
inside the kernel before its load.

* The GPU parity tests, run in a child process against the checked build,
  pass unchanged: on every shape, stage and storage they exercise no index
  fails its test, and the results are the normal build's.
* A column index planted out of range after the handle's setup is caught by
  the sweep's test and reported as AMGD_ERR_CHECK by the next synchronising
  call; the load itself is redirected to row 0 and never leaves the buffer.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checked_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1106_5990_gb300 import _build
    _build.build()
    return _build.build(checked=True)


def _child(args, **env_extra):
    env = dict(os.environ, AMGD_CHECKED="1", **env_extra)
    return subprocess.run([sys.executable, *args], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=1800)


def test_child_loads_the_checked_build(checked_lib):
    p = _child(["-c", "from paper_1106_5990_gb300 import amgd; print(amgd.amgd_checked_build())"])
    assert p.returncode == 0 and p.stdout.strip() == "1", p.stdout + p.stderr
    p = subprocess.run([sys.executable, "-c", "from paper_1106_5990_gb300 import amgd; "
                        "print(amgd.amgd_checked_build())"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600,
                       env={k: v for k, v in os.environ.items() if k != "AMGD_CHECKED"})
    assert p.returncode == 0 and p.stdout.strip() == "0", p.stdout + p.stderr


def test_parity_tests_pass_under_the_checked_build(checked_lib):
    p = _child(["-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                "tests/test_gpu_parity.py", "tests/test_gpu_mixed.py", "tests/test_gpu_depth.py"])
    assert p.returncode == 0, p.stdout[-4000:] + p.stderr[-4000:]


PLANTED = r'''
from paper_1106_5990_gb300 import amgd, inputs
assert amgd.amgd_checked_build() == 1
rp, col, val = inputs.poisson2d_5pt(40)                  # 1600 rows, slot 77 exists
with amgd.Handle(rp, col, val, 8, 1) as h:
    h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, 4, 1, 4, 0)   # the direct sweep kernel
    h.relax(1, 0.7)
    try:
        h.get_vectors()                                    # synchronises: reads the status
    except amgd.AmgdError as e:
        assert e.status == amgd.AMGD_ERR_CHECK, e
        print("caught")
    else:
        raise SystemExit("the planted column was not reported")
'''


def test_planted_column_is_caught(checked_lib):
    p = _child(["-c", PLANTED], AMGD_TEST_BAD_COLUMN="77")
    assert p.returncode == 0 and p.stdout.strip().endswith("caught"), p.stdout + p.stderr
