"""The GPU parity suites under the bounds-checking build of the library.

compute-sanitizer is not available, so the library is also built with -DCCC_BOUNDS_CHECK
(include/ccc_checked.h): every output index of the tally kernels, the 2-way table reads
of the 3-way genotype-class route and the shared-memory stores of the code expansion are
tested on the device, and an index outside its buffer records CCC_EBOUNDS and skips the
access.  This test builds that library and runs the 2-way, 3-way, s-state, K-split,
phase, thresholded, batched and packed-operand parity suites against it in a child
pytest (CCC_LIBRARY selects it).  Each of their calls asserts ccc_status == CCC_OK, so an
index outside its buffer fails them; test_gpu_checked_hook.py checks that the checks fire.
"""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

SUITES = ["tests/test_gpu_2way.py", "tests/test_gpu_pair.py", "tests/test_gpu_packed.py",
          "tests/test_gpu_split.py", "tests/test_gpu_phases.py", "tests/test_gpu_filter.py",
          "tests/test_gpu_3way.py", "tests/test_gpu_multi.py", "tests/test_gpu_batched.py"]
HOOK = "tests/test_gpu_checked_hook.py"


def test_parity_suites_under_the_checked_build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if os.environ.get("CCC_LIBRARY"):
        pytest.skip("this process already runs another build of the library")
    from paper_1705_08213_gb300 import build
    build.build()
    lib = build.build(checked=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CCC_LIBRARY=lib)

    def child(files):
        p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu",
                            "-p", "no:cacheprovider", *files],
                           cwd=root, env=env, capture_output=True, text=True, timeout=1800)
        assert p.returncode == 0, p.stdout[-6000:] + p.stderr[-2000:]
        return p.stdout.strip().splitlines()[-1]

    assert " passed" in child(SUITES)
    last = child([HOOK])  # the hook tests run only under the checked build: none may skip
    assert " passed" in last and "skipped" not in last, last
