"""Device-side failure detection without a GPU fault.

Every pipeline of the library waits on mbarriers through one bounded loop.  A
wait that nothing can complete must give up after its limit, record
CCC_ETIMEOUT in the status word and return; the CUDA context stays usable, so a
correct call right after it still matches the oracle.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, run_2way

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


@pytest.mark.parametrize("limit_ms", [5, 50])
def test_wait_gives_up_and_reports_timeout(limit_ms):
    import torch

    import paper_1705_08213_gb300 as ccc
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    ccc.ccc_check_bounded_wait(status, limit_ms * 1000000)
    e1.record(stream)
    torch.cuda.synchronize()
    assert int(status.item()) == ccc.CCC_ETIMEOUT
    ms = e0.elapsed_time(e1)
    assert limit_ms * 0.9 <= ms < limit_ms + 500, ms
    # first error wins: a second timeout leaves the recorded code alone
    ccc.ccc_check_bounded_wait(status, 1000000)
    torch.cuda.synchronize()
    assert int(status.item()) == ccc.CCC_ETIMEOUT


def test_context_usable_after_timeout():
    import torch

    import paper_1705_08213_gb300 as ccc
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ccc.ccc_check_bounded_wait(status, 20000000)
    torch.cuda.synchronize()
    assert int(status.item()) == ccc.CCC_ETIMEOUT
    n_v, n_f = 200, 500
    geno = synth.panel_hwe(n_v, n_f, seed=31, p_missing=0.02)
    t, c = run_2way(geno, n_f, 0)  # asserts the call's own status is CCC_OK
    et, ec = oracle.ccc2_all(geno, n_f)
    assert_tally_equal(t, et, "after timeout")
    assert_ccc_close(c, ec, what="after timeout")
