"""The allocation-free 2-way entry point agrees with the oracle and with the workspace entry point.

ccc2_tally_metric_noalloc serves callers that cannot allocate device memory
(a host framework that owns all device allocations, plug-ins handed only their
input and output buffers): it keeps its scratch in a fixed array built into
the library.  This file is collected last so that, if it fails, a run that
stops at the first failure has already run every other test.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import CCC_RTOL, assert_ccc_close, assert_tally_equal, run_2way, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _noalloc(geno_np, n_f, norm=0, tile=0, with_status=True, stream=None, want_ccc=True):
    import torch

    import paper_1705_08213_gb300 as ccc
    g = to_device(geno_np)
    n_v = geno_np.shape[0]
    npairs = ccc.ccc2_count(n_v)
    tally = torch.full((max(npairs, 1), 4), -7, dtype=torch.int32, device="cuda")
    out = torch.full((max(npairs, 1), 4), -7.0, dtype=torch.float32, device="cuda")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda") if with_status else None
    opts = ccc.ccc_opts_default(path=ccc.CCC_PATH_TC, norm=norm, tile=tile)
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())
    ccc.ccc2_tally_metric_noalloc(g, n_f, tally, out if want_ccc else None, opts, status=status,
                                  stream=stream)
    torch.cuda.synchronize()
    if with_status:
        assert int(status.item()) == ccc.CCC_OK
    return tally[:npairs].cpu().numpy(), out[:npairs].cpu().numpy()


def test_noalloc_matches_workspace_entry_point_twice():
    # Two calls in a row; the second panel is smaller, so anything left over in
    # the shared built-in scratch from the first call would show up.
    cases = [(synth.panel_hwe(300, 1000, seed=31, p_missing=0.02, pad_seed=3), 1000, 0),
             (synth.panel_uniform(129, 777, seed=32, p_missing=0.05, pad_seed=4), 777, 1)]
    for geno, n_f, norm in cases:
        t_ref, c_ref = run_2way(geno, n_f, 0, norm=norm)
        t, c = _noalloc(geno, n_f, norm=norm)
        assert_tally_equal(t, t_ref, "noalloc tallies")
        assert_ccc_close(c, c_ref.astype(np.float64), rtol=CCC_RTOL, what="noalloc CCC")


@pytest.mark.parametrize("tile", [0, 1])
@pytest.mark.parametrize("norm", [0, 1])
def test_noalloc_against_oracle(tile, norm):
    # Several 128-SNP tiles with a ragged tail, K past one 128-entry stage with a tail.
    n_v, n_f = 333, 1111
    geno = synth.panel_hwe(n_v, n_f, seed=33 + norm, p_missing=0.03, pad_seed=5)
    t, c = _noalloc(geno, n_f, norm=norm, tile=tile)
    et, ec = oracle.ccc2_all(geno, n_f, norm=norm)
    assert_tally_equal(t, et, "noalloc tallies vs oracle")
    assert_ccc_close(c, ec, rtol=CCC_RTOL, what="noalloc CCC vs oracle")


def test_noalloc_nearly_full_scratch():
    # n_v = 2,048 and n_f = 7,680 take 17,408 + 4,352 x 7,680 = 33,440,768 of the 33,554,432
    # scratch bytes (99.7%); one more individual does not fit (the rejection test below).
    n_v, n_f = 2048, 7680
    geno = synth.panel_hwe(n_v, n_f, seed=34, p_missing=0.01, pad_seed=6)
    t, c = _noalloc(geno, n_f)
    t_ref, c_ref = run_2way(geno, n_f, 0)
    assert_tally_equal(t, t_ref, "noalloc tallies, nearly full scratch")
    assert_ccc_close(c, c_ref.astype(np.float64), rtol=CCC_RTOL, what="noalloc CCC, full scratch")
    rows = np.array([0, 1, 127, 128, 1023, 1900, 2046])
    et, ec = oracle.ccc2_rows(geno, n_f, rows)
    idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, n_v), n_v) for i in rows])
    assert_tally_equal(t[idx], et, "noalloc sampled rows vs oracle")
    assert_ccc_close(c[idx], ec, rtol=CCC_RTOL, what="noalloc sampled rows vs oracle")


def test_noalloc_without_status_on_a_side_stream_and_tallies_only():
    import torch
    geno = synth.panel_hwe(200, 600, seed=35, p_missing=0.02, pad_seed=7)
    t_ref, c_ref = run_2way(geno, 600, 0)
    side = torch.cuda.Stream()
    t, c = _noalloc(geno, 600, with_status=False, stream=side)
    assert_tally_equal(t, t_ref, "noalloc tallies, status=None, side stream")
    assert np.array_equal(c.view(np.int32), c_ref.view(np.int32)), "CCC bits differ"
    t2, c2 = _noalloc(geno, 600, want_ccc=False)
    assert_tally_equal(t2, t_ref, "noalloc tallies only")
    assert np.all(c2 == -7.0), "a tallies-only call wrote CCC values"


def test_noalloc_rejects_panels_beyond_the_scratch():
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 2048, 7681  # one individual past the 32 MiB limit at this n_v
    geno = torch.zeros((n_v, synth.default_ld(n_f)), dtype=torch.int64, device="cuda")
    tally = torch.empty((16, 4), dtype=torch.int32, device="cuda")
    out = torch.empty((16, 4), dtype=torch.float32, device="cuda")
    opts = ccc.ccc_opts_default(path=ccc.CCC_PATH_TC)
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc2_tally_metric_noalloc(geno, n_f, tally, out, opts)
    assert e.value.status == ccc.CCC_ERANGE
    opts = ccc.ccc_opts_default(path=ccc.CCC_PATH_POPC)
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc2_tally_metric_noalloc(geno[:8], 100, tally, out, opts)
    assert e.value.status == ccc.CCC_EINVAL
    for field, value in (("tile", 3), ("split", 2), ("group", -1), ("tile", 7)):
        opts = ccc.ccc_opts_default(path=ccc.CCC_PATH_TC)
        setattr(opts, field, value)
        with pytest.raises(ccc.CCCError) as e:
            ccc.ccc2_tally_metric_noalloc(geno[:8], 100, tally, out, opts)
        assert e.value.status == ccc.CCC_EINVAL, (field, value)


def test_noalloc_on_two_devices():
    # The scratch address and the kernels' launch set-up are per device.
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    geno = synth.panel_hwe(150, 500, seed=36, p_missing=0.02, pad_seed=8)
    et, ec = oracle.ccc2_all(geno, 500)
    for d in (0, 1):
        with torch.cuda.device(d):
            t, c = _noalloc(geno, 500)
        assert_tally_equal(t, et, f"noalloc tallies on device {d}")
        assert_ccc_close(c, ec, rtol=CCC_RTOL, what=f"noalloc CCC on device {d}")
