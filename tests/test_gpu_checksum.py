"""The result checksum (ccc_checksum) against the oracle's twin.

* Tallies: the device checksum of every tally of a 2-way, 3-way and
  multi-allelic call equals the oracle's checksum of its own tallies.
* Additivity: the checksums of the phases of a call, each with its global word
  offset, add up (mod 2^128) to the checksum of the full call, for tallies and
  CCC values (bit patterns).
* CCC values bit for bit across routes: fused epilogue = metric from stored
  tallies, and streamed to host memory = computed on the device.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import run_2way, run_3way, run_multi, to_device, workspace

pytestmark = pytest.mark.gpu

M128 = 1 << 128


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _dev_checksum(arr_np, base=0):
    import torch

    import paper_1705_08213_gb300 as ccc
    t = torch.from_numpy(np.ascontiguousarray(arr_np)).cuda()
    return ccc.ccc_checksum(t, base)


def test_2way_tallies_match_oracle_checksum():
    n_v, n_f = 1500, 6000
    geno = synth.panel_hwe(n_v, n_f, seed=41, p_missing=0.01)
    t, c = run_2way(geno, n_f, 0)
    et, _ = oracle.ccc2_all(geno, n_f)
    assert _dev_checksum(t) == oracle.checksum(et)
    # the popcount path gives the same checksum
    tp, cp = run_2way(geno, n_f, 1)
    assert _dev_checksum(tp) == _dev_checksum(t)
    assert _dev_checksum(cp) == _dev_checksum(c)


def test_3way_tallies_match_oracle_checksum():
    n_v, n_f = 300, 2000
    geno = synth.panel_hwe(n_v, n_f, seed=42, p_missing=0.01)
    t, c = run_3way(geno, n_f, 0)
    et, _ = oracle.ccc3_slabs(geno, n_f)
    assert _dev_checksum(t) == oracle.checksum(et)


def test_multi_tallies_match_oracle_checksum():
    s, n_v, n_f = 4, 700, 2000
    gm = synth.panel_multi(n_v, n_f, s, seed=43, p_missing=0.02)
    t, c = run_multi(gm, n_f, s)
    et, _ = oracle.ccc2_multi_all(gm, n_f, s)
    assert _dev_checksum(t) == oracle.checksum(et)


def test_phase_checksums_add_up():
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 2000, 3000
    geno = synth.panel_hwe(n_v, n_f, seed=44, p_missing=0.02)
    t_full, c_full = run_2way(geno, n_f, 0)
    whole_t, whole_c = _dev_checksum(t_full), _dev_checksum(c_full)
    g = to_device(geno)
    opts = ccc.ccc_opts_default()
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(workspace=ws)
    bounds = ccc.ccc2_phase_bounds(n_v, 5)
    sum_t = sum_c = 0
    for i0, i1 in zip(bounds, bounds[1:]):
        cnt = ccc.ccc2_rows_count(n_v, i0, i1)
        if cnt == 0:
            continue
        t = torch.empty((cnt, 4), dtype=torch.int32, device="cuda")
        c = torch.empty((cnt, 4), dtype=torch.float32, device="cuda")
        ccc.ccc2_tally_metric_rows(g, n_f, i0, i1, t, c, opts)
        base = 4 * ccc.ccc2_index(i0, i0 + 1, n_v)
        sum_t += ccc.ccc_checksum(t, base)
        sum_c += ccc.ccc_checksum(c, base)
    assert sum_t % M128 == whole_t
    assert sum_c % M128 == whole_c


def test_ccc_bits_equal_across_routes():
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 1200, 2500
    geno = synth.panel_hwe(n_v, n_f, seed=45, p_missing=0.03)
    for norm in (0, 1):
        _, c_fused = run_2way(geno, n_f, 0, norm=norm, fused=True)
        _, c_split = run_2way(geno, n_f, 0, norm=norm, fused=False)
        assert _dev_checksum(c_fused) == _dev_checksum(c_split)
    g = to_device(geno)
    opts = ccc.ccc_opts_default()
    ws = workspace(ccc.ccc2_stream_workspace_size(g, n_f, 4, opts))
    opts = ccc.ccc_opts_default(workspace=ws)
    npairs = ccc.ccc2_count(n_v)
    ht = torch.empty((npairs, 4), dtype=torch.int32, pin_memory=True)
    hc = torch.empty((npairs, 4), dtype=torch.float32, pin_memory=True)
    ccc.ccc2_stream(g, n_f, 4, ht, hc, opts)
    torch.cuda.synchronize()
    t_dev, c_dev = run_2way(geno, n_f, 0)
    assert _dev_checksum(ht.numpy()) == _dev_checksum(t_dev)
    assert _dev_checksum(hc.numpy()) == _dev_checksum(c_dev)


def test_checksum_of_empty_and_single_words():
    import torch

    import paper_1705_08213_gb300 as ccc
    assert ccc.ccc_checksum(torch.zeros(0, dtype=torch.int32, device="cuda")) == 0
    v = np.array([5, 0, 2 ** 31 - 1], dtype=np.int32)
    for base in (0, 99, (1 << 45) + 1):
        assert _dev_checksum(v, base) == oracle.checksum(v.astype(np.int64), base)
