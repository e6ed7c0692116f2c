"""Invariants on every pair and triple of full-size workloads, against the oracle.

With no missing entries, every SNP has rho(0) + rho(1) = 2 at every individual,
so (Eqs. 1, 2, 5)
  2-way:  sum_b r_ij^{ab} = 2 s_i^a,   sum_a r_ij^{ab} = 2 s_j^b,
  3-way:  sum_c r_ijk^{abc} = 2 r_ij^{ab},  sum_b r_ijk^{abc} = 2 r_ik^{ac},
          sum_a r_ijk^{abc} = 2 r_jk^{bc},
  s states: sum_b r_ij^{ab} = 2 s_i^a  (a < s).
The allele sums s_i^a and the 2-way tables come from the CPU oracle; the device
tallies of the full-size calls (the launches bench.py times) are checked on
every pair (triple) with torch reductions on the device.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_device, to_device_bytes, workspace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _row_index(n_v, i0, i1, dev):
    """(i, j) of the pairs of rows [i0, i1) in the triangle order, on the device."""
    import torch
    lens = torch.arange(n_v - 1 - i0, n_v - 1 - i1, -1, device=dev)
    i = torch.repeat_interleave(torch.arange(i0, i1, device=dev), lens)
    start = torch.cumsum(lens, 0) - lens
    pos = torch.arange(int(lens.sum()), device=dev) - torch.repeat_interleave(start, lens)
    return i, i + 1 + pos


def test_2way_full_size_every_pair_marginals():
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 20000, 16384
    geno = synth.panel_hwe(n_v, n_f, seed=1, p_missing=0.0)
    s0, s1, npres = oracle.allele_counts(geno, n_f)
    assert np.all(npres == n_f)
    g = to_device(geno)
    opts = ccc.ccc_opts_default()
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(workspace=ws)
    npairs = ccc.ccc2_count(n_v)
    tally = torch.empty((npairs, 4), dtype=torch.int32, device="cuda")
    out = torch.empty((npairs, 4), dtype=torch.float32, device="cuda")
    ccc.ccc2_tally_metric(g, n_f, tally, out, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    S = torch.from_numpy(np.stack([s0, s1], 1)).cuda()
    for i0 in range(0, n_v, 2500):
        i1 = min(n_v, i0 + 2500)
        ii, jj = _row_index(n_v, i0, i1, "cuda")
        p0 = ccc.ccc2_index(i0, i0 + 1, n_v) if i0 < n_v - 1 else npairs
        t = tally[p0:p0 + ii.numel()].to(torch.int64)
        assert torch.equal(t[:, 0] + t[:, 1], 2 * S[ii, 0])
        assert torch.equal(t[:, 2] + t[:, 3], 2 * S[ii, 1])
        assert torch.equal(t[:, 0] + t[:, 2], 2 * S[jj, 0])
        assert torch.equal(t[:, 1] + t[:, 3], 2 * S[jj, 1])


def test_3way_full_size_every_triple_marginals():
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f = 1536, 8192
    geno = synth.panel_hwe(n_v, n_f, seed=4, p_missing=0.0)
    t2, _ = oracle.ccc2_all(geno, n_f)  # [npairs, 4], (a, b) = 00, 01, 10, 11
    T2 = torch.from_numpy(t2).cuda()
    g = to_device(geno)
    opts = ccc.ccc_opts_default()
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_3WAY))
    opts = ccc.ccc_opts_default(workspace=ws)
    nt = ccc.ccc3_count(n_v, 0, n_v)
    tally = torch.empty((nt, 8), dtype=torch.int32, device="cuda")
    out = torch.empty((nt, 8), dtype=torch.float32, device="cuda")
    ccc.ccc3_tally_metric(g, n_f, 0, n_v, tally, out, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK

    def pidx(i, j):
        return i * (2 * n_v - i - 1) // 2 + (j - i - 1)

    checked = 0
    for j in range(1, n_v - 1):
        nk = n_v - 1 - j
        t0 = ccc.ccc3_index(0, j, j + 1, n_v)
        t = tally[t0:t0 + j * nk].to(torch.int64).view(j, nk, 2, 2, 2)  # [i, k, a, b, c]
        i = torch.arange(j, device="cuda")
        k = torch.arange(j + 1, n_v, device="cuda")
        rij = T2[pidx(i, torch.full_like(i, j))].view(j, 1, 2, 2)          # (a, b)
        rik = T2[pidx(i[:, None], k[None, :])].view(j, nk, 2, 2)           # (a, c)
        rjk = T2[pidx(torch.full_like(k, j), k)].view(1, nk, 2, 2)          # (b, c)
        assert torch.equal(t.sum(4), 2 * rij.expand(j, nk, 2, 2))
        assert torch.equal(t.sum(3), 2 * rik)
        assert torch.equal(t.sum(2), 2 * rjk.expand(j, nk, 2, 2))
        checked += j * nk
    assert checked == nt


def test_multi_full_size_every_pair_marginals():
    import torch

    import paper_1705_08213_gb300 as ccc
    s, n_v, n_f = 4, 10000, 16384
    gm = synth.panel_multi(n_v, n_f, s, seed=6, p_missing=0.0)
    cnt = oracle.multi_counts(gm, n_f, s)
    assert np.all(cnt[:, s] == n_f)
    g = to_device_bytes(gm)
    opts = ccc.ccc_opts_default()
    ws = workspace(ccc.ccc_multi_workspace_size(g, n_f, s, opts))
    opts = ccc.ccc_opts_default(workspace=ws)
    npairs = ccc.ccc2_count(n_v)
    tally = torch.empty((npairs, s * s), dtype=torch.int32, device="cuda")
    out = torch.empty((npairs, s * s), dtype=torch.float32, device="cuda")
    ccc.ccc2_multi_tally_metric(g, n_f, s, tally, out, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    S = torch.from_numpy(cnt[:, :s]).cuda()
    for i0 in range(0, n_v, 2000):
        i1 = min(n_v, i0 + 2000)
        ii, jj = _row_index(n_v, i0, i1, "cuda")
        p0 = ccc.ccc2_index(i0, i0 + 1, n_v) if i0 < n_v - 1 else npairs
        t = tally[p0:p0 + ii.numel()].to(torch.int64).view(-1, s, s)
        assert torch.equal(t.sum(2), 2 * S[ii])
        assert torch.equal(t.sum(1), 2 * S[jj])
