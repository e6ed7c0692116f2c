"""GPU thresholded 2-way output (ccc2_filter) against the oracle.

The kept set must equal the oracle's set of pairs whose largest CCC value
exceeds the threshold, except pairs within 1e-6 relative of it (either answer
is right there); every kept pair's tallies must equal the oracle's and its CCC
values agree within 1e-6.
"""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import CCC_RTOL, assert_ccc_close, to_device, workspace

pytestmark = pytest.mark.gpu

HIT_DTYPE = np.dtype([("i", np.int32), ("j", np.int32), ("tally", np.int32, 4), ("ccc", np.float32, 4)])


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _filter(geno, n_f, path, threshold, cap, norm=0):
    import torch

    import paper_1705_08213_gb300 as ccc
    g = to_device(geno)
    opts = ccc.ccc_opts_default(path=path, norm=norm)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(path=path, norm=norm, workspace=ws)
    hits = torch.zeros(max(cap, 1) * HIT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n_hits = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    ccc.ccc2_filter(g, n_f, threshold, hits if cap > 0 else None, cap, n_hits, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    total = int(n_hits.item())
    rec = np.frombuffer(hits.cpu().numpy().tobytes(), dtype=HIT_DTYPE)[:min(total, cap)]
    return total, rec


def _expected(geno, n_f, threshold, norm=0):
    t, c = oracle.ccc2_all(geno, n_f, norm=norm)
    n_v = geno.shape[0]
    ii, jj = np.triu_indices(n_v, 1)
    mx = c.max(1)
    tie = np.abs(mx - threshold) <= CCC_RTOL * threshold
    keep = (mx > threshold) & ~tie
    return t, c, ii, jj, keep, tie


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("norm", [0, 1])
def test_filter_matches_oracle_set(path, norm):
    n_v, n_f, tau = 600, 1000, 0.155
    geno = synth.panel_hwe(n_v, n_f, seed=5, p_missing=0.01, pad_seed=2)
    synth.plant_near_duplicates(geno, n_f, 60, seed=17)
    t, c, ii, jj, keep, tie = _expected(geno, n_f, tau, norm)
    assert keep.sum() >= 10
    total, rec = _filter(geno, n_f, path, tau, cap=10000, norm=norm)
    assert total == len(rec)
    got = {(int(h["i"]), int(h["j"])) for h in rec}
    assert len(got) == len(rec)  # no pair twice
    want = {(int(i), int(j)) for i, j in zip(ii[keep], jj[keep])}
    either = {(int(i), int(j)) for i, j in zip(ii[tie], jj[tie])}
    assert want <= got <= want | either
    idx = oracle.pair_index(rec["i"].astype(np.int64), rec["j"].astype(np.int64), n_v)
    np.testing.assert_array_equal(rec["tally"], t[idx])
    assert_ccc_close(rec["ccc"], c[idx], what="hit CCC")
    assert np.all(rec["ccc"].max(1) > tau)


@pytest.mark.parametrize("path", [0, 1])
def test_filter_cap_and_count_only(path):
    n_v, n_f, tau = 300, 512, 0.155
    geno = synth.panel_hwe(n_v, n_f, seed=6, p_missing=0.01)
    synth.plant_near_duplicates(geno, n_f, 40, seed=18)
    _, _, ii, jj, keep, tie = _expected(geno, n_f, tau)
    n_keep = int(keep.sum())
    assert n_keep >= 8
    total, rec = _filter(geno, n_f, path, tau, cap=5)
    assert n_keep <= total <= n_keep + int(tie.sum())
    assert len(rec) == 5
    keep_set = {(int(i), int(j)) for i, j in zip(ii[keep | tie], jj[keep | tie])}
    assert {(int(h["i"]), int(h["j"])) for h in rec} <= keep_set
    total0, rec0 = _filter(geno, n_f, path, tau, cap=0)
    assert total0 == total and len(rec0) == 0
    # a threshold above every value keeps nothing; a negative one keeps every pair
    assert _filter(geno, n_f, path, 1.0, cap=4)[0] == 0
    assert _filter(geno, n_f, path, -1.0, cap=0)[0] == n_v * (n_v - 1) // 2


def test_filter_full_size_planted_pairs():
    """The large thresholded workload as bench.py runs it: 200,000 SNPs x 4,096 individuals,
    1,000 planted near-duplicate pairs, threshold 0.16.  Every kept pair is re-verified
    against the oracle (tallies exact, CCC within 1e-6); the kept set equals the oracle's
    set on the planted pairs and on sampled full rows of the triangle."""
    import torch

    import paper_1705_08213_gb300 as ccc
    n_v, n_f, tau = 200000, 4096, 0.16
    geno = synth.panel_hwe(n_v, n_f, seed=5, p_missing=0.01)
    planted = synth.plant_near_duplicates(geno, n_f, 1000, seed=1005)
    total, rec = _filter(geno, n_f, 0, tau, cap=1 << 16)
    assert total == len(rec) and total > 0
    pi = rec["i"].astype(np.int64)
    pj = rec["j"].astype(np.int64)
    et, ec = oracle.ccc2_pairs(geno, n_f, pi, pj)
    np.testing.assert_array_equal(rec["tally"], et)
    assert_ccc_close(rec["ccc"], ec, what="full-size hits")
    got = set(zip(pi.tolist(), pj.tolist()))
    # planted pairs: kept exactly when the oracle's max CCC exceeds the threshold
    a = np.minimum(planted[:, 0], planted[:, 1])
    b = np.maximum(planted[:, 0], planted[:, 1])
    _, pc = oracle.ccc2_pairs(geno, n_f, a, b)
    for x, y, m in zip(a.tolist(), b.tolist(), pc.max(1)):
        if abs(m - tau) > 1e-6 * tau:
            assert ((x, y) in got) == (m > tau), (x, y, m)
    # sampled rows of the triangle: the kept pairs of those rows are exactly the oracle's
    rows = np.array([0, 77777, 123456, 199998])
    rt, rc = oracle.ccc2_rows(geno, n_f, rows)
    o = 0
    for i in rows.tolist():
        js = np.arange(i + 1, n_v)
        mx = rc[o:o + js.size].max(1)
        sure = np.abs(mx - tau) > 1e-6 * tau
        want = {(i, int(j)) for j in js[(mx > tau) & sure]}
        either = {(i, int(j)) for j in js[~sure]}
        have = {p for p in got if p[0] == i}
        assert want <= have <= want | either
        o += js.size
