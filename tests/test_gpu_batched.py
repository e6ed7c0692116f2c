"""GPU batched 2-way panels (ccc2_batched): one persistent launch over many panels."""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_ccc_close, assert_tally_equal, run_2way, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_08213_gb300 import build
    build.build()


def _batch(shapes, seed):
    return [synth.panel_hwe(n_v, n_f, seed=seed, panel=k, p_missing=0.02, pad_seed=k)
            for k, (n_v, n_f) in enumerate(shapes)]


def _run_batched(genos_np, shapes, path=0, tune=False, group=0, order=0, split=0, solo=0,
                 operand=0, tile=0, opts_out=None):
    import torch

    import paper_1705_08213_gb300 as ccc
    genos = [to_device(g) for g in genos_np]
    n_fs = [n_f for _, n_f in shapes]
    tallies = [torch.full((max(ccc.ccc2_count(n_v), 1), 4), -7, dtype=torch.int32, device="cuda")
               for n_v, _ in shapes]
    cccs = [torch.full((max(ccc.ccc2_count(n_v), 1), 4), -7.0, dtype=torch.float32, device="cuda")
            for n_v, _ in shapes]
    opts = ccc.ccc_opts_default(path=path, operand=operand, tile=tile)
    opts.group, opts.order, opts.split, opts.solo = group, order, split, solo
    ws = torch.empty(ccc.ccc2_batched_workspace_size(genos, n_fs, opts), dtype=torch.uint8,
                     device="cuda")
    opts.workspace = ws.data_ptr()
    opts.workspace_bytes = ws.numel()
    if tune:
        g, o = ccc.ccc2_batched_tune(genos, n_fs, tallies, cccs, opts)
        assert g in (4, 8, 16) and o in (0, 1)
    else:
        ccc.ccc2_batched(genos, n_fs, tallies, cccs, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    if opts_out is not None:
        opts_out.append(opts)
    return ([t[:ccc.ccc2_count(n_v)].cpu().numpy() for t, (n_v, _) in zip(tallies, shapes)],
            [c[:ccc.ccc2_count(n_v)].cpu().numpy() for c, (n_v, _) in zip(cccs, shapes)])


@pytest.mark.parametrize("path", [0, 1])
def test_small_panels_against_oracle(path):
    shapes = [(130, 700), (1, 50), (2, 33), (65, 1000), (300, 129), (200, 4000)]
    genos = _batch(shapes, seed=51)
    ts, cs = _run_batched(genos, shapes, path=path)
    for g, (n_v, n_f), t, c in zip(genos, shapes, ts, cs):
        et, ec = oracle.ccc2_all(g, n_f)
        assert_tally_equal(t, et, f"panel n_v={n_v} n_f={n_f}")
        assert_ccc_close(c, ec, what=f"panel n_v={n_v} n_f={n_f}")


def test_batched_equals_single_calls_many_panels():
    rng = np.random.default_rng(3)
    shapes = [(int(rng.integers(2, 700)), int(rng.integers(1, 3000))) for _ in range(70)]
    genos = _batch(shapes, seed=52)
    for group, order in ((0, 0), (4, 1), (16, 0)):
        ts, cs = _run_batched(genos, shapes, group=group, order=order)
        for g, (n_v, n_f), t, c in zip(genos[:12], shapes[:12], ts[:12], cs[:12]):
            t1, c1 = run_2way(g, n_f, 0)
            np.testing.assert_array_equal(t, t1)
            np.testing.assert_array_equal(c, c1)
        for g, (n_v, n_f), t in zip(genos[60:], shapes[60:], ts[60:]):  # second launch chunk
            np.testing.assert_array_equal(t, run_2way(g, n_f, 0)[0])


def test_autotune_then_correct():
    shapes = [(500, 2000), (900, 3000), (260, 5000), (40, 100)]
    genos = _batch(shapes, seed=53)
    ts, cs = _run_batched(genos, shapes, tune=True)
    for g, (n_v, n_f), t, c in zip(genos, shapes, ts, cs):
        t1, c1 = run_2way(g, n_f, 0)
        np.testing.assert_array_equal(t, t1)
        np.testing.assert_array_equal(c, c1)


def test_cuda_graph_capture_and_replay():
    import torch

    import paper_1705_08213_gb300 as ccc
    shapes = [(300, 1000), (700, 2500), (64, 128)]
    genos_np = _batch(shapes, seed=54)
    genos = [to_device(g) for g in genos_np]
    n_fs = [n_f for _, n_f in shapes]
    tallies = [torch.zeros((ccc.ccc2_count(n_v), 4), dtype=torch.int32, device="cuda")
               for n_v, _ in shapes]
    cccs = [torch.zeros((ccc.ccc2_count(n_v), 4), dtype=torch.float32, device="cuda")
            for n_v, _ in shapes]
    opts = ccc.ccc_opts_default()
    ws = torch.empty(ccc.ccc2_batched_workspace_size(genos, n_fs, opts), dtype=torch.uint8,
                     device="cuda")
    opts = ccc.ccc_opts_default(workspace=ws)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ccc.ccc2_batched(genos, n_fs, tallies, cccs, opts, stream=s)  # first call outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        ccc.ccc2_batched(genos, n_fs, tallies, cccs, opts, stream=s)
    for t in tallies:
        t.zero_()
    for c in cccs:
        c.zero_()
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    for g, (n_v, n_f), t, c in zip(genos_np, shapes, tallies, cccs):
        et, ec = oracle.ccc2_all(g, n_f)
        assert_tally_equal(t.cpu().numpy(), et, "graph replay")
        assert_ccc_close(c.cpu().numpy(), ec, what="graph replay")


def test_batched_full_size_workload():
    """The batched workload as bench.py runs it: 64 panels, n_v ~ U{500..8000},
    n_f ~ U{2000..50000} (shape seed 2), Hardy-Weinberg (seed 2, panel index k).  The
    batched call equals one ccc2_tally_metric call per panel on every panel, and sampled
    rows of three panels equal the oracle."""
    import torch

    import paper_1705_08213_gb300 as ccc
    rng = np.random.default_rng(2)
    shapes = [(int(rng.integers(500, 8001)), int(rng.integers(2000, 50001))) for _ in range(64)]
    genos_np = [synth.panel_hwe(v, f, seed=2, panel=k, p_missing=0.01)
                for k, (v, f) in enumerate(shapes)]
    genos = [to_device(g) for g in genos_np]
    n_fs = [f for _, f in shapes]
    tallies = [torch.empty((ccc.ccc2_count(v), 4), dtype=torch.int32, device="cuda") for v, _ in shapes]
    cccs = [torch.empty((ccc.ccc2_count(v), 4), dtype=torch.float32, device="cuda") for v, _ in shapes]
    opts = ccc.ccc_opts_default()
    ws = torch.empty(ccc.ccc2_batched_workspace_size(genos, n_fs, opts), dtype=torch.uint8,
                     device="cuda")
    opts = ccc.ccc_opts_default(workspace=ws)
    ccc.ccc2_batched_tune(genos, n_fs, tallies, cccs, opts)
    ccc.ccc2_batched(genos, n_fs, tallies, cccs, opts)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    del ws
    o1 = ccc.ccc_opts_default()
    ws1 = torch.empty(max(ccc.ccc_workspace_size(g, f, o1, ccc.CCC_OP_2WAY)
                          for g, f in zip(genos, n_fs)), dtype=torch.uint8, device="cuda")
    o1 = ccc.ccc_opts_default(workspace=ws1)
    for g, f, t, c in zip(genos, n_fs, tallies, cccs):
        t1 = torch.empty_like(t)
        c1 = torch.empty_like(c)
        ccc.ccc2_tally_metric(g, f, t1, c1, o1)
        assert torch.equal(t1, t)
        assert torch.equal(c1, c)
        del t1, c1
    for k in (0, 31, 63):
        n_v, n_f = shapes[k]
        rows = np.array([0, n_v // 2, n_v - 2])
        et, ec = oracle.ccc2_rows(genos_np[k], n_f, rows)
        idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, n_v), n_v) for i in rows])
        it = torch.from_numpy(idx).cuda()
        assert_tally_equal(tallies[k][it].cpu().numpy(), et, f"panel {k}")
        assert_ccc_close(cccs[k][it].cpu().numpy(), ec, what=f"panel {k}")


def _tune_launches(genos_np, shapes):
    """Launches of one ccc2_batched_tune call, its choice and its results."""
    import paper_1705_08213_gb300 as ccc
    n0 = ccc.ccc_launch_count()
    t, c = _run_batched(genos_np, shapes, tune=True)
    return ccc.ccc_launch_count() - n0, t, c


def test_tune_cache_by_shape_buckets_and_file(tmp_path, monkeypatch):
    """ccc2_batched_tune times a dozen schedules and runs the chosen one.  A batch whose
    panel sizes fall in the same (n_v, n_f) power-of-two buckets then takes the cached
    choice and runs once; with CCC_TUNE_CACHE set the choice goes to a file that a cleared
    cache reads back.  Results stay those of the plain call."""
    import paper_1705_08213_gb300 as ccc
    shapes = [(300, 1000), (700, 2100), (1500, 600)]
    same_buckets = [(400, 1020), (600, 2050), (1100, 700)]
    genos = _batch(shapes, seed=31)
    genos_b = _batch(same_buckets, seed=32)
    ref_t, ref_c = _run_batched(genos, shapes)
    ccc.ccc_tune_cache_clear()
    first, t, c = _tune_launches(genos, shapes)
    for a, b in zip(t + c, ref_t + ref_c):
        np.testing.assert_array_equal(a, b)
    hit, _, _ = _tune_launches(genos, shapes)
    assert first > 5 * hit and hit > 0, (first, hit)
    hit_b, t_b, _ = _tune_launches(genos_b, same_buckets)
    assert hit_b < first / 2, (first, hit_b)
    et, _ = oracle.ccc2_all(genos_b[0], same_buckets[0][1])
    assert_tally_equal(t_b[0], et, "cached schedule")
    # the same through a file (the candidates a tuning run times depend on which one wins
    # each choice, so only "several runs" versus "one run" is compared)
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("CCC_TUNE_CACHE", str(path))
    ccc.ccc_tune_cache_clear()
    tuned = _tune_launches(genos, shapes)[0]
    assert tuned > 3 * hit, (tuned, hit)
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("ccc-tune-v2 ")
    f = lines[0].split()
    assert int(f[2]) in (4, 8, 16) and int(f[3]) in (0, 1) and int(f[4]) in (1, 2)
    assert int(f[5]) in (0, 1) and int(f[6]) in (-1, 512, 1024, 2048)
    ccc.ccc_tune_cache_clear()  # forget the process's copy: the file answers
    from_file, t_f, c_f = _tune_launches(genos, shapes)
    assert from_file < tuned / 3, (tuned, from_file)
    for a, b in zip(t_f + c_f, ref_t + ref_c):
        np.testing.assert_array_equal(a, b)
    assert len(path.read_text().splitlines()) == 1  # a cache hit appends nothing
    monkeypatch.delenv("CCC_TUNE_CACHE")
    ccc.ccc_tune_cache_clear()


def test_tune_stores_the_whole_schedule_in_opts():
    shapes = [(500, 2000), (260, 9000), (40, 100)]
    genos = _batch(shapes, seed=55)
    got = []
    ts, cs = _run_batched(genos, shapes, tune=True, opts_out=got)
    o = got[0]
    assert o.tile in (1, 2) and o.split in (0, 1) and o.solo in (-1, 512, 1024, 2048)
    assert o.group in (4, 8, 16) and o.order in (0, 1)
    for g, (n_v, n_f), t, c in zip(genos, shapes, ts, cs):
        et, ec = oracle.ccc2_all(g, n_f)
        assert_tally_equal(t, et, f"tuned n_v={n_v}")
        assert_ccc_close(c, ec, what=f"tuned n_v={n_v}")


def test_batched_fp4_equals_e4m3():
    import paper_1705_08213_gb300 as ccc
    rng = np.random.default_rng(5)
    shapes = [(int(rng.integers(2, 900)), int(rng.integers(1, 6000))) for _ in range(20)]
    genos = _batch(shapes, seed=56)
    t4, c4 = _run_batched(genos, shapes, operand=ccc.CCC_OPERAND_E2M1)
    t8, c8 = _run_batched(genos, shapes, operand=ccc.CCC_OPERAND_E4M3)
    for a, b in zip(t4 + c4, t8 + c8):
        np.testing.assert_array_equal(a, b)
    for g, (n_v, n_f), t in zip(genos[:5], shapes[:5], t4[:5]):
        assert_tally_equal(t, oracle.ccc2_all(g, n_f)[0], f"fp4 batched n_v={n_v}")


@pytest.mark.parametrize("operand", [0, 1])
def test_batched_k_split_in_the_shared_launch(operand):
    """Few small panels with long vectors: the shared launch has 8 SM-pair tiles for 76 SM
    pairs, so its tiles run as K parts (automatic), whose summed tallies and CCC values equal
    the oracle; every split setting gives the same results."""
    shapes = [(300, 40000), (200, 30000), (130, 50000)]
    genos = _batch(shapes, seed=57)
    ref = [oracle.ccc2_all(g, f) for g, (_, f) in zip(genos, shapes)]
    outs = {}
    for split in (0, 1, 5):
        outs[split] = _run_batched(genos, shapes, split=split, operand=operand)
    for k, (et, ec) in enumerate(ref):
        assert_tally_equal(outs[0][0][k], et, f"auto split panel {k}")
        assert_ccc_close(outs[0][1][k], ec, what=f"auto split panel {k}")
        for split in (1, 5):
            np.testing.assert_array_equal(outs[split][0][k], outs[0][0][k])
            np.testing.assert_array_equal(outs[split][1][k], outs[0][1][k])


def test_batched_solo_thresholds_agree():
    # One panel of 300 SM-pair tiles beside small ones: solo 100 runs it alone, the default
    # (1024) and -1 put it in the shared launch.
    shapes = [(3000, 1500), (200, 800), (90, 300), (500, 2100)]
    genos = _batch(shapes, seed=58)
    outs = [_run_batched(genos, shapes, solo=solo) for solo in (0, 100, -1)]
    for k, (g, (n_v, n_f)) in enumerate(zip(genos, shapes)):
        for o in outs[1:]:
            np.testing.assert_array_equal(o[0][k], outs[0][0][k])
            np.testing.assert_array_equal(o[1][k], outs[0][1][k])
    rows = np.array([0, 1500, 2998])
    et, ec = oracle.ccc2_rows(genos[0], 1500, rows)
    idx = np.concatenate([oracle.pair_index(i, np.arange(i + 1, 3000), 3000) for i in rows])
    assert_tally_equal(outs[1][0][0][idx], et, "solo panel rows")
    assert_ccc_close(outs[1][1][0][idx], ec, what="solo panel rows")
