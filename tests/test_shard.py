"""The rank partition of paper_1705_08213_gb300.shard, on CPU ranks.

* Index level, for many shapes and world sizes: the ranges of all ranks are
  contiguous, cover the triangle (tetrahedron) exactly once and balance work.
* Two gloo processes (world size 2): each computes its shard of one panel with
  the oracle (2-way rows, 3-way slabs, multi-allelic rows), the shards are
  gathered, and rank 0 checks that their concatenation in rank order is the
  full result, with no pair or triple twice; the max-over-ranks timing
  reduction of the benchmark runs over the same process group.
* The individuals axis (n_pf, Sec. 4): two gloo ranks tally their slices of
  the individuals and an all-reduce sums the partial tallies; the sum equals
  the tallies over all individuals.
"""

import os

import numpy as np
import pytest

from paper_1705_08213_gb300 import build as cbuild


@pytest.fixture(scope="module", autouse=True)
def _lib():
    cbuild.build()


def _pairs(n_v, i0, i1):
    return sum(n_v - 1 - i for i in range(i0, i1))


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_ranges_cover_once_and_balance(world):
    from paper_1705_08213_gb300 import shard
    for n_v in (1, 2, 3, 65, 300, 4096, 20000):
        r2 = [shard.pair_range(n_v, world, r) for r in range(world)]
        assert r2[0][0] == 0 and r2[-1][1] == n_v
        assert all(a[1] == b[0] for a, b in zip(r2, r2[1:]))
        counts = [_pairs(n_v, a, b) for a, b in r2]
        assert sum(counts) == n_v * (n_v - 1) // 2
        offs = [shard.pair_offset(n_v, a) for a, _ in r2]
        assert offs == list(np.cumsum([0] + counts[:-1]))
        if n_v >= 4096:
            assert max(counts) <= 1.15 * sum(counts) / world
        r3 = [shard.slab_range(n_v, world, r) for r in range(world)]
        assert r3[0][0] == 0 and r3[-1][1] == n_v
        assert all(a[1] == b[0] for a, b in zip(r3, r3[1:]))
        t3 = [shard.triple_offset(n_v, b) - shard.triple_offset(n_v, a) for a, b in r3]
        assert sum(t3) == n_v * (n_v - 1) * (n_v - 2) // 6
        if n_v >= 4096:
            assert max(t3) <= 1.05 * sum(t3) / world
        for s in (2, 4, 7):
            rm = [shard.multi_pair_range(n_v, s, world, r) for r in range(world)]
            assert rm[0][0] == 0 and rm[-1][1] == n_v
            assert all(a[1] == b[0] for a, b in zip(rm, rm[1:]))
            assert all(a % (8 * (32 // s)) == 0 for a, _ in rm[1:] if a < n_v)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1705_08213_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_v, n_f = 90, 200
        geno = synth.panel_hwe(n_v, n_f, seed=3, p_missing=0.02)
        i0, i1 = shard.pair_range(n_v, world, rank)
        t2, c2 = oracle.ccc2_rows(geno, n_f, np.arange(i0, i1))
        ii = np.concatenate([np.full(n_v - 1 - i, i) for i in range(i0, i1)] or [np.zeros(0, int)])
        jj = np.concatenate([np.arange(i + 1, n_v) for i in range(i0, i1)] or [np.zeros(0, int)])
        n3 = 30
        g3 = np.ascontiguousarray(geno[:n3])
        j0, j1 = shard.slab_range(n3, world, rank)
        t3, c3 = oracle.ccc3_slabs(g3, n_f, j0, j1)
        s, nm = 4, 70
        gm = synth.panel_multi(nm, n_f, s, seed=4, p_missing=0.02)
        m0, m1 = shard.multi_pair_range(nm, s, world, rank)
        tm, cm = oracle.ccc2_multi_rows(gm, n_f, s, np.arange(m0, m1))
        mine = {"rank": rank, "t2": t2, "c2": c2, "ij": (ii, jj), "off2": shard.pair_offset(n_v, i0),
                "t3": t3, "c3": c3, "off3": shard.triple_offset(n3, j0), "tm": tm, "cm": cm}
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        import torch
        t = torch.tensor([10.0 + rank])  # per-rank step time
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            full2 = oracle.ccc2_all(geno, n_f)
            full3 = oracle.ccc3_slabs(g3, n_f)
            fullm = oracle.ccc2_multi_all(gm, n_f, s)
            res = {
                "t2": np.concatenate([g["t2"] for g in gathered]),
                "c2": np.concatenate([g["c2"] for g in gathered]),
                "off2": [g["off2"] for g in gathered],
                "pairs": np.concatenate([np.stack(g["ij"], 1) for g in gathered]),
                "t3": np.concatenate([g["t3"] for g in gathered]),
                "c3": np.concatenate([g["c3"] for g in gathered]),
                "off3": [g["off3"] for g in gathered],
                "tm": np.concatenate([g["tm"] for g in gathered]),
                "cm": np.concatenate([g["cm"] for g in gathered]),
                "full2": full2, "full3": full3, "fullm": fullm, "tmax": float(t.item()),
                "n_v": n_v,
            }
            np.save(os.path.join(out_dir, "res.npy"), np.array([res], dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_the_full_result(tmp_path):
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    world = 2
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = np.load(tmp_path / "res.npy", allow_pickle=True)[0]
    t2, c2 = res["full2"]
    np.testing.assert_array_equal(res["t2"], t2)
    np.testing.assert_array_equal(res["c2"], c2)
    n_v = res["n_v"]
    pairs = res["pairs"]
    assert len({(int(i), int(j)) for i, j in pairs}) == len(pairs) == n_v * (n_v - 1) // 2
    assert res["off2"][0] == 0 and res["off2"][1] == len(res["t2"]) - (len(t2) - res["off2"][1])
    t3, c3 = res["full3"]
    np.testing.assert_array_equal(res["t3"], t3)
    np.testing.assert_array_equal(res["c3"], c3)
    tm, cm = res["fullm"]
    np.testing.assert_array_equal(res["tm"], tm)
    np.testing.assert_array_equal(res["cm"], cm)
    assert res["tmax"] == 11.0


def test_field_ranges_cover_the_individuals():
    from paper_1705_08213_gb300 import shard
    for n_f in (1, 63, 64, 65, 1000, 16384, 100000):
        for world in (1, 2, 3, 8):
            r = [shard.field_range(n_f, world, k) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == n_f
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            assert all(a % 64 == 0 for a, _ in r)
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 64 + (n_f % 64)


def _field_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1705_08213_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_v, n_f = 60, 1000
        geno = synth.panel_hwe(n_v, n_f, seed=8, p_missing=0.03)
        q0, q1 = shard.field_range(n_f, world, rank)
        # this rank's individuals: whole words from q0 (a multiple of 64) on
        sl = np.ascontiguousarray(geno[:, q0 // 32:])
        t2, _ = oracle.ccc2_all(sl, q1 - q0)
        t3, _ = oracle.ccc3_slabs(np.ascontiguousarray(sl[:25]), q1 - q0)
        p2 = torch.from_numpy(t2.copy())
        p3 = torch.from_numpy(t3.copy())
        shard.allreduce_tallies(p2)
        shard.allreduce_tallies(p3)
        if rank == 0:
            np.save(os.path.join(out_dir, "field.npy"),
                    np.array([{"t2": p2.numpy(), "t3": p3.numpy(),
                               "full2": oracle.ccc2_all(geno, n_f)[0],
                               "full3": oracle.ccc3_slabs(np.ascontiguousarray(geno[:25]), n_f)[0]}],
                             dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_field_slices(tmp_path):
    """The n_pf axis: each rank tallies its slice of the individuals, an all-reduce sums the
    partial tallies; the sum equals the tallies over all individuals (2-way and 3-way)."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.start_processes(_field_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = np.load(tmp_path / "field.npy", allow_pickle=True)[0]
    np.testing.assert_array_equal(res["t2"], res["full2"])
    np.testing.assert_array_equal(res["t3"], res["full3"])


# ---------------------------------------------------------------- block-circulant (n_pv axis)


@pytest.mark.parametrize("world", [1, 2, 3, 4, 5, 8])
def test_circulant_blocks_cover_every_pair_once(world):
    """Sec. 4's block-circulant subset: every unordered pair of vector blocks (and every
    diagonal block) lies in exactly one rank's block row, every pair i < j of the triangle
    is computed once, and a rank holds only the blocks of its row (about half the panel)."""
    from paper_1705_08213_gb300 import shard
    blocks_seen = {}
    for r in range(world):
        for q in shard.circulant_plan(1000, world, r)["blocks"]:
            key = (min(r, q), max(r, q))
            blocks_seen[key] = blocks_seen.get(key, 0) + 1
    assert sorted(blocks_seen) == [(p, q) for p in range(world) for q in range(p, world)]
    assert all(v == 1 for v in blocks_seen.values())
    for n_v in (1, 2, 129, 700, 4096):
        b = shard.vector_blocks(n_v, world)
        counts = np.zeros(n_v * (n_v - 1) // 2, np.int64)
        held = []
        work = []
        for r in range(world):
            plan = shard.circulant_plan(n_v, world, r)
            lo, hi, swap = shard.circulant_pairs(plan)
            assert np.all(lo < hi)
            np.add.at(counts, lo * (2 * n_v - lo - 1) // 2 + (hi - lo - 1), 1)
            held.append(plan["snps"].size)
            work.append(lo.size)
            assert len(plan["blocks"]) <= world // 2 + 1
            assert np.array_equal(plan["snps"][:plan["rows"][1]], np.arange(b[r], b[r + 1]))
        assert np.all(counts == 1)
        if n_v >= 4096 and world > 2:
            assert max(held) <= (world // 2 + 1) * (n_v / world + 128)
            assert max(work) <= 1.6 * sum(work) / world


def _circulant_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_1705_08213_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_v, n_f = 300, 500
        geno = synth.panel_hwe(n_v, n_f, seed=9, p_missing=0.03)
        plan = shard.circulant_plan(n_v, world, rank)
        local = shard.circulant_local_panel(geno, plan)  # the only vectors this rank holds
        t, c = oracle.ccc2_rows(np.ascontiguousarray(local), n_f, np.arange(*plan["rows"]))
        idx, t, c = shard.circulant_scatter(plan, t, c)
        mine = {"idx": idx, "t": t, "c": c, "held": local.shape[0]}
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        tm = torch.tensor([float(rank)])
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        if rank == 0:
            et, ec = oracle.ccc2_all(geno, n_f)
            np.save(os.path.join(out_dir, "circ.npy"),
                    np.array([{"parts": gathered, "et": et, "ec": ec, "n_v": n_v,
                               "tmax": float(tm.item())}], dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_block_circulant(tmp_path):
    """Two ranks, each holding only its block row's vectors: the union of their result
    blocks is the full triangle, each pair once, equal to the oracle on the full panel."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.start_processes(_circulant_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = np.load(tmp_path / "circ.npy", allow_pickle=True)[0]
    n_v = res["n_v"]
    idx = np.concatenate([p["idx"] for p in res["parts"]])
    assert idx.size == n_v * (n_v - 1) // 2 and np.unique(idx).size == idx.size
    t = np.concatenate([p["t"] for p in res["parts"]])
    c = np.concatenate([p["c"] for p in res["parts"]])
    np.testing.assert_array_equal(t, res["et"][idx])
    np.testing.assert_allclose(c, res["ec"][idx], rtol=1e-12, atol=0)
    assert all(p["held"] < n_v for p in res["parts"][1:]) or len(res["parts"]) == 1
    assert res["tmax"] == 1.0
