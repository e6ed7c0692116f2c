"""Coverage of the 2-way tile orders on the host (no GPU).

The SM-pair tally kernels visit the upper triangle of the Gram product R R^T
(Sec. 3.1: only pairs i < j, by the symmetry of Sec. 2.1) as a persistent grid:
cluster c takes tiles c, c + clusters, ...  tests/host/sched_order.cu prints
that visit order from the kernels' own scheduler code compiled for the host;
here every pair i < j of the rows asked for must fall in exactly one visited
tile, and every visited tile must hold at least one pair (no wasted tile
beyond the partial last blocks)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sched_bin(tmp_path_factory):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("sched") / "sched_order")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
                    "-I", os.path.join(ROOT, "paper_1705_08213_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "sched_order.cu"), "-o", out], check=True,
                   capture_output=True)
    return out


def visits(binary, kind, n_v, I0, I1, group, clusters):
    p = subprocess.run([binary, str(kind), str(n_v), str(I0), str(I1), str(group), str(clusters)],
                       check=True, capture_output=True, text=True)
    a = np.array([list(map(int, l.split())) for l in p.stdout.split("\n") if l], dtype=np.int64)
    return a.reshape(-1, 3)


CASES = [(2, 0, 1, 8, 1), (129, 0, 2, 8, 3), (1000, 0, 8, 4, 3), (1000, 2, 5, 16, 7),
         (2049, 0, 17, 16, 76), (3000, 0, 24, 1, 5), (3000, 7, 24, 32, 2), (241, 0, 2, 16, 1),
         (3840, 0, 30, 16, 11)]


# (SNPs per row block, per column block) of each tile kind of sched_order.cu
SHAPES = {0: (128, 128), 1: (128, 120), 2: (64, 48), 3: (80, 60)}


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
@pytest.mark.parametrize("n_v,I0,I1,group,clusters", CASES)
def test_tile_order_covers_triangle_once(sched_bin, kind, n_v, I0, I1, group, clusters):
    snpi, snpj = SHAPES[kind]
    v = visits(sched_bin, kind, n_v, I0, I1, group, clusters)
    tiles = [tuple(t) for t in v[:, 1:]]
    assert len(set(tiles)) == len(tiles), "a tile visited twice"
    # cluster c's visits are its share of the strided order: the counts differ by at most one
    counts = np.bincount(v[:, 0], minlength=clusters)
    assert counts.max() - counts.min() <= 1
    cover = np.zeros((n_v, n_v), dtype=np.int32)
    for I, J in tiles:
        i0, i1 = snpi * I, min(snpi * I + snpi, n_v)
        j0, j1 = snpj * J, min(snpj * J + snpj, n_v)
        assert 0 <= I < (n_v + snpi - 1) // snpi and 0 <= J < (n_v + snpj - 1) // snpj
        ii, jj = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), indexing="ij")
        m = ii < jj
        if i1 - i0 > 1 or j1 - j0 > 1:
            # a tile holds a pair unless only the partial last blocks make it empty
            assert m.any() or i1 == n_v or j1 == n_v
        cover[ii[m], jj[m]] += 1
    rows = np.zeros(n_v, dtype=bool)
    rows[snpi * I0:min(snpi * I1, n_v)] = True
    want = np.triu(np.ones((n_v, n_v), dtype=np.int32), 1) * rows[:, None]
    np.testing.assert_array_equal(cover, want)
