"""The C ABI library loads and exports every symbol that include/ccc.h declares.

Host-only calls (index helpers, workspace sizing, argument checks that fail
before any device work) run here without a GPU.
"""

import ctypes
import os
import re
import subprocess

import pytest

import paper_1705_08213_gb300 as ccc
from paper_1705_08213_gb300 import build as cbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ccc.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    cbuild.build()
    return ccc.load()


def declared_functions(headers=(HEADER,)):
    text = "".join(open(h).read() for h in headers)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("ccc_allele_counts", "ccc2_tally", "ccc2_metric", "ccc2_tally_metric", "ccc3_tally",
              "ccc3_metric", "ccc3_tally_metric", "ccc_workspace_size", "ccc_status",
              "ccc2_index", "ccc3_index", "ccc_strerror", "ccc_launch_count"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", ccc.lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions(HEADERS) if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_python_binding_names_match_header():
    for n in declared_functions(HEADERS):
        assert hasattr(ccc, n), n


def test_index_helpers(lib):
    n_v = 11
    t = 0
    for i in range(n_v):
        for j in range(i + 1, n_v):
            assert ccc.ccc2_index(i, j, n_v) == t
            t += 1
    assert ccc.ccc2_count(n_v) == t
    assert ccc.ccc2_index(3, 3, n_v) == -1
    t = 0
    for j in range(n_v):
        for i in range(j):
            for k in range(j + 1, n_v):
                assert ccc.ccc3_index(i, j, k, n_v) == t
                t += 1
    assert ccc.ccc3_count(n_v, 0, n_v) == t
    assert ccc.ccc3_count(n_v, 3, 7) == ccc.ccc3_index(0, 7, 8, n_v) - ccc.ccc3_index(0, 3, 4, n_v)
    assert ccc.ccc3_index(2, 1, 5, n_v) == -1


def test_opts_default_and_strerror(lib):
    o = ccc.ccc_opts_default()
    assert o.path == ccc.CCC_PATH_TC and o.norm == ccc.CCC_NORM_PERSNP
    assert abs(o.gamma - 2.0 / 3.0) < 1e-16
    assert ccc.ccc_strerror(ccc.CCC_ETIMEOUT) == "device-side wait timed out"
    assert ccc.ccc_strerror(12345) == "unknown status"


def test_workspace_size(lib):
    o = ccc.ccc_opts_default(operand=ccc.CCC_OPERAND_E4M3)
    tc = ccc.ccc_workspace_size((1000, 32), 2000, o, ccc.CCC_OP_2WAY)
    # e4m3 operand matrix: (round_up(2000, 256) + 256) rows x round_up(2000, 128) bytes dominates
    assert tc >= (2048 + 256) * 2048
    # e2m1 (the automatic choice for SM-pair tiles): rows of round_up(2000, 256) / 2 bytes
    fp4 = ccc.ccc_workspace_size((1000, 32), 2000, ccc.ccc_opts_default(), ccc.CCC_OP_2WAY)
    assert (2048 + 256) * 1024 <= fp4 < tc
    assert fp4 == ccc.ccc_workspace_size((1000, 32), 2000,
                                         ccc.ccc_opts_default(operand=ccc.CCC_OPERAND_E2M1),
                                         ccc.CCC_OP_2WAY)
    # one-SM tiles have no FP4 variant: automatic = e4m3
    assert tc == ccc.ccc_workspace_size((1000, 32), 2000, ccc.ccc_opts_default(tile=1),
                                        ccc.CCC_OP_2WAY)
    o.path = ccc.CCC_PATH_POPC
    pc = ccc.ccc_workspace_size((1000, 32), 2000, o, ccc.CCC_OP_2WAY)
    assert pc >= 1000 * 32 * 32
    m = ccc.ccc_workspace_size((1000, 32), 2000, o, ccc.CCC_OP_METRIC)
    assert 1000 * 8 <= m < pc
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc_workspace_size((0, 2), 10, o, ccc.CCC_OP_2WAY)
    assert e.value.status == ccc.CCC_EINVAL
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc_workspace_size((10, 2), ccc.CCC_MAX_NF + 1, o, ccc.CCC_OP_2WAY)
    assert e.value.status == ccc.CCC_ERANGE
    o.path = 7
    with pytest.raises(ccc.CCCError):
        ccc.ccc_workspace_size((10, 2), 10, o, ccc.CCC_OP_2WAY)


def test_workspace_size_3way_variants(lib):
    """3-way tile variants: the genotype-class route (automatic, tile 3) holds the 2-way
    tallies of all pairs and per-slab compacted rows (2 n_v rows x 256 bytes); the
    masked-operand route (tile 1) holds L_j batches.  2-way tile 3 (the codes expanded in
    shared memory by the tally kernel) holds no e4m3 operand matrix."""
    n_v, ld, n_f = 1536, 256, 8192
    sizes = {}
    for tile in (0, 1, 2, 3):
        o = ccc.ccc_opts_default(tile=tile)
        sizes[tile] = ccc.ccc_workspace_size((n_v, ld), n_f, o, ccc.CCC_OP_3WAY)
    assert sizes[0] == sizes[3]
    assert sizes[3] >= 16 * n_v * (n_v - 1) // 2 + n_v * 2 * n_v * 256
    assert sizes[2] < sizes[1] and sizes[2] < sizes[3]
    w3 = ccc.ccc_workspace_size((n_v, ld), n_f, ccc.ccc_opts_default(tile=3), ccc.CCC_OP_2WAY)
    w2 = ccc.ccc_workspace_size((n_v, ld), n_f,
                                ccc.ccc_opts_default(tile=2, operand=ccc.CCC_OPERAND_E4M3),
                                ccc.CCC_OP_2WAY)
    assert w2 - w3 >= 2 * n_v * n_f  # (2 n_v rows) x (n_f bytes) of e4m3 counts
    w2f = ccc.ccc_workspace_size((n_v, ld), n_f, ccc.ccc_opts_default(tile=2), ccc.CCC_OP_2WAY)
    assert w2f - w3 >= n_v * n_f  # (2 n_v rows) x (n_f / 2 bytes) of e2m1 counts
    o = ccc.ccc_opts_default(tile=3)
    o.tile = 4
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc_workspace_size((n_v, ld), n_f, o, ccc.CCC_OP_3WAY)
    assert e.value.status == ccc.CCC_EINVAL
    o = ccc.ccc_opts_default(operand=3)
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc_workspace_size((n_v, ld), n_f, o, ccc.CCC_OP_2WAY)
    assert e.value.status == ccc.CCC_EINVAL


def test_argument_errors_before_device_work(lib):
    o = ccc.ccc_opts_default()
    P = ctypes.POINTER
    # null panel / bad stride / odd ld / n_f too large: rejected before any device call
    assert lib.ccc2_tally(None, None, ctypes.byref(o), None) == ccc.CCC_EINVAL
    p = ccc.ccc_panel(16, 100, 10, 3)  # ld odd
    assert lib.ccc2_tally(ctypes.byref(p), ctypes.c_void_p(256), ctypes.byref(o), None) == ccc.CCC_EINVAL
    p = ccc.ccc_panel(16, 100, 10, 2)  # ld < ceil(100/32) = 4
    assert lib.ccc2_tally(ctypes.byref(p), ctypes.c_void_p(256), ctypes.byref(o), None) == ccc.CCC_EINVAL
    p = ccc.ccc_panel(8, 100, 10, 4)  # misaligned genotype pointer
    assert lib.ccc2_tally(ctypes.byref(p), ctypes.c_void_p(256), ctypes.byref(o), None) == ccc.CCC_EINVAL
    p = ccc.ccc_panel(16, ccc.CCC_MAX_NF + 1, 10, 65536)
    assert lib.ccc2_tally(ctypes.byref(p), ctypes.c_void_p(256), ctypes.byref(o), None) == ccc.CCC_ERANGE
    p = ccc.ccc_panel(16, 100, 10, 4)
    assert lib.ccc3_tally(ctypes.byref(p), 5, 3, ctypes.c_void_p(256), ctypes.byref(o), None) == ccc.CCC_EINVAL
    assert lib.ccc3_tally(ctypes.byref(p), 0, 11, ctypes.c_void_p(256), ctypes.byref(o), None) == ccc.CCC_EINVAL
    o.norm = 5
    assert lib.ccc2_tally(ctypes.byref(p), ctypes.c_void_p(256), ctypes.byref(o), None) == ccc.CCC_EINVAL
    o = ccc.ccc_opts_default()
    o.gamma = -0.5
    assert lib.ccc2_metric(ctypes.c_void_p(256), ctypes.c_void_p(256), 10, ctypes.byref(o),
                           ctypes.c_void_p(256), None) == ccc.CCC_EINVAL


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(ccc, "_lib", None)
    monkeypatch.setattr(ccc, "lib_path", str(tmp_path / "nope.so"))
    with pytest.raises(ccc.CCCError):
        ccc.load()


def test_phase_bounds_and_row_counts(lib):
    for n_v in (1, 2, 63, 64, 65, 300, 20000, 200000):
        total = ccc.ccc2_count(n_v)
        assert ccc.ccc2_rows_count(n_v, 0, n_v) == total
        for n_ph in (1, 2, 3, 7, 64):
            b = ccc.ccc2_phase_bounds(n_v, n_ph)
            assert b[0] == 0 and b[-1] == n_v and all(x <= y for x, y in zip(b, b[1:]))
            assert all(x % 64 == 0 or x == n_v for x in b[1:-1])
            counts = [ccc.ccc2_rows_count(n_v, x, y) for x, y in zip(b, b[1:])]
            assert sum(counts) == total
            if n_v >= 20000:  # balanced to within one 64-row band
                assert max(counts) - min(counts) <= 2 * 64 * n_v
    assert ccc.ccc2_rows_count(10, 3, 2) == -1
    o = ccc.ccc_opts_default()
    a = ccc.ccc2_stream_workspace_size((20000, 512), 16384, 8, o)
    assert a > ccc.ccc_workspace_size((20000, 512), 16384, o, ccc.CCC_OP_2WAY)


def test_phase_bounds_3way(lib):
    """Slab ranges of ccc3_stream: contiguous, covering, about equal triple counts."""
    for n_v in (1, 2, 3, 40, 1536, 5000):
        total = ccc.ccc3_count(n_v, 0, n_v)
        for n_ph in (1, 2, 5, 8, 64):
            b = ccc.ccc3_phase_bounds(n_v, n_ph)
            assert b[0] == 0 and b[-1] == n_v and all(x <= y for x, y in zip(b, b[1:]))
            counts = [ccc.ccc3_count(n_v, x, y) for x, y in zip(b, b[1:])]
            assert sum(counts) == total
            if n_v >= 1536:  # within one slab of the even split
                assert max(counts) - total / n_ph <= n_v * n_v / 4 + 1
    o = ccc.ccc_opts_default()
    base = ccc.ccc_workspace_size((1536, 256), 8192, o, ccc.CCC_OP_3WAY)
    ws = ccc.ccc3_stream_workspace_size((1536, 256), 8192, 8, o)
    # two staging slots of the largest phase, 64 bytes per triple
    assert ws >= base + 2 * 64 * (ccc.ccc3_count(1536, 0, 1536) // 8)


def test_multi_workspace_size(lib):
    """Markers with s states: the operand holds 32 rows per floor(32 / s) markers, padded to
    256-row blocks, of round_up(n_f, 128) bytes; the popcount path is not offered."""
    o = ccc.ccc_opts_default()
    n_v, n_f = 1000, 2000
    for s, per_quarter in ((2, 16), (3, 10), (4, 8), (5, 6), (8, 4), (9, 3), (15, 2)):
        rows = -(-n_v // per_quarter) * 32
        rows = -(-rows // 256) * 256
        size = ccc.ccc_multi_workspace_size((n_v, 2000), n_f, s, o)
        assert rows * 2048 <= size < rows * 2048 + n_v * s * 4 + 4096, s
    for bad_s in (1, 16):
        with pytest.raises(ccc.CCCError) as e:
            ccc.ccc_multi_workspace_size((n_v, 2000), n_f, bad_s, o)
        assert e.value.status == ccc.CCC_EINVAL
    o.path = ccc.CCC_PATH_POPC
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc_multi_workspace_size((n_v, 2000), n_f, 4, o)
    assert e.value.status == ccc.CCC_EUNSUPPORTED
    o = ccc.ccc_opts_default(tile=1)
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc_multi_workspace_size((n_v, 2000), n_f, 4, o)
    assert e.value.status == ccc.CCC_EINVAL


def test_multi_argument_errors_before_device_work(lib):
    o = ccc.ccc_opts_default()
    t = ctypes.c_void_p(256)
    M = ccc.ccc_panel_multi
    assert lib.ccc2_multi_tally(None, t, ctypes.byref(o), None) == ccc.CCC_EINVAL
    for p in (M(16, 100, 10, 104, 4, 0),      # ld not a multiple of 16
              M(16, 100, 10, 96, 4, 0),       # ld < n_f
              M(8, 100, 10, 112, 4, 0),       # misaligned entries
              M(16, 100, 10, 112, 1, 0),      # s < 2
              M(16, 100, 10, 112, 16, 0),     # s > 15
              M(16, 0, 10, 112, 4, 0)):       # no individuals
        assert lib.ccc2_multi_tally(ctypes.byref(p), t, ctypes.byref(o), None) == ccc.CCC_EINVAL
    p = M(16, ccc.CCC_MAX_NF + 1, 10, 1 << 22, 4, 0)
    assert lib.ccc2_multi_tally(ctypes.byref(p), t, ctypes.byref(o), None) == ccc.CCC_ERANGE
    p = M(16, 100, 10, 112, 4, 0)
    assert lib.ccc2_multi_tally(ctypes.byref(p), ctypes.c_void_p(260), ctypes.byref(o), None) \
        == ccc.CCC_EINVAL  # tally not 16-byte aligned
    assert lib.ccc2_multi_tally_metric(ctypes.byref(p), t, None, ctypes.byref(o), None) == ccc.CCC_EINVAL
    o.path = ccc.CCC_PATH_POPC
    assert lib.ccc2_multi_tally(ctypes.byref(p), t, ctypes.byref(o), None) == ccc.CCC_EUNSUPPORTED
    o = ccc.ccc_opts_default()
    assert lib.ccc2_multi_metric(t, t, 10, 16, ctypes.byref(o), t, None) == ccc.CCC_EINVAL
    assert lib.ccc2_multi_metric(None, t, 10, 4, ctypes.byref(o), t, None) == ccc.CCC_EINVAL


def test_multi_phase_bounds(lib):
    """Phase bounds for markers with s states: cover [0, n_v], inner bounds on multiples of
    8 floor(32 / s) markers (a 256-row operand block), pair counts about equal."""
    for s, n_v, n_phases in ((4, 10000, 8), (3, 777, 5), (15, 100, 3), (2, 5, 4)):
        b = ccc.ccc2_multi_phase_bounds(n_v, s, n_phases)
        assert b[0] == 0 and b[-1] == n_v
        assert all(x <= y for x, y in zip(b, b[1:]))
        step = 8 * (32 // s)
        assert all(x % step == 0 for x in b[1:-1] if x < n_v)
        counts = [ccc.ccc2_rows_count(n_v, x, y) for x, y in zip(b, b[1:])]
        assert sum(counts) == n_v * (n_v - 1) // 2
        if n_v >= 1000:
            assert max(counts) <= 1.6 * (sum(counts) / n_phases)
    with pytest.raises(ccc.CCCError):
        ccc.ccc2_multi_phase_bounds(10, 16, 2)


def test_bounded_wait_selftest_arguments(lib):
    assert lib.ccc_check_bounded_wait(None, 10000000, None) == ccc.CCC_EINVAL
    for bad in (0, 999999, 2000000001):
        assert lib.ccc_check_bounded_wait(ctypes.c_void_p(256), bad, None) == ccc.CCC_EINVAL


def test_checked_build_exports_the_same_entry_points_and_its_hook(lib):
    """The bounds-checking build (-DCCC_BOUNDS_CHECK, include/ccc_checked.h) exports every
    entry point of include/*.h; its hook works there and returns CCC_EUNSUPPORTED from the
    normal build."""
    checked = cbuild.build(checked=True)

    def exported(path):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                             check=True).stdout
        return {ln.split()[-1] for ln in out.splitlines() if ln.strip()}

    names = exported(checked)
    for n in declared_functions():
        assert n in names, n
    for n in declared_functions(HEADERS):
        assert n in names, n
    hook = ctypes.CDLL(checked).ccc_checked_shrink_outputs
    hook.argtypes = [ctypes.c_int64]
    assert hook(-1) == ccc.CCC_EINVAL
    assert hook(0) == ccc.CCC_OK
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc_checked_shrink_outputs(3)  # this process loaded the normal build
    assert e.value.status == ccc.CCC_EUNSUPPORTED


def test_binding_refuses_outputs_smaller_than_the_call_writes():
    """The Python binding checks every output tensor's size before the library writes
    through the raw pointer (a (pairs, 4) array for an s-state call would be overrun)."""
    import torch
    n_v = 10
    npairs = ccc.ccc2_count(n_v)
    geno = torch.zeros((n_v, 32), dtype=torch.int64)
    o = ccc.ccc_opts_default()
    small = torch.zeros((npairs - 1, 4), dtype=torch.int32)
    for call in (lambda: ccc.ccc2_tally(geno, 1000, small, o),
                 lambda: ccc.ccc2_tally_metric(geno, 1000, small, None, o),
                 lambda: ccc.ccc2_tally_metric_rows(geno, 1000, 0, n_v, small, None, o),
                 lambda: ccc.ccc3_tally(geno, 1000, 0, n_v, small, o)):
        with pytest.raises(ccc.CCCError) as e:
            call()
        assert e.value.status == ccc.CCC_EINVAL
    mgeno = torch.zeros((n_v, 1024), dtype=torch.uint8)
    t4 = torch.zeros((npairs, 4), dtype=torch.int32)  # an s = 4 table needs 16 per pair
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc2_multi_tally_metric(mgeno, 1000, 4, t4, None, o)
    assert e.value.status == ccc.CCC_EINVAL
    with pytest.raises(ccc.CCCError) as e:
        ccc.ccc2_filter(geno, 1000, 0.5, torch.zeros(39, dtype=torch.uint8), 1,
                        torch.zeros(1, dtype=torch.int64), o)
    assert e.value.status == ccc.CCC_EINVAL
