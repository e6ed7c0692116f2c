"""Helpers for the GPU parity tests: run the C ABI on seeded panels, compare with the oracle."""

from __future__ import annotations

import numpy as np

CCC_RTOL = 1e-6  # relative tolerance on CCC values (single-precision epilogue vs fp64 oracle)


def torch_mod():
    import torch
    return torch


def to_device(geno_np):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(geno_np).view(np.int64)).cuda()


def workspace(nbytes):
    torch = torch_mod()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")


def run_2way(geno_np, n_f, path, norm=0, gamma=2.0 / 3.0, fused=True, tile=0, split=0, operand=0,
             group=0):
    """Tallies (int32 [npairs, 4]) and CCC (float32 [npairs, 4]) through the C ABI.

    split: ccc_opts.split (0 automatic, 1 off); operand: ccc_opts.operand (0 automatic,
    1 e4m3, 2 e2m1); group: ccc_opts.group (0 the kernel's default tile order)."""
    import paper_1705_08213_gb300 as ccc
    torch = torch_mod()
    g = to_device(geno_np)
    n_v = geno_np.shape[0]
    npairs = ccc.ccc2_count(n_v)
    opts = ccc.ccc_opts_default(path=path, norm=norm, gamma=gamma, tile=tile)
    if operand:
        opts.operand = operand
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_2WAY))
    opts = ccc.ccc_opts_default(path=path, norm=norm, gamma=gamma, workspace=ws, tile=tile)
    opts.split = split
    opts.group = group
    if operand:
        opts.operand = operand
    tally = torch.full((max(npairs, 1), 4), -7, dtype=torch.int32, device="cuda")
    out = torch.full((max(npairs, 1), 4), -7.0, dtype=torch.float32, device="cuda")
    if fused:
        ccc.ccc2_tally_metric(g, n_f, tally, out, opts)
    else:
        counts = torch.zeros((n_v, 3), dtype=torch.int32, device="cuda")
        ccc.ccc_allele_counts(g, n_f, counts)
        ccc.ccc2_tally(g, n_f, tally, opts)
        wsm = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_METRIC))
        optm = ccc.ccc_opts_default(path=path, norm=norm, gamma=gamma, workspace=wsm)
        ccc.ccc2_metric(tally, counts, n_v, optm, out)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    return tally[:npairs].cpu().numpy(), out[:npairs].cpu().numpy()


def run_3way(geno_np, n_f, path, j_begin=0, j_end=None, norm=0, gamma=2.0 / 3.0, fused=True,
             tile=0, operand=0):
    import paper_1705_08213_gb300 as ccc
    torch = torch_mod()
    g = to_device(geno_np)
    n_v = geno_np.shape[0]
    j_end = n_v if j_end is None else j_end
    nt = ccc.ccc3_count(n_v, j_begin, j_end)
    opts = ccc.ccc_opts_default(path=path, norm=norm, gamma=gamma, tile=tile, operand=operand)
    ws = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_3WAY))
    opts = ccc.ccc_opts_default(path=path, norm=norm, gamma=gamma, workspace=ws, tile=tile,
                                operand=operand)
    tally = torch.full((max(nt, 1), 8), -7, dtype=torch.int32, device="cuda")
    out = torch.full((max(nt, 1), 8), -7.0, dtype=torch.float32, device="cuda")
    if fused:
        ccc.ccc3_tally_metric(g, n_f, j_begin, j_end, tally, out, opts)
    else:
        counts = torch.zeros((n_v, 3), dtype=torch.int32, device="cuda")
        ccc.ccc_allele_counts(g, n_f, counts)
        ccc.ccc3_tally(g, n_f, j_begin, j_end, tally, opts)
        wsm = workspace(ccc.ccc_workspace_size(g, n_f, opts, ccc.CCC_OP_METRIC))
        optm = ccc.ccc_opts_default(path=path, norm=norm, gamma=gamma, workspace=wsm)
        ccc.ccc3_metric(tally, counts, n_v, j_begin, j_end, optm, out)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    return tally[:nt].cpu().numpy(), out[:nt].cpu().numpy()


def assert_ccc_close(got, expect, rtol=CCC_RTOL, what=""):
    got = np.asarray(got, dtype=np.float64)
    expect = np.asarray(expect, dtype=np.float64)
    assert got.shape == expect.shape, (got.shape, expect.shape)
    err = np.abs(got - expect)
    bad = err > rtol * np.abs(expect)
    if np.any(bad):
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{what}: {bad.sum()} CCC values beyond rtol {rtol}; first "
                             f"{[(tuple(i), got[tuple(i)], expect[tuple(i)]) for i in idx]}")


def assert_tally_equal(got, expect, what=""):
    got = np.asarray(got, dtype=np.int64)
    expect = np.asarray(expect, dtype=np.int64)
    assert got.shape == expect.shape, (got.shape, expect.shape)
    if not np.array_equal(got, expect):
        bad = np.argwhere(got != expect)[:5]
        raise AssertionError(f"{what}: {int((got != expect).sum())} tallies differ; first "
                             f"{[(tuple(i), got[tuple(i)], expect[tuple(i)]) for i in bad]}")


def to_device_bytes(geno_np):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(geno_np, dtype=np.uint8)).cuda()


def run_multi(geno_np, n_f, s, norm=0, gamma=2.0 / 3.0, fused=True, group=0, operand=0, split=0):
    """Multi-allelic tallies (int32 [npairs, s*s]) and CCC (float32 [npairs, s*s]) via the C ABI.

    operand: ccc_opts.operand (0 automatic: e2m1 for s <= 8 without K split); split:
    ccc_opts.split (0 automatic, 1 off)."""
    import paper_1705_08213_gb300 as ccc
    torch = torch_mod()
    g = to_device_bytes(geno_np)
    n_v = geno_np.shape[0]
    npairs = ccc.ccc2_count(n_v)
    opts = ccc.ccc_opts_default(norm=norm, gamma=gamma)
    ws = workspace(ccc.ccc_multi_workspace_size(g, n_f, s, opts))
    opts = ccc.ccc_opts_default(norm=norm, gamma=gamma, workspace=ws)
    opts.group = group
    opts.operand = operand
    opts.split = split
    tally = torch.full((max(npairs, 1), s * s), -7, dtype=torch.int32, device="cuda")
    out = torch.full((max(npairs, 1), s * s), -7.0, dtype=torch.float32, device="cuda")
    if fused:
        ccc.ccc2_multi_tally_metric(g, n_f, s, tally, out, opts)
    else:
        counts = torch.zeros((n_v, s + 1), dtype=torch.int32, device="cuda")
        ccc.ccc_multi_counts(g, n_f, s, counts)
        ccc.ccc2_multi_tally(g, n_f, s, tally, opts)
        ccc.ccc2_multi_metric(tally, counts, n_v, s, opts, out)
    torch.cuda.synchronize()
    assert ccc.ccc_status(opts) == ccc.CCC_OK
    return tally[:npairs].cpu().numpy(), out[:npairs].cpu().numpy()
