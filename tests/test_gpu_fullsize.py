"""Parity at the benchmark's full size (64^3 tet cube, 262,144 vertices, 13.4M
triplets, 8 right-hand sides, 3-level MAS with 32-node domains, tol 1e-6) in
the launch configuration bench.py times.  Integer results are compared in
full; floating point either in full against bounds from the arithmetic, on
sampled domains the oracle inverts one by one, or through properties that
hold at any size (true residual, iteration counts against the oracle's
stored counts)."""

import ctypes
import json
import os

import numpy as np
import pytest
import torch

import fp64bounds
from oracle import assembly, mas, partition, pcg
from synth.workloads import rhs, stiffness_sweep

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sweep64_pcg_iterations.json")
N, L, NRHS = 32, 3, 8


@pytest.fixture(scope="module")
def B():
    from paper_2411_06224_gb300.build import build

    build()
    from paper_2411_06224_gb300 import binding

    return binding


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def full(B):
    s = stiffness_sweep(Es=(1e9,), n=64)[0]
    ctx = B.gs_create(0)
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, N)
    M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                       dev(s.contacts, torch.int32), domain_size=N, max_levels=L)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    yield dict(s=s, ctx=ctx, mat=mat, M=M, mp=mp, nd=nd, rid=rid, cid=cid, au=au, V=V)
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)
    B.gs_destroy(ctx)


def test_full_assembly_and_partition(B, full):
    s = full["s"]
    rid, cid, au = B.gs_mat_export(full["ctx"], full["mat"])
    assert np.array_equal(rid.cpu().numpy(), full["rid"]) and np.array_equal(cid.cpu().numpy(), full["cid"])
    _, _, abs_sum = assembly.assemble(s.rows, s.cols, np.abs(s.blocks))
    assert np.all(np.abs(au.cpu().numpy() - full["au"]) <= 1e-13 * abs_sum)
    mo, _ = partition.map_remap(partition.recursive_bisection(s.X, N), N)
    assert np.array_equal(full["mp"], mo)
    # the device partition, bit for bit
    md, ndd = B.gs_partition_device(full["ctx"], dev(s.X, torch.float64), N, B.GS_PART_RCB)
    assert ndd == full["nd"] and np.array_equal(md.cpu().numpy(), mo)


def test_full_levels_spmv_apply(B, full):
    s, V, ctx = full["s"], full["V"], full["ctx"]
    om = mas.build_mas(full["mp"], N, L, s.adj_ptr, s.adj, s.contacts, full["rid"], full["cid"], full["au"])
    nl, items = B.gs_mas_info(full["M"])
    assert nl == om.levels.n_levels == L and items == [int(v) for v in om.levels.n_items]
    for l in range(nl):
        assert np.array_equal(B.gs_mas_export_coarse(ctx, full["M"], l, V).cpu().numpy(), om.levels.coarse[l])
    # sampled domain inverses against the oracle's, per level
    rng = np.random.default_rng(0)
    for l in range(nl):
        nd = om.levels.n_domains(l)
        inv = B.gs_mas_export_inverse(ctx, full["M"], l, nd, N).cpu().numpy()
        for d in rng.choice(nd, size=min(nd, 12), replace=False):
            ref = om.invs[l][d]
            kappa = np.linalg.cond(om.mats[l][d]) if np.all(np.diag(om.mats[l][d]) != 0) else 1e12
            assert np.linalg.norm(inv[d] - ref) <= 1e-12 * kappa * np.linalg.norm(ref)
    # SpMV and apply over every node
    A = pcg.SymmetricMatrix(V, full["rid"], full["cid"], full["au"])
    x = np.random.default_rng(1).normal(size=(NRHS, 3 * V))
    y = torch.empty((NRHS, 3 * V), dtype=torch.float64, device="cuda")
    B.gs_spmv(ctx, full["mat"], dev(x, torch.float64), y, nrhs=NRHS, variant=B.GS_SPMV_ROW)
    Aabs = pcg.SymmetricMatrix(V, full["rid"], full["cid"], np.abs(full["au"]))
    for k in range(NRHS):
        assert np.all(np.abs(y[k].cpu().numpy() - A(x[k])) <= 1e-13 * Aabs(np.abs(x[k])))
    # the float-float product, against its own per-row bound
    yf = torch.empty_like(y)
    B.gs_spmv(ctx, full["mat"], dev(x, torch.float64), yf, nrhs=NRHS, variant=B.GS_SPMV_ROW_FF)
    rid, cid = full["rid"], full["cid"]
    m = 3.0 * (np.bincount(rid, minlength=V) + np.bincount(cid[rid != cid], minlength=V))
    gamma = np.repeat(((3 * m + 1) * (m + 4) + 6) * 2.0 ** -48, 3)
    worst = 0.0
    for k in range(NRHS):
        sc = Aabs(np.abs(x[k]))
        err = np.abs(yf[k].cpu().numpy() - A(x[k]))
        assert np.all(err <= gamma * sc)
        worst = max(worst, (err / (1e-13 * sc)).max())
    print("float-float SpMV at 64^3: max error / (1e-13 |A||x|) =", worst)
    z = torch.empty_like(y)
    B.gs_mas_apply(ctx, full["M"], dev(x, torch.float64), z, nrhs=NRHS)
    z0 = om(x)
    dz = np.abs(z.cpu().numpy() - z0)
    bound = fp64bounds.apply_bound(om, x)
    assert np.all(dz <= bound), (dz / bound).max()
    # the allocation-free apply holds this size's coarse-level scratch (8 RHS)
    zn = torch.full_like(z, np.nan)
    before = B.gs_ctx_alloc_stats(ctx)
    st = B.lib().gs_mas_apply_noalloc(ctx, full["M"], ctypes.c_void_p(dev(x, torch.float64).data_ptr()),
                                      ctypes.c_void_p(zn.data_ptr()), NRHS)
    assert st == B.GS_OK, B.lib().gs_last_error()
    torch.cuda.synchronize()
    assert B.gs_ctx_alloc_stats(ctx) == before
    assert ((zn - z).abs().amax() / z.abs().amax()).item() <= 1e-12


def test_full_pcg_counts_and_residuals(B, full):
    V, ctx = full["V"], full["ctx"]
    b = rhs(3 * V, NRHS)
    x = torch.zeros((NRHS, 3 * V), dtype=torch.float64, device="cuda")
    it, rel, _ = B.gs_pcg_solve(ctx, full["mat"], full["M"], dev(b, torch.float64), x, nrhs=NRHS, tol=1e-6,
                                variant=B.GS_SPMV_ROW)
    A = pcg.SymmetricMatrix(V, full["rid"], full["cid"], full["au"])
    xg = x.cpu().numpy()
    g = json.load(open(GOLDEN))["iterations"]["1e+09"]
    for k in range(NRHS):
        assert abs(int(it[k]) - g[k]) <= 2, (list(it), g)
        assert np.linalg.norm(b[k] - A(xg[k])) <= 1.05e-6 * np.linalg.norm(b[k])
    # the same solve on the float-float SpMV
    xf = torch.zeros_like(x)
    itf, _, _ = B.gs_pcg_solve(ctx, full["mat"], full["M"], dev(b, torch.float64), xf, nrhs=NRHS, tol=1e-6,
                               variant=B.GS_SPMV_ROW_FF)
    xfg = xf.cpu().numpy()
    for k in range(NRHS):
        assert abs(int(itf[k]) - g[k]) <= 2, (list(itf), g)
        assert np.linalg.norm(b[k] - A(xfg[k])) <= 1.05e-6 * np.linalg.norm(b[k])
    print("FP64 SpMV iterations", list(it), "float-float", list(itf), "oracle", g)
    # mixed precision on the same system: the true FP64 residual meets the
    # tolerance.  Both solves stop on a residual test, so their distance is
    # bounded only by cond(A) * 2e-6; it is stated, with a sanity bound.
    xm = torch.zeros_like(x)
    itm, relm, outer, _ = B.gs_pcg_solve_mixed(ctx, full["mat"], full["M"], dev(b, torch.float64), xm, nrhs=NRHS,
                                               tol=1e-6)
    xmg = xm.cpu().numpy()
    errs = []
    for k in range(NRHS):
        assert np.linalg.norm(b[k] - A(xmg[k])) <= 1.0001e-6 * np.linalg.norm(b[k])
        errs.append(np.linalg.norm(xmg[k] - xg[k]) / np.linalg.norm(xg[k]))
    print("mixed: inner iterations", list(itm), "outer", outer, "rel. error vs FP64 solve", errs)
    assert max(errs) <= 1e-3
