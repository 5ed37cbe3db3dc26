"""Launch-shape autotuner: every shape it may pick gives the oracle's result
(the SpMV and the MAS apply within the rounding of a reordered sum -- the
apply's restriction adds coarse sums with atomics, so it is not bitwise
repeatable even at one shape -- and the batched and mixed solves to the 1e-6
true residual), and the tuner leaves the fastest measured shape set in the
context."""

import numpy as np
import pytest
import torch

from oracle import assembly, mas, pcg
from synth.workloads import make_tet_system, rhs, uneven_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2411_06224_gb300.build import build

    build()
    from paper_2411_06224_gb300 import binding

    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.gs_create(0)
    yield c
    B.gs_destroy(c)


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def build(B, ctx, s, N=16, L=3, node_off=None):
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    if node_off is None:
        mp, nd = B.gs_partition(s.X, N)
    else:
        mp, nd = B.gs_partition_batch(s.X, node_off, N)
    M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                       dev(s.contacts, torch.int32), domain_size=N, max_levels=L)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    return mat, M, mp, (rid, cid, au)


def test_tune_set_rejects_values_outside_the_lists(B, ctx):
    for param, bad in ((B.GS_TUNE_SPMV_LANES, 3), (B.GS_TUNE_SPMV_LANES, 0), (B.GS_TUNE_APPLY_RHS, 16), (B.GS_TUNE_SPMV32_LANES, 8),
                       (B.GS_TUNE_BATCH_CHUNK, 3000), (B.GS_TUNE_BATCH_CHUNK, 512), (B.GS_TUNE_BF16_TC, 2),
                       (B.GS_TUNE_F64_TC, 5), (B.GS_TUNE_SPMV_WINDOW, 128), (B.GS_TUNE_SPMV_WINDOW, 3000),
                       (B.GS_TUNE_SPMV_WINDOW, 131072), (B.GS_TUNE_SPMV_WS, 2), (B.GS_TUNE_SPMV_FF_RHS, 3),
                       (B.GS_TUNE_COUNT, 2)):
        with pytest.raises(B.GsError):
            B.gs_tune_set(ctx, param, bad)
    from paper_2411_06224_gb300 import autotune

    assert autotune.current(ctx) == {"spmv_lanes": 2, "apply_rhs_per_thread": 4, "spmv32_lanes": 2,
                                     "batch_chunk": 4096, "bf16_tensor_cores": 1, "fp64_on_tensor_cores": 4,
                                     "spmv_row_window": 1024, "spmv_work_stealing": 1, "spmv_ff_rhs_per_pass": 8}


def test_every_shape_gives_the_oracle_result(B, ctx):
    from paper_2411_06224_gb300 import autotune

    s = make_tet_system(13, E=1e8, n_contacts=100, contact_mode="near", seed=21)
    V, nrhs = s.n_vertices, 6
    mat, M, mp, (rid, cid, au) = build(B, ctx, s)
    A = pcg.SymmetricMatrix(V, rid, cid, au)
    Absa = pcg.SymmetricMatrix(V, rid, cid, np.abs(au))
    Mo = mas.build_mas(mp, 16, 3, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    x = np.random.default_rng(3).normal(size=(nrhs, 3 * V))
    xd = dev(x, torch.float64)
    y = torch.empty_like(xd)
    Ax = np.stack([A(v) for v in x])
    bound = 1e-13 * np.stack([Absa(np.abs(v)) for v in x])
    by_lanes = {}
    for window in autotune.CANDIDATES[B.GS_TUNE_SPMV_WINDOW]:
        B.gs_tune_set(ctx, B.GS_TUNE_SPMV_WINDOW, window)
        for ws in autotune.CANDIDATES[B.GS_TUNE_SPMV_WS]:
            B.gs_tune_set(ctx, B.GS_TUNE_SPMV_WS, ws)
            for lanes in autotune.CANDIDATES[B.GS_TUNE_SPMV_LANES]:
                B.gs_tune_set(ctx, B.GS_TUNE_SPMV_LANES, lanes)
                B.gs_spmv(ctx, mat, xd, y, nrhs=nrhs)
                assert np.all(np.abs(y.cpu().numpy() - Ax) <= bound), (window, ws, lanes)
                # the row order and the schedule only decide which thread takes a
                # row, not the order of the row's sum: bitwise the same for all
                if lanes in by_lanes:
                    assert torch.equal(y, by_lanes[lanes]), (window, ws, lanes)
                else:
                    by_lanes[lanes] = y.clone()
    B.gs_tune_set(ctx, B.GS_TUNE_SPMV_WINDOW, 1024)
    # the float-float SpMV: every lane count, schedule and RHS-per-thread shape
    # within its per-row bound, and bitwise the same for a given summation order
    m = 3.0 * (np.bincount(rid, minlength=V) + np.bincount(cid[rid != cid], minlength=V))
    ff_bound = np.repeat(((3 * m + 1) * (m + 4) + 6) * 2.0 ** -48, 3) * (bound / 1e-13)
    ff_by_lanes = {}
    for ws in autotune.CANDIDATES[B.GS_TUNE_SPMV_WS]:
        B.gs_tune_set(ctx, B.GS_TUNE_SPMV_WS, ws)
        for rpp in autotune.CANDIDATES[B.GS_TUNE_SPMV_FF_RHS]:
            B.gs_tune_set(ctx, B.GS_TUNE_SPMV_FF_RHS, rpp)
            for lanes in autotune.CANDIDATES[B.GS_TUNE_SPMV_LANES]:
                B.gs_tune_set(ctx, B.GS_TUNE_SPMV_LANES, lanes)
                B.gs_spmv(ctx, mat, xd, y, nrhs=nrhs, variant=B.GS_SPMV_ROW_FF)
                assert np.all(np.abs(y.cpu().numpy() - Ax) <= ff_bound), (ws, rpp, lanes)
                # with fewer RHS per thread each lane walks all blocks in order:
                # the one-lane sums
                key = 1 if rpp < 8 and nrhs > rpp else lanes
                if key in ff_by_lanes:
                    assert torch.equal(y, ff_by_lanes[key]), (ws, rpp, lanes)
                else:
                    ff_by_lanes[key] = y.clone()
    B.gs_tune_set(ctx, B.GS_TUNE_SPMV_FF_RHS, 8)
    B.gs_tune_set(ctx, B.GS_TUNE_SPMV_LANES, 2)
    B.gs_tune_set(ctx, B.GS_TUNE_SPMV_WS, 1)
    zs = {}
    B.gs_tune_set(ctx, B.GS_TUNE_F64_TC, 0)  # the RHS-per-thread shape belongs to the FP64-core kernel
    for rpt in autotune.CANDIDATES[B.GS_TUNE_APPLY_RHS]:
        B.gs_tune_set(ctx, B.GS_TUNE_APPLY_RHS, rpt)
        B.gs_mas_apply(ctx, M, xd, y, nrhs=nrhs)
        zs[rpt] = y.cpu().numpy()
    B.gs_tune_set(ctx, B.GS_TUNE_F64_TC, 1)  # the digit storage this preconditioner was built with
    B.gs_mas_apply(ctx, M, xd, y, nrhs=nrhs)
    zs["tensor_cores"] = y.cpu().numpy()
    z0 = np.stack([Mo(v) for v in x])
    for rpt, z in zs.items():
        np.testing.assert_allclose(z, zs[4], rtol=1e-10, atol=1e-12 * np.abs(zs[4]).max())
        np.testing.assert_allclose(z, z0, rtol=1e-10, atol=1e-12 * np.abs(z0).max())
    b = rhs(3 * V, 4)
    for lanes in autotune.CANDIDATES[B.GS_TUNE_SPMV32_LANES]:
        B.gs_tune_set(ctx, B.GS_TUNE_SPMV32_LANES, lanes)
        xm = torch.zeros((4, 3 * V), dtype=torch.float64, device="cuda")
        B.gs_pcg_solve_mixed(ctx, mat, M, dev(b, torch.float64), xm, nrhs=4, tol=1e-6)
        for k, xk in enumerate(xm.cpu().numpy()):
            assert np.linalg.norm(b[k] - A(xk)) <= 1.05e-6 * np.linalg.norm(b[k]), lanes
    best = autotune.tune(ctx, mat, M, nrhs=nrhs, reps=3, mixed=True, fp64=True)
    assert {"spmv_lanes", "fp64_on_tensor_cores", "spmv32_lanes"} <= set(best)
    cur = autotune.current(ctx)
    for name, (v, times) in best.items():
        assert cur[name] == v and v in times and times[v] == min(times.values()) and times[v] > 0
    print("tuned", best)
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)


def test_batch_chunk_shapes_solve_every_system(B, ctx):
    from paper_2411_06224_gb300 import autotune

    bt = uneven_batch(n_sys=5, v_range=(300, 6000), e_range=(1e5, 1e9), seed=31)
    V = bt.n_vertices
    mat, M, _, (rid, cid, au) = build(B, ctx, bt, node_off=bt.node_off)
    A = pcg.SymmetricMatrix(V, rid, cid, au)
    b = rhs(3 * V, 1)[0]
    for chunk in autotune.CANDIDATES[B.GS_TUNE_BATCH_CHUNK]:
        B.gs_tune_set(ctx, B.GS_TUNE_BATCH_CHUNK, chunk)
        x = torch.zeros(3 * V, dtype=torch.float64, device="cuda")
        B.gs_pcg_solve_batch(ctx, mat, M, bt.node_off, dev(b, torch.float64), x, tol=1e-6)
        r = b - A(x.cpu().numpy())
        for s in range(len(bt.systems)):
            sl = slice(3 * int(bt.node_off[s]), 3 * int(bt.node_off[s + 1]))
            assert np.linalg.norm(r[sl]) <= 1.05e-6 * np.linalg.norm(b[sl]), (chunk, s)
    best = autotune.tune(ctx, mat, M, nrhs=1, reps=3, node_off=bt.node_off)
    assert autotune.current(ctx)["batch_chunk"] == best["batch_chunk"][0]
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)
