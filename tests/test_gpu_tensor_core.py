"""BF16 level-0 MAS product on the tensor cores (tcgen05.mma, FP32 accumulation
in TMEM) against the oracle's Eq. 6 apply with the inverses rounded to BF16
(double -> float -> bf16, nearest even) and against the FP32-core kernel on
the same BF16 inverses.

Error budget per output entry, relative to sum_j |M_ij| |r_j| over all
levels: the right-hand side enters as hi + lo BF16 parts of its FP32 value
(|r - hi - lo| <= 2^-18 |r|), products are exact in FP32 and the sums
accumulate in FP32 (<= 96 * 2^-24); 1e-5 covers both with room."""

import numpy as np
import pytest
import torch

from oracle import assembly, mas, pcg
from synth.workloads import make_tet_system, rhs

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


def round_bf16(a):
    """double -> float -> bfloat16 with round-to-nearest-even, back to double."""
    f = np.asarray(a).astype(np.float32).view(np.uint32)
    f = (f + (((f >> 16) & 1) + 0x7FFF)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def setup(B, ctx, n, N, L, seed):
    s = make_tet_system(n, E=1e8, n_contacts=60, contact_mode="near", seed=seed)
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, N)
    M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                       dev(s.contacts, torch.int32), domain_size=N, max_levels=L, precision=B.GS_PREC_BF16)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    om = mas.build_mas(mp, N, L, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    return s, mat, M, om, (rid, cid, au)


@pytest.mark.parametrize("n,N,L,nrhs", [(11, 32, 3, 1), (11, 32, 3, 3), (11, 32, 3, 8), (9, 16, 2, 5),
                                        (7, 32, 1, 8), (12, 16, 3, 8)])
def test_tensor_core_apply_matches_rounded_oracle(B, ctx, n, N, L, nrhs):
    s, mat, M, om, _ = setup(B, ctx, n, N, L, seed=40 + n)
    V = s.n_vertices
    inv_r = [round_bf16(v) for v in om.invs]
    r = np.random.default_rng(nrhs).normal(size=(nrhs, 3 * V)) * np.logspace(-3, 3, 3 * V)
    z = torch.empty((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    out = {}
    for tc in (1, 0):
        B.gs_tune_set(ctx, B.GS_TUNE_BF16_TC, tc)
        B.gs_mas_apply(ctx, M, dev(r, torch.float64), z, nrhs=nrhs)
        out[tc] = z.cpu().numpy()
    B.gs_tune_set(ctx, B.GS_TUNE_BF16_TC, 1)
    z0 = mas.apply(om.levels, inv_r, r, om.C)
    bound = 1e-5 * mas.apply(om.levels, [np.abs(v) for v in inv_r], np.abs(r), om.C)
    for tc, zz in out.items():
        assert np.all(np.abs(zz - z0) <= bound + 1e-300), (tc, np.max(np.abs(zz - z0) / (bound + 1e-300)))
    # the two kernels round differently (hi/lo split, accumulation order)
    assert not np.array_equal(out[0], out[1])
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)


def test_more_than_eight_rhs_use_the_fp32_core_kernel(B, ctx):
    s, mat, M, om, _ = setup(B, ctx, 8, 32, 2, seed=50)
    V, nrhs = s.n_vertices, 9
    r = np.random.default_rng(9).normal(size=(nrhs, 3 * V))
    z = torch.empty((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    B.gs_mas_apply(ctx, M, dev(r, torch.float64), z, nrhs=nrhs)
    inv_r = [round_bf16(v) for v in om.invs]
    z0 = mas.apply(om.levels, inv_r, r, om.C)
    bound = 1e-5 * mas.apply(om.levels, [np.abs(v) for v in inv_r], np.abs(r), om.C)
    assert np.all(np.abs(z.cpu().numpy() - z0) <= bound + 1e-300)
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)


@pytest.mark.parametrize("nrhs", [1, 4, 8])
def test_mixed_solve_with_tensor_core_apply(B, ctx, nrhs):
    s, mat, M, om, (rid, cid, au) = setup(B, ctx, 12, 32, 3, seed=60)
    V = s.n_vertices
    A = pcg.SymmetricMatrix(V, rid, cid, au)
    b = rhs(3 * V, nrhs)
    its = {}
    for tc in (1, 0):
        B.gs_tune_set(ctx, B.GS_TUNE_BF16_TC, tc)
        x = torch.zeros((nrhs, 3 * V), dtype=torch.float64, device="cuda")
        it, rel, outer, _ = B.gs_pcg_solve_mixed(ctx, mat, M, dev(b, torch.float64), x, nrhs=nrhs, tol=1e-6)
        for k, xk in enumerate(x.cpu().numpy()):
            assert np.linalg.norm(b[k] - A(xk)) <= 1.0001e-6 * np.linalg.norm(b[k]), (tc, k)
        its[tc] = int(max(it))
    B.gs_tune_set(ctx, B.GS_TUNE_BF16_TC, 1)
    # the same preconditioner up to ~2^-16 relative: the iteration counts stay close
    assert its[1] <= 1.2 * its[0] + 5, its
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)
