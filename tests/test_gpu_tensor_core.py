"""BF16 level-0 product of the MAS on the tensor cores: z = W^T (W r) with the
BF16 inverse Cholesky factor W (two tcgen05.mma per domain, the second with W
read as a transposed MN-major operand; FP32 accumulation in TMEM), against
the oracle's Eq. 6 apply with the same factor rounded the same way
(double -> float -> bf16) and against the FP32-core kernel on the same
factors.  The error bound is derived in tests/lowprec.py."""

import numpy as np
import pytest
import torch

import lowprec
from oracle import assembly, mas, pcg
from synth.workloads import make_tet_system, make_tet_systems, rhs

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


def setup(B, ctx, s, N, L):
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, N)
    M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                       dev(s.contacts, torch.int32), domain_size=N, max_levels=L, precision=B.GS_PREC_BF16)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    om = mas.build_mas(mp, N, L, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    return mat, M, om, (rid, cid, au)


def cube(n, seed):
    return make_tet_system(n, E=1e8, n_contacts=60, contact_mode="near", seed=seed)


@pytest.mark.parametrize("n,N,L,nrhs", [(11, 32, 3, 1), (11, 32, 3, 3), (11, 32, 3, 8), (9, 16, 2, 5),
                                        (7, 32, 1, 8), (12, 16, 3, 8)])
def test_tensor_core_apply_matches_rounded_oracle(B, ctx, n, N, L, nrhs):
    s = cube(n, 40 + n)
    V = s.n_vertices
    mat, M, om, _ = setup(B, ctx, s, N, L)
    ops, ops_abs = lowprec.effective_inverses(om, 2)
    r = np.random.default_rng(nrhs).normal(size=(nrhs, 3 * V)) * np.logspace(-3, 3, 3 * V)
    z = torch.empty((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    out = {}
    for tc in (1, 0):
        B.gs_tune_set(ctx, B.GS_TUNE_BF16_TC, tc)
        B.gs_mas_apply(ctx, M, dev(r, torch.float64), z, nrhs=nrhs)
        out[tc] = z.cpu().numpy()
    B.gs_tune_set(ctx, B.GS_TUNE_BF16_TC, 1)
    z0 = mas.apply(om.levels, ops, r, om.C)
    bound = lowprec.BOUND * mas.apply(om.levels, ops_abs, np.abs(r), om.C)
    for tc, zz in out.items():
        assert np.all(np.abs(zz - z0) <= bound + 1e-300), (tc, np.max(np.abs(zz - z0) / (bound + 1e-300)))
    # the two kernels round differently (hi/lo splits, accumulation order)
    assert not np.array_equal(out[0], out[1])
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)


def test_more_than_eight_rhs_use_the_fp32_core_kernel(B, ctx):
    s = cube(8, 50)
    V, nrhs = s.n_vertices, 9
    mat, M, om, _ = setup(B, ctx, s, 32, 2)
    r = np.random.default_rng(9).normal(size=(nrhs, 3 * V))
    z = torch.empty((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    B.gs_mas_apply(ctx, M, dev(r, torch.float64), z, nrhs=nrhs)
    ops, ops_abs = lowprec.effective_inverses(om, 2)
    z0 = mas.apply(om.levels, ops, r, om.C)
    bound = lowprec.BOUND * mas.apply(om.levels, ops_abs, np.abs(r), om.C)
    assert np.all(np.abs(z.cpu().numpy() - z0) <= bound + 1e-300)
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)


@pytest.mark.parametrize("nrhs", [1, 4, 8])
def test_mixed_solve_with_tensor_core_apply(B, ctx, nrhs):
    s = cube(12, 60)
    V = s.n_vertices
    mat, M, om, (rid, cid, au) = setup(B, ctx, s, 32, 3)
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
    # the same preconditioner up to ~2^-16 relative: the iteration counts stay
    # close.  The FP32 recurrence also feels the atomic (unordered) coarse
    # restriction and is checked every 8 iterations, so allow two checks' slack.
    assert its[1] <= 1.5 * its[0] + 16, its
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)


def test_bf16_factored_form_converges_where_stiff_contacts_spoil_a_rounded_inverse(B, ctx):
    """E = 1e5 with contact stiffness up to 1e6: domain condition numbers reach
    ~1e4, where a BF16-rounded inverse turns indefinite; W^T W stays SPD and
    FP64 PCG with it converges close to the FP64 preconditioner's count."""
    s = make_tet_systems(24, [1e5], n_contacts=200_000 * 24 ** 3 // 64 ** 3, contact_mode="near", seed=1002)[0]
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, 32)
    b = dev(rhs(3 * V, 8), torch.float64)
    its = {}
    for prec in (0, 2):
        M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                           dev(s.contacts, torch.int32), domain_size=32, max_levels=3, precision=prec)
        x = torch.zeros_like(b)
        it, _, _ = B.gs_pcg_solve(ctx, mat, M, b, x, nrhs=8, tol=1e-6, max_iter=5000)
        its[prec] = int(max(it))
        B.gs_mas_destroy(M)
    assert its[2] <= 1.5 * its[0] + 10, its
    B.gs_mat_destroy(mat)
