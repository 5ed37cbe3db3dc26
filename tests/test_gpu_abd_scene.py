"""Coupled FEM / affine-body scene (synth.abd): the two-level assembly with
body inertia, orthogonality Hessians on the bodies' own rows and the three
contact kinds; the MAS-PCG solve on the reduced system; and the adjoint with
an FP32 preconditioner (FP64 PCG, FP64 reductions) against the oracle's
dense-solve gradient.

A small scene is compared in full; the 100^3 + 2,000-body scene is checked
through the reduced matrix's action, A_red v = J^T A_full J v + (body
blocks) v, which holds at any size."""

import numpy as np
import pytest
import torch

from oracle import adjoint, assembly, mas, pcg
from synth.abd import make_abd_scene

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


def assemble(B, ctx, s):
    return B.gs_assemble_abd(ctx, s.n_nodes, s.n_fem, s.n_bodies, dev(s.body_of_node, torch.int32),
                             dev(s.xbar, torch.float64), dev(s.rows, torch.int32), dev(s.cols, torch.int32),
                             dev(s.blocks, torch.float64))


@pytest.fixture(scope="module")
def small():
    return make_abd_scene(n=9, n_bodies=16, n_contacts=3000, seed=77)


def test_scene_assembly_matches_oracle(B, ctx, small):
    s = small
    mat = assemble(B, ctx, s)
    rid, cid, au = B.gs_mat_export(ctx, mat)
    r0, c0, a0 = assembly.assemble_abd(s.rows, s.cols, s.blocks, s.body_of_node, s.xbar, s.n_fem)
    assert np.array_equal(rid.cpu().numpy(), r0) and np.array_equal(cid.cpu().numpy(), c0)
    assert np.abs(au.cpu().numpy() - a0).max() <= 1e-12 * np.abs(a0).max()
    B.gs_mat_destroy(mat)


@pytest.mark.parametrize("prec", [0, 1])
def test_scene_solve_and_fp32_preconditioned_adjoint(B, ctx, small, prec):
    s = small
    n = s.n_red
    N, L = 16, 3
    mat = assemble(B, ctx, s)
    mp, nd = B.gs_partition(s.X, N)
    M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                       dev(s.contacts, torch.int32), domain_size=N, max_levels=L, precision=prec)
    rid, cid, au = assembly.assemble_abd(s.rows, s.cols, s.blocks, s.body_of_node, s.xbar, s.n_fem)
    A = pcg.SymmetricMatrix(n, rid, cid, au)
    rng = np.random.default_rng(5)
    b = rng.normal(size=(1, 3 * n))
    xt = rng.normal(size=(1, 3 * n))
    x = torch.zeros((1, 3 * n), dtype=torch.float64, device="cuda")
    it, rel, _ = B.gs_pcg_solve(ctx, mat, M, dev(b, torch.float64), x, nrhs=1, tol=1e-12)
    xg = x.cpu().numpy()
    # the recurrence residual stops at 1e-12; the true residual trails it by rounding
    assert np.linalg.norm(b[0] - A(xg[0])) <= 1e-11 * np.linalg.norm(b[0])
    if prec == 0:  # the oracle's MAS on the reduced system: same recurrence
        Mo = mas.build_mas(mp, N, L, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
        _, it_o, _ = pcg.pcg(A, Mo, b, tol=1e-12)
        assert abs(int(it[0]) - int(it_o[0])) <= 2, (it, it_o)
    # adjoint of L = ||x - x_t||^2 with the same (FP32 when prec = 1) preconditioner
    g = 2.0 * (xg - xt)
    dLdH = torch.zeros((au.shape[0], 3, 3), dtype=torch.float64, device="cuda")
    lam, _ = B.gs_adjoint(ctx, mat, M, x, dev(g, torch.float64), nrhs=1, tol=1e-12, dLdH=dLdH)
    xo = adjoint.solve_dense(n, rid, cid, au, b)
    _, go = adjoint.loss_and_grad(xo, xt)
    lo = adjoint.solve_dense(n, rid, cid, au, go)
    Go = adjoint.block_gradients(rid, cid, xo, lo)
    lam_g = lam.cpu().numpy()
    err_l = np.linalg.norm(lam_g - lo) / np.linalg.norm(lo)
    err_G = np.linalg.norm(dLdH.cpu().numpy() - Go) / np.linalg.norm(Go)
    print("prec", prec, "iterations", list(it), "lambda error", err_l, "dL/dH error", err_G)
    assert err_l <= 1e-5 and err_G <= 1e-5
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)


def _reduced_action_oracle(s, v, absolute=False):
    """A_red v from the oracle's level-1 (full-space) assembly and the Jacobians.

    absolute: the same products over absolute values, |J|^T |A_in| |J| |v| with
    |A_in| the sums of the input blocks' absolute values -- the scale against
    which reordered sums are bounded."""
    ab = np.abs if absolute else (lambda a: a)
    v = ab(v)
    n_full = s.n_nodes
    node = (s.rows < n_full) & (s.cols < n_full)
    rid, cid, au = assembly.assemble(s.rows[node], s.cols[node], ab(s.blocks[node]))
    # J v: x_i = v_i (FEM) or p + sum_k xbar_ik a_k (body corner)
    vr = v.reshape(-1, 3)
    xf = np.zeros((n_full, 3))
    xf[: s.n_fem] = vr[: s.n_fem]
    b = s.body_of_node[s.n_fem :]
    q = vr[s.n_fem :].reshape(s.n_bodies, 4, 3)
    w = ab(np.concatenate([np.ones((b.size, 1)), s.xbar[s.n_fem :]], 1))  # (corners, 4)
    xf[s.n_fem :] = np.einsum("ca,cay->cy", w, q[b])
    yf = pcg.spmv(rid, cid, au, xf[None])[0]
    # J^T y
    y = np.zeros((s.n_red, 3))
    y[: s.n_fem] = yf[: s.n_fem]
    yb = np.zeros((s.n_bodies, 4, 3))
    np.add.at(yb, b, w[:, :, None] * yf[s.n_fem :, None, :])
    y[s.n_fem :] = yb.reshape(-1, 3)
    # the bodies' own blocks (indices n_full + 4b + a -> reduced row n_fem + 4b + a)
    own = ~node
    r2 = np.where(s.rows[own] >= n_full, s.rows[own] - n_full + s.n_fem, -1)
    c2 = np.where(s.cols[own] >= n_full, s.cols[own] - n_full + s.n_fem, -1)
    assert np.all(r2 >= 0) and np.all(c2 >= 0)  # the generator mixes no node with a body row
    rid2, cid2, au2 = assembly.assemble(r2, c2, ab(s.blocks[own]))
    y += pcg.spmv(rid2, cid2, au2, vr[None])[0]
    return y.reshape(-1)


def test_full_size_scene_reduced_action():
    """100^3 cube + 2,000 bodies + 500k contacts: the assembled reduced matrix acts like J^T A J."""
    from paper_2411_06224_gb300.build import build

    build()
    from paper_2411_06224_gb300 import binding as B

    ctx = B.gs_create(0)
    s = make_abd_scene()
    mat = assemble(B, ctx, s)
    n = s.n_red
    assert B.gs_mat_info(mat)[0] == n
    rng = np.random.default_rng(11)
    v = rng.normal(size=3 * n)
    y = torch.empty((1, 3 * n), dtype=torch.float64, device="cuda")
    B.gs_spmv(ctx, mat, dev(v[None], torch.float64), y, nrhs=1)
    y0 = _reduced_action_oracle(s, v)
    scale = _reduced_action_oracle(s, v, absolute=True)
    assert np.all(np.abs(y.cpu().numpy()[0] - y0) <= 1e-12 * scale)
    # forward and adjoint MAS-PCG with the FP32 preconditioner, in the launch
    # configuration of the benchmark (N = 32, 3 levels, tol 1e-6)
    mp, nd = B.gs_partition(s.X, 32)
    M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                       dev(s.contacts, torch.int32), domain_size=32, max_levels=3, precision=B.GS_PREC_FP32)
    b = dev(rng.normal(size=(1, 3 * n)), torch.float64)
    xt = dev(rng.normal(size=(1, 3 * n)), torch.float64)
    x = torch.zeros_like(b)
    it, _, _ = B.gs_pcg_solve(ctx, mat, M, b, x, nrhs=1, tol=1e-6)
    g = 2.0 * (x - xt)
    nnzb = B.gs_mat_info(mat)[1]
    dLdH = torch.zeros((nnzb, 3, 3), dtype=torch.float64, device="cuda")
    lam, it_a = B.gs_adjoint(ctx, mat, M, x, g, nrhs=1, tol=1e-6, dLdH=dLdH)
    Ax = torch.empty_like(x)
    for vec, rhs_ in ((x, b), (lam, g)):  # true residuals through the library's FP64 SpMV
        B.gs_spmv(ctx, mat, vec, Ax, nrhs=1)
        assert float((rhs_ - Ax).norm() / rhs_.norm()) <= 1.05e-6
    # dL/dH on sampled stored blocks against the outer-product formula
    rid, cid, _ = B.gs_mat_export(ctx, mat)
    pick = rng.choice(nnzb, 4096, replace=False)
    r_, c_ = rid.cpu().numpy()[pick], cid.cpu().numpy()[pick]
    xs = x.cpu().numpy().reshape(1, -1, 3)
    ls = lam.cpu().numpy().reshape(1, -1, 3)
    Gs = adjoint.block_gradients(r_, c_, xs, ls)
    Gg = dLdH.cpu().numpy()[pick]
    assert np.abs(Gg - Gs).max() <= 1e-12 * np.abs(Gs).max()
    print("abd scene: reduced rows", n, "stored blocks", nnzb, "forward iterations", list(it), "adjoint", list(it_a))
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)
    B.gs_destroy(ctx)
