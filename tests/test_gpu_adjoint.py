"""Gradients through the solve (torch.autograd -> gs_adjoint) against the
oracle's dense-solve gradient and central finite differences."""

import numpy as np
import pytest
import torch

from oracle import adjoint, assembly
from synth.workloads import make_tet_system

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


def _setup(B, ctx, n=6, mixed=False, seed=31):
    from paper_2411_06224_gb300.autograd import System

    s = make_tet_system(n, E=1e6, n_contacts=8, contact_mode="random", seed=seed)
    sysm = System(ctx, s.n_vertices, s.rows, s.cols, s.X, s.adj_ptr, s.adj, s.contacts, domain_size=16, max_levels=3,
                  tol=1e-12, mixed=mixed)
    return s, sysm


@pytest.mark.parametrize("mixed", [False, True])
def test_gradients_match_oracle_dense_solve(B, ctx, mixed):
    from paper_2411_06224_gb300.autograd import solve

    s, sysm = _setup(B, ctx, mixed=mixed)
    n = s.n_vertices
    rng = np.random.default_rng(3)
    b_np = rng.normal(size=(2, 3 * n))
    xt_np = rng.normal(size=(2, 3 * n)) * 1e-4
    blocks = torch.tensor(s.blocks, dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(b_np, dtype=torch.float64, device="cuda", requires_grad=True)
    x = solve(blocks, b, sysm)
    L = ((x - torch.tensor(xt_np, device="cuda")) ** 2).sum()
    L.backward()
    # oracle: dense solves
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    xo = adjoint.solve_dense(n, rid, cid, au, b_np)
    _, g = adjoint.loss_and_grad(xo, xt_np)
    lam = adjoint.solve_dense(n, rid, cid, au, g)
    G = adjoint.block_gradients(rid, cid, xo, lam)
    keep = s.rows <= s.cols
    keys = (s.rows.astype(np.int64) << 32) | s.cols
    pos = np.searchsorted((rid.astype(np.int64) << 32) | cid, keys)
    dIn = np.where(keep[:, None, None], G[np.minimum(pos, len(G) - 1)], 0.0)
    gb = b.grad.cpu().numpy()
    gB = blocks.grad.cpu().numpy()
    assert np.linalg.norm(gb - lam) <= 1e-8 * np.linalg.norm(lam)
    assert np.linalg.norm(gB - dIn) <= 1e-8 * np.linalg.norm(dIn)


def test_gradients_match_finite_differences(B, ctx):
    from paper_2411_06224_gb300.autograd import solve

    s, sysm = _setup(B, ctx, seed=32)
    n = s.n_vertices
    rng = np.random.default_rng(4)
    b0 = torch.tensor(rng.normal(size=(1, 3 * n)), dtype=torch.float64, device="cuda")
    xt = torch.tensor(rng.normal(size=(1, 3 * n)) * 1e-4, dtype=torch.float64, device="cuda")
    bl0 = torch.tensor(s.blocks, dtype=torch.float64, device="cuda")

    def L(bl, bb):
        with torch.no_grad():
            return float(((solve(bl, bb, sysm) - xt) ** 2).sum())

    blocks = bl0.clone().requires_grad_(True)
    b = b0.clone().requires_grad_(True)
    ((solve(blocks, b, sysm) - xt) ** 2).sum().backward()
    db = torch.tensor(rng.normal(size=b0.shape), device="cuda")
    eps = 1e-6 * float(b0.norm() / db.norm())
    fd = (L(bl0, b0 + eps * db) - L(bl0, b0 - eps * db)) / (2 * eps)
    assert abs(fd - float((b.grad * db).sum())) <= 1e-4 * abs(fd)
    dB = torch.tensor(rng.normal(size=s.blocks.shape), device="cuda")
    eps = 1e-6 * float(bl0.norm() / dB.norm())
    fd = (L(bl0 + eps * dB, b0) - L(bl0 - eps * dB, b0)) / (2 * eps)
    assert abs(fd - float((blocks.grad * dB).sum())) <= 1e-4 * abs(fd)
