"""Low-precision MAS forms (FP32 inverses; BF16 inverse Cholesky factors at
level 0; FP32 accumulation) against the FP64 oracle's levels with the same
roundings applied, and the precision forms
on a stiff cloth sheet (cubic strain limiting, E = 1e8): every solve must
reach the 1e-6 true residual and agree with the oracle's FP64 solution."""

import numpy as np
import pytest
import torch

import lowprec
from oracle import assembly, mas, partition, pcg
from synth.cloth import make_cloth_system
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


@pytest.fixture(scope="module")
def cloth():
    return make_cloth_system(48, seed=5)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("name", ["cube", "cloth"])
def test_low_precision_apply_matches_rounded_oracle(B, ctx, cloth, prec, name):
    s = cloth if name == "cloth" else make_tet_system(11, E=1e8, n_contacts=80, contact_mode="near", seed=12)
    V, N, L, nrhs = s.n_vertices, 32, 3, 4
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, N)
    M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                       dev(s.contacts, torch.int32), domain_size=N, max_levels=L, precision=prec)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    om = mas.build_mas(mp, N, L, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    ops, ops_abs = lowprec.effective_inverses(om, prec)
    r = np.random.default_rng(prec).normal(size=(nrhs, 3 * V))
    z = torch.empty((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    B.gs_mas_apply(ctx, M, dev(r, torch.float64), z, nrhs=nrhs)
    z0 = mas.apply(om.levels, ops, r, om.C)
    bound = lowprec.BOUND * mas.apply(om.levels, ops_abs, np.abs(r), om.C)
    assert np.all(np.abs(z.cpu().numpy() - z0) <= bound + 1e-300)
    B.gs_mas_destroy(M)
    B.gs_mat_destroy(mat)


def test_precision_forms_on_stiff_cloth(B, ctx, cloth):
    s = cloth
    V, N, L, nrhs = s.n_vertices, 32, 3, 4
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, N)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    A = pcg.SymmetricMatrix(V, rid, cid, au)
    om = mas.build_mas(mp, N, L, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    b = rhs(3 * V, nrhs)
    xo, it_o, _ = pcg.pcg(A, om, b, tol=1e-6)
    counts, errors = {}, {}
    for prec in (0, 1, 2):
        M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                           None, domain_size=N, max_levels=L, precision=prec)
        for solver in ("fp64_outer", "mixed"):
            x = torch.zeros((nrhs, 3 * V), dtype=torch.float64, device="cuda")
            if solver == "fp64_outer":
                it, rel, _ = B.gs_pcg_solve(ctx, mat, M, dev(b, torch.float64), x, nrhs=nrhs, tol=1e-6,
                                            max_iter=20000)
            else:
                it, rel, _, _ = B.gs_pcg_solve_mixed(ctx, mat, M, dev(b, torch.float64), x, nrhs=nrhs, tol=1e-6,
                                                     max_iter=20000)
            xg = x.cpu().numpy()
            err = 0.0
            for k in range(nrhs):
                true = np.linalg.norm(b[k] - A(xg[k])) / np.linalg.norm(b[k])
                assert true <= 1.05e-6, (prec, solver, true)
                err = max(err, np.linalg.norm(xg[k] - xo[k]) / np.linalg.norm(xo[k]))
            # the FP64 path follows the oracle's recurrence: 1e-5 solution error;
            # the other forms stop on the same residual test along another
            # recurrence, so their error is stated (bounded by cond(A) * 2e-6)
            assert err <= (1e-5 if (prec, solver) == (0, "fp64_outer") else 1e-3), (prec, solver, err)
            counts[(prec, solver)] = int(max(it))
            errors[(prec, solver)] = err
        B.gs_mas_destroy(M)
    # FP64 outer PCG with FP64 inverses follows the oracle's recurrence; on this
    # stiff sheet (~340 iterations, the recurrence losing orthogonality) the
    # round-off of a differently ordered FP64 product moves the count by a few
    assert abs(counts[(0, "fp64_outer")] - int(max(it_o))) <= max(2, 0.01 * int(max(it_o)))
    print("max iterations", counts, "oracle", list(it_o), "rel. error vs oracle", errors)
    B.gs_mat_destroy(mat)
