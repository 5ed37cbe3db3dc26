"""The float-float SpMV (GS_SPMV_ROW_FF) and PCG on it, through the C ABI,
against the FP64 oracle.

The product keeps about 47 significant bits.  Its stated error per output is
((3m+1)(m+4) + 6) u^2 (|A||x|)_i with u = 2^-24 and m = 3 x the stored blocks
of row i (both triangles): the two-sum chain of the exact products is exact,
the float sum of the small parts has at most 3m + 1 roundings over terms that
add up to at most (m + 4) u sum|t|, and the splits, the dropped lo*lo parts
and the final FP64 addition add at most 6 u^2 sum|t|.  Every output is checked
against that bound; the largest ratio to the FP64 kernels' 1e-13 (|A||x|)_i
bound is printed as well.
"""

import numpy as np
import pytest
import torch

from oracle import assembly, mas, partition, pcg
from synth.workloads import make_tet_system, plain_small, rhs

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


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


_CASES = {}


def case(name):
    if name not in _CASES:
        if name == "cube8":
            _CASES[name] = make_tet_system(8, E=1e6, n_contacts=40, contact_mode="random", seed=11)
        elif name == "cube11":  # ragged last domain, near contacts (duplicate keys)
            _CASES[name] = make_tet_system(11, E=1e8, n_contacts=120, contact_mode="near", seed=12)
        elif name == "plain16":
            _CASES[name] = plain_small()
    return _CASES[name]


def ff_bound(V, rid, cid, au, x):
    """Per-output bound of the float-float product for x of shape (K, V, 3)."""
    blocks = np.bincount(rid, minlength=V) + np.bincount(cid[rid != cid], minlength=V)
    m = 3.0 * blocks
    gamma = ((3 * m + 1) * (m + 4) + 6) * U * U  # (V,)
    absax = pcg.spmv(rid, cid, np.abs(au), np.abs(x))  # (K, V, 3)
    return (gamma[None, :, None] * absax).reshape(x.shape[0], -1), absax.reshape(x.shape[0], -1)


def _spmv(B, ctx, mat, x, variant):
    K = x.shape[0]
    y = torch.full((K, x[0].size), np.nan, dtype=torch.float64, device="cuda")
    B.gs_spmv(ctx, mat, dev(x.reshape(K, -1), torch.float64), y, nrhs=K, variant=variant)
    return y.cpu().numpy()


@pytest.mark.parametrize("name", ["cube8", "cube11"])
@pytest.mark.parametrize("nrhs", [1, 3, 8, 12])
@pytest.mark.parametrize("lanes,ws,rpp", [(1, 1, 8), (2, 1, 8), (4, 1, 8), (8, 1, 8), (2, 0, 8), (2, 1, 4), (2, 1, 2),
                                          (2, 0, 2), (2, 1, 1)])
def test_ff_spmv_within_its_bound(B, ctx, name, nrhs, lanes, ws, rpp):
    s = case(name)
    V = s.n_vertices
    B.gs_tune_set(ctx, B.GS_TUNE_SPMV_LANES, lanes)
    B.gs_tune_set(ctx, B.GS_TUNE_SPMV_WS, ws)
    B.gs_tune_set(ctx, B.GS_TUNE_SPMV_FF_RHS, rpp)
    try:
        mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32),
                            dev(s.blocks, torch.float64))
        rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
        x = np.random.default_rng(nrhs).normal(size=(nrhs, V, 3))
        y = _spmv(B, ctx, mat, x, B.GS_SPMV_ROW_FF)
        y0 = pcg.spmv(rid, cid, au, x).reshape(nrhs, -1)
        bound, absax = ff_bound(V, rid, cid, au, x)
        err = np.abs(y - y0)
        assert np.all(err <= bound), (err / bound).max()
        print(name, nrhs, lanes, ws, rpp, "max error / (1e-13 |A||x|):", (err / (1e-13 * absax)).max())
        # bit-reproducible
        assert np.array_equal(y, _spmv(B, ctx, mat, x, B.GS_SPMV_ROW_FF))
        B.gs_mat_destroy(mat)
    finally:
        B.gs_tune_set(ctx, B.GS_TUNE_SPMV_LANES, 2)
        B.gs_tune_set(ctx, B.GS_TUNE_SPMV_WS, 1)
        B.gs_tune_set(ctx, B.GS_TUNE_SPMV_FF_RHS, 8)


def test_ff_spmv_scale_invariance_and_zero_rhs(B, ctx):
    # The operand is scaled by powers of two per RHS, so scaling x by 2^e
    # scales y by exactly 2^e (far outside the float range), and an all-zero
    # RHS gives an all-zero result next to non-zero ones.
    s = case("cube8")
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    x = np.random.default_rng(3).normal(size=(4, V, 3))
    x[2] = 0.0
    y = _spmv(B, ctx, mat, x, B.GS_SPMV_ROW_FF)
    assert np.all(y[2] == 0.0)
    for e in (-600, 600):
        ys = _spmv(B, ctx, mat, np.ldexp(x, e), B.GS_SPMV_ROW_FF)
        assert np.array_equal(ys, np.ldexp(y, e)), e
    B.gs_mat_destroy(mat)


def test_ff_spmv_rows_of_very_different_scales(B, ctx):
    # D A D with D = 10^6 on a third of the nodes: rows differ by 1e12 in
    # scale and the per-row power-of-two scaling of the matrix has to keep
    # every row's error relative to its own |A||x|.
    s = case("cube11")
    V = s.n_vertices
    d = np.where(np.random.default_rng(4).random(V) < 1 / 3, 1e6, 1.0)
    blocks = s.blocks * (d[s.rows][:, None, None] * d[s.cols][:, None, None])
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(blocks, torch.float64))
    rid, cid, au = assembly.assemble(s.rows, s.cols, blocks)
    x = np.random.default_rng(5).normal(size=(3, V, 3)) / d[None, :, None]
    y = _spmv(B, ctx, mat, x, B.GS_SPMV_ROW_FF)
    y0 = pcg.spmv(rid, cid, au, x).reshape(3, -1)
    bound, _ = ff_bound(V, rid, cid, au, x)
    assert np.all(np.abs(y - y0) <= bound)
    B.gs_mat_destroy(mat)


class _Built:
    def __init__(self, B, ctx, s, N, L):
        V = s.n_vertices
        self.V = V
        self.mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32),
                                 dev(s.blocks, torch.float64))
        self.map, nd = B.gs_partition(s.X, N)
        self.mas = B.gs_build_mas(ctx, self.mat, dev(self.map, torch.int32), nd, dev(s.adj_ptr, torch.int32),
                                  dev(s.adj, torch.int32), dev(s.contacts, torch.int32), domain_size=N,
                                  max_levels=L)
        self.rid, self.cid, self.au = assembly.assemble(s.rows, s.cols, s.blocks)
        self.omas = mas.build_mas(self.map, N, L, s.adj_ptr, s.adj, s.contacts, self.rid, self.cid, self.au)
        self.B = B

    def close(self):
        self.B.gs_mas_destroy(self.mas)
        self.B.gs_mat_destroy(self.mat)


@pytest.mark.parametrize("name,N,L", [("cube8", 16, 3), ("cube11", 32, 3), ("plain16", 32, 2)])
def test_ff_pcg_converges_like_oracle(B, ctx, name, N, L):
    bt = _Built(B, ctx, case(name), N, L)
    V, nrhs = bt.V, 4
    b = rhs(3 * V, nrhs)
    b[2] = 0.0
    x = torch.zeros((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    it, rel, _ = B.gs_pcg_solve(ctx, bt.mat, bt.mas, dev(b, torch.float64), x, nrhs=nrhs, tol=1e-6,
                                variant=B.GS_SPMV_ROW_FF)
    mv = lambda v: pcg.spmv(bt.rid, bt.cid, bt.au, v.reshape(-1, 3)).ravel()
    x0, it0, _ = pcg.pcg(mv, lambda v: bt.omas(v), b, tol=1e-6)
    xg = x.cpu().numpy()
    assert it[2] == 0 and np.all(xg[2] == 0)
    for q in (0, 1, 3):
        true = np.linalg.norm(b[q] - mv(xg[q])) / np.linalg.norm(b[q])
        assert true <= 1.05e-6 and rel[q] <= 1e-6
        assert abs(int(it[q]) - int(it0[q])) <= 1, (list(it), list(it0))
        assert np.linalg.norm(xg[q] - x0[q]) / np.linalg.norm(x0[q]) <= 1e-5
    bt.close()


@pytest.mark.parametrize("k", [1, 5, 25])
def test_ff_pcg_fixed_iterations_follow_oracle_recurrence(B, ctx, k):
    # Along the same Krylov recurrence every product differs from the exact
    # one by the float-float rounding (measured up to 1.75e-13 (|A||x|)_i,
    # about 1e3 times FP64's), and CG amplifies per-step differences: on this
    # E = 1e8 cube a relative perturbation of 1e-16 per product already moves
    # the 25th iterate by 1e-10.  So the bound is the FP64 path's 1e-9, or ten
    # times the oracle's own spread when its products are perturbed by
    # 2e-13 (|A||x|)_i with seeded random signs, whichever is larger.
    bt = _Built(B, ctx, case("cube11"), 32, 3)
    V, nrhs = bt.V, 3
    b = rhs(3 * V, nrhs)
    x = torch.zeros((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    it, _, st = B.gs_pcg_solve(ctx, bt.mat, bt.mas, dev(b, torch.float64), x, nrhs=nrhs, tol=0.0, max_iter=k,
                               raise_on_maxiter=False, variant=B.GS_SPMV_ROW_FF)
    assert st == B.GS_ERR_MAXITER and list(it) == [k] * nrhs
    mv = lambda v: pcg.spmv(bt.rid, bt.cid, bt.au, v.reshape(-1, 3)).ravel()
    x0, _, _ = pcg.pcg(mv, lambda v: bt.omas(v), b, fixed_iters=k)
    rng = np.random.default_rng(77)
    absa = np.abs(bt.au)

    def mv_perturbed(v):
        ab = pcg.spmv(bt.rid, bt.cid, absa, np.abs(v).reshape(-1, 3)).ravel()
        return mv(v) + 2e-13 * ab * rng.uniform(-1.0, 1.0, size=ab.shape)

    x1, _, _ = pcg.pcg(mv_perturbed, lambda v: bt.omas(v), b, fixed_iters=k)
    xg = x.cpu().numpy()
    for q in range(nrhs):
        rms = np.sqrt(np.mean(x0[q] ** 2))
        spread = np.max(np.abs(x1[q] - x0[q]) / (np.abs(x0[q]) + rms))
        tol = max(1e-9, 10.0 * spread)
        assert np.all(np.abs(xg[q] - x0[q]) <= tol * (np.abs(x0[q]) + rms)), (q, tol)
    bt.close()
