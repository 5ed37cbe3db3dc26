"""CUDA path vs the FP64 oracle, through the C ABI, on small seeded systems.

Integer work (keys, partition, level maps) must match bit for bit.  Floating
point is compared against bounds derived from the arithmetic: a sum of m
terms evaluated in another order differs by at most about m * eps * sum|t|,
so reductions are checked against (sum of |terms|) * 1e-13, and quantities
that pass through a domain inverse against cond(domain) * 1e-13.
"""

import numpy as np
import pytest
import torch

import fp64bounds
from oracle import assembly, mas, partition, pcg
from synth.workloads import make_tet_system, plain_small, rhs

pytestmark = pytest.mark.gpu

EPS_SUM = 1e-13


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
        elif name == "cube11":  # 1331 vertices: ragged last domain for N = 32 and 16
            _CASES[name] = make_tet_system(11, E=1e8, n_contacts=120, contact_mode="near", seed=12)
        elif name == "plain16":
            _CASES[name] = plain_small()
    return _CASES[name]


class Built:
    def __init__(self, B, ctx, s, N=32, L=2, prec=0):
        self.s = s
        V = s.n_vertices
        self.V = V
        self.mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32),
                                 dev(s.blocks, torch.float64))
        self.map, self.ndom = B.gs_partition(s.X, N)
        self.mas = B.gs_build_mas(ctx, self.mat, dev(self.map, torch.int32), self.ndom, dev(s.adj_ptr, torch.int32),
                                  dev(s.adj, torch.int32), dev(s.contacts, torch.int32), domain_size=N,
                                  max_levels=L, precision=prec)
        self.rid, self.cid, self.au = assembly.assemble(s.rows, s.cols, s.blocks)
        self.omas = mas.build_mas(self.map, N, L, s.adj_ptr, s.adj, s.contacts, self.rid, self.cid, self.au)
        self.B = B
        self.N = N

    def close(self):
        self.B.gs_mas_destroy(self.mas)
        self.B.gs_mat_destroy(self.mat)


# ------------------------------------------------------------------ assembly (Sec. 5.2)
@pytest.mark.parametrize("name", ["cube8", "cube11", "plain16"])
def test_assembly_keys_exact_values_bounded(B, ctx, name):
    s = case(name)
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    rid, cid, au = B.gs_mat_export(ctx, mat)
    r0, c0, a0 = assembly.assemble(s.rows, s.cols, s.blocks)
    _, _, abs_sum = assembly.assemble(s.rows, s.cols, np.abs(s.blocks))
    assert np.array_equal(rid.cpu().numpy(), r0) and np.array_equal(cid.cpu().numpy(), c0)
    assert np.all(np.abs(au.cpu().numpy() - a0) <= EPS_SUM * abs_sum + 1e-300)
    B.gs_mat_destroy(mat)


def test_assembly_duplicates_lower_inputs_and_warp_crossing_runs(B, ctx):
    rng = np.random.default_rng(7)
    n = 50
    rows = rng.integers(0, n, 20000).astype(np.int32)
    cols = rng.integers(0, n, 20000).astype(np.int32)
    # one key repeated 3000 times: a run spanning ~100 warps (atomic path)
    rows[:3000], cols[:3000] = 3, 17
    blocks = rng.normal(size=(20000, 3, 3))
    perm = rng.permutation(20000)
    rows, cols, blocks = rows[perm], cols[perm], blocks[perm]
    mat = B.gs_assemble(ctx, n, dev(rows, torch.int32), dev(cols, torch.int32), dev(blocks, torch.float64))
    rid, cid, au = B.gs_mat_export(ctx, mat)
    r0, c0, a0 = assembly.assemble(rows, cols, blocks)
    _, _, abs_sum = assembly.assemble(rows, cols, np.abs(blocks))
    assert np.array_equal(rid.cpu().numpy(), r0) and np.array_equal(cid.cpu().numpy(), c0)
    assert np.all(np.abs(au.cpu().numpy() - a0) <= EPS_SUM * abs_sum)
    B.gs_mat_destroy(mat)


def test_assembly_edge_cases(B, ctx):
    e32 = torch.zeros(0, dtype=torch.int32, device="cuda")
    e64 = torch.zeros((0, 3, 3), dtype=torch.float64, device="cuda")
    mat = B.gs_assemble(ctx, 5, e32, e32, e64)
    assert B.gs_mat_info(mat) == (5, 0)
    B.gs_mat_destroy(mat)
    # only lower-triangle inputs: nothing is consumed
    r = dev([3, 4], torch.int32)
    c = dev([1, 0], torch.int32)
    mat = B.gs_assemble(ctx, 5, r, c, dev(np.ones((2, 3, 3)), torch.float64))
    assert B.gs_mat_info(mat) == (5, 0)
    B.gs_mat_destroy(mat)
    # out-of-range index is rejected
    with pytest.raises(B.GsError) as e:
        B.gs_assemble(ctx, 5, dev([0, 5], torch.int32), dev([1, 1], torch.int32), dev(np.ones((2, 3, 3)), torch.float64))
    assert e.value.status == B.GS_ERR_INVALID


# ------------------------------------------------------------------ ABD two-level reduction (Sec. 5.1)
def test_abd_two_level_matches_oracle(B, ctx):
    rng = np.random.default_rng(8)
    n_fem, n_bodies, per = 40, 6, 8
    n_full = n_fem + n_bodies * per
    body = np.array([-1] * n_fem + [b for b in range(n_bodies) for _ in range(per)], dtype=np.int32)
    xbar = rng.normal(size=(n_full, 3))
    K = 3000
    # node indices, plus the bodies' own reduced rows n_full + 4b + a (12 x 12 body Hessians)
    rows = rng.integers(0, n_full + 4 * n_bodies, K).astype(np.int32)
    cols = rng.integers(0, n_full + 4 * n_bodies, K).astype(np.int32)
    lo, hi = np.minimum(rows, cols), np.maximum(rows, cols)
    blocks = rng.normal(size=(K, 3, 3))
    mat = B.gs_assemble_abd(ctx, n_full, n_fem, n_bodies, dev(body, torch.int32), dev(xbar, torch.float64),
                            dev(lo, torch.int32), dev(hi, torch.int32), dev(blocks, torch.float64))
    rid, cid, au = B.gs_mat_export(ctx, mat)
    r0, c0, a0 = assembly.assemble_abd(lo, hi, blocks, body, xbar, n_fem)
    assert np.array_equal(rid.cpu().numpy(), r0) and np.array_equal(cid.cpu().numpy(), c0)
    scale = np.abs(a0).max()
    assert np.abs(au.cpu().numpy() - a0).max() <= 1e-12 * scale * 50
    B.gs_mat_destroy(mat)


# ------------------------------------------------------------------ SpMV (Sec. 5.3)
@pytest.mark.parametrize("name", ["cube8", "cube11"])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 3, 8])
def test_spmv_matches_oracle(B, ctx, name, variant, nrhs):
    s = case(name)
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    x = np.random.default_rng(nrhs).normal(size=(nrhs, V, 3))
    y = torch.empty((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    B.gs_spmv(ctx, mat, dev(x.reshape(nrhs, -1), torch.float64), y, nrhs=nrhs, variant=variant)
    y0 = pcg.spmv(rid, cid, au, x).reshape(nrhs, -1)
    bound = pcg.spmv(rid, cid, np.abs(au), np.abs(x)).reshape(nrhs, -1) * EPS_SUM
    assert np.all(np.abs(y.cpu().numpy() - y0) <= bound)
    if variant == 1:  # row gather is bit-reproducible
        y2 = torch.empty_like(y)
        B.gs_spmv(ctx, mat, dev(x.reshape(nrhs, -1), torch.float64), y2, nrhs=nrhs, variant=variant)
        assert torch.equal(y, y2)
    B.gs_mat_destroy(mat)


# ------------------------------------------------------------------ MAS (Sec. 3, supp. Alg. 2-5, Eq. 4-6)
@pytest.mark.parametrize("name,N,L", [("cube8", 16, 3), ("cube11", 32, 3), ("cube11", 16, 4), ("plain16", 32, 2),
                                      ("cube11", 5, 5)])
def test_mas_levels_bit_exact(B, ctx, name, N, L):
    bt = Built(B, ctx, case(name), N=N, L=L)
    nl, items = B.gs_mas_info(bt.mas)
    assert nl == bt.omas.levels.n_levels
    assert items == [int(v) for v in bt.omas.levels.n_items]
    for l in range(nl):
        c = B.gs_mas_export_coarse(ctx, bt.mas, l, bt.V).cpu().numpy()
        assert np.array_equal(c, bt.omas.levels.coarse[l]), f"level {l}"
    bt.close()


def _domain_cond(Md, real):
    idx = (3 * np.nonzero(real)[0][:, None] + np.arange(3)).ravel()
    return np.linalg.cond(Md[np.ix_(idx, idx)]) if idx.size else 1.0


@pytest.mark.parametrize("name,N,L", [("cube8", 16, 3), ("cube11", 32, 3), ("plain16", 32, 2)])
def test_mas_inverses_match_oracle(B, ctx, name, N, L):
    bt = Built(B, ctx, case(name), N=N, L=L)
    lv = bt.omas.levels
    for l in range(lv.n_levels):
        nd = lv.n_domains(l)
        inv = B.gs_mas_export_inverse(ctx, bt.mas, l, nd, N).cpu().numpy()
        real = np.zeros(nd * N, dtype=bool)
        real[: lv.n_items[l]] = lv.real[l]
        for d in range(nd):
            ref = bt.omas.invs[l][d]
            kappa = _domain_cond(bt.omas.mats[l][d], real[d * N : d * N + N])
            err = np.linalg.norm(inv[d] - ref) / max(np.linalg.norm(ref), 1e-300)
            assert err <= EPS_SUM * kappa * 10 + 1e-14, (l, d, err, kappa)
            pad = ~np.repeat(real[d * N : d * N + N], 3)
            assert np.all(inv[d][pad] == 0) and np.all(inv[d][:, pad] == 0)
    bt.close()


@pytest.mark.parametrize("name,N,L", [("cube8", 16, 3), ("cube11", 32, 3), ("cube11", 7, 4)])
@pytest.mark.parametrize("nrhs", [1, 4, 8])
def test_mas_apply_matches_oracle(B, ctx, name, N, L, nrhs):
    bt = Built(B, ctx, case(name), N=N, L=L)
    V = bt.V
    r = np.random.default_rng(nrhs).normal(size=(nrhs, 3 * V))
    z = torch.empty((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    B.gs_mas_apply(ctx, bt.mas, dev(r, torch.float64), z, nrhs=nrhs)
    z0 = bt.omas(r)
    # entry by entry: sum reordering plus each domain's inverse error
    bound = fp64bounds.apply_bound(bt.omas, r)
    dz = np.abs(z.cpu().numpy() - z0)
    assert np.all(dz <= bound), (dz / bound).max()
    bt.close()


def test_mas_rejects_indefinite(B, ctx):
    rows = dev([0, 0, 1], torch.int32)
    cols = dev([0, 1, 1], torch.int32)
    blocks = dev(np.stack([np.eye(3), 2 * np.eye(3), np.eye(3)]), torch.float64)
    mat = B.gs_assemble(ctx, 2, rows, cols, blocks)
    with pytest.raises(B.GsError) as e:
        B.gs_build_mas(ctx, mat, dev([0, 1], torch.int32), 1, dev([0, 1, 2], torch.int32), dev([1, 0], torch.int32),
                       None, domain_size=2, max_levels=1)
    assert e.value.status == B.GS_ERR_NOT_SPD
    B.gs_mat_destroy(mat)


# ------------------------------------------------------------------ PCG (Sec. 3.2)
@pytest.mark.parametrize("name,N,L", [("cube8", 16, 3), ("cube11", 32, 3)])
@pytest.mark.parametrize("k", [1, 5, 25])
def test_pcg_fixed_iterations_follow_oracle_recurrence(B, ctx, name, N, L, k):
    bt = Built(B, ctx, case(name), N=N, L=L)
    V, nrhs = bt.V, 3
    b = rhs(3 * V, nrhs)
    x = torch.zeros((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    it, _, st = B.gs_pcg_solve(ctx, bt.mat, bt.mas, dev(b, torch.float64), x, nrhs=nrhs, tol=0.0, max_iter=k,
                               raise_on_maxiter=False)
    assert st == B.GS_ERR_MAXITER and list(it) == [k] * nrhs
    mv = lambda v: pcg.spmv(bt.rid, bt.cid, bt.au, v.reshape(-1, 3)).ravel()
    x0, _, _ = pcg.pcg(mv, lambda v: bt.omas(v), b, fixed_iters=k)
    # entry by entry along the same recurrence: rounding differences, relative
    # to the entry with a floor at the RHS's root-mean-square entry
    xg = x.cpu().numpy()
    for q in range(nrhs):
        rms = np.sqrt(np.mean(x0[q] ** 2))
        assert np.all(np.abs(xg[q] - x0[q]) <= 1e-9 * (np.abs(x0[q]) + rms)), q
    bt.close()


@pytest.mark.parametrize("name,N,L", [("cube8", 16, 3), ("cube11", 32, 3), ("plain16", 32, 2)])
@pytest.mark.parametrize("variant", [0, 1])
def test_pcg_converges_like_oracle(B, ctx, name, N, L, variant):
    bt = Built(B, ctx, case(name), N=N, L=L)
    V, nrhs = bt.V, 4
    b = rhs(3 * V, nrhs)
    b[2] = 0.0  # a zero right-hand side: x = 0, no iterations
    x = torch.zeros((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    it, rel, _ = B.gs_pcg_solve(ctx, bt.mat, bt.mas, dev(b, torch.float64), x, nrhs=nrhs, tol=1e-6, variant=variant)
    mv = lambda v: pcg.spmv(bt.rid, bt.cid, bt.au, v.reshape(-1, 3)).ravel()
    x0, it0, _ = pcg.pcg(mv, lambda v: bt.omas(v), b, tol=1e-6)
    xg = x.cpu().numpy()
    assert it[2] == 0 and np.all(xg[2] == 0)
    for q in (0, 1, 3):
        true = np.linalg.norm(b[q] - mv(xg[q])) / np.linalg.norm(b[q])
        assert true <= 1.05e-6 and rel[q] <= 1e-6
        assert abs(int(it[q]) - int(it0[q])) <= 1
        assert np.linalg.norm(xg[q] - x0[q]) / np.linalg.norm(x0[q]) <= 1e-5
    bt.close()


def test_one_level_apply_is_block_jacobi(B, ctx):
    s = make_tet_system(4, E=1e6, n_contacts=3, seed=5)  # 64 vertices: two domains of 32
    bt = Built(B, ctx, s, N=32, L=2)
    V = bt.V
    r = np.random.default_rng(1).normal(size=(1, 3 * V))
    bt1 = Built(B, ctx, s, N=32, L=1)
    z = torch.empty((1, 3 * V), dtype=torch.float64, device="cuda")
    B.gs_mas_apply(ctx, bt1.mas, dev(r, torch.float64), z, nrhs=1)
    A = assembly.to_dense(V, bt.rid, bt.cid, bt.au)
    part = bt.map // 32
    zz = np.zeros(3 * V)
    bound = np.zeros(3 * V)
    for q in range(part.max() + 1):
        nodes = np.nonzero(part == q)[0]
        idx = (3 * nodes[:, None] + np.arange(3)).ravel()
        Ad = A[np.ix_(idx, idx)]
        zz[idx] = np.linalg.solve(Ad, r[0][idx])
        # entry by entry, the two terms of the apply bound in fp64bounds: the
        # sums' rounding and the domain inverse's error (kappa_d ||A_d^-1||_2 ||r_d||_2)
        ev = np.linalg.eigvalsh(Ad)
        inv_abs = np.abs(np.linalg.inv(Ad))
        bound[idx] = (fp64bounds.C_SUM * (inv_abs @ np.abs(r[0][idx]))
                      + fp64bounds.C_DOMAIN * (ev[-1] / ev[0]) / ev[0] * np.linalg.norm(r[0][idx]))
    assert np.all(np.abs(z.cpu().numpy()[0] - zz) <= bound)
    bt.close()
    bt1.close()
