"""FP64 MAS products on the BF16 tensor cores by exact digit splitting (every
partial product exact in the FP32 accumulator) against the FP64-core kernel
and the oracle.

GS_TUNE_F64_TC = 1 / 2: both operands cut into 7 base-256 digits, 7 BF16 digit
matrices per inverse.  Error model per output (i, k) with a_i, b_k the row /
column exponents (|M_ij| < 2^(a_i-1), |r_jk| < 2^(b_k-1)):
  |dz| <= 2^(a_i-57) sum_j |r_jk| + 2^(b_k-57) sum_j |M_ij| + 2^(a_i+b_k-56).

GS_TUNE_F64_TC = 3: the symmetric inverse scaled by D = diag(2^c_i),
c_i = ceil(e_i / 2) with max_k |M_ik| < 2^e_i, so every entry of D^-1 M D^-1 is
below 1; its block lower triangle stored as 8 base-128 digit bytes per entry,
r~ = D r cut into 8 digits with column exponent b_k (|r~_jk| < 2^(b_k-1)):
  |dz| <= 2^(c_i-56) sum_j 2^c_j |r_jk| + 2^(b_k-57) sum_j |M_ij| 2^-c_j
          + 2^(c_i+b_k-61).

Both plus the FP64 rounding of the final combination and of the coarse-level
sum, covered by 3e-14 (|M||r|)."""

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


def exps(a, axis):
    """Per-row (axis=1) or per-column (axis=0) exponent e with |a| < 2^(e-1)."""
    m = np.max(np.abs(a), axis=axis)
    e = np.where(m > 0, np.frexp(m)[1] + 1, -1000)
    return e


def sym_terms(M, rk):
    """Per-entry bound of the symmetric digit-byte product (GS_TUNE_F64_TC = 3)
    for one domain: M (ld, ld), rk (ld,) one right-hand side."""
    R = np.max(np.abs(M), axis=1)
    e = np.frexp(R)[1]  # R < 2^e
    c = np.where(R > 0, -((-e) // 2), 0).astype(np.float64)  # ceil(e / 2)
    live = R > 0
    rt = np.where(live, np.abs(rk) * 2.0 ** c, 0.0)
    b = np.frexp(np.max(rt))[1] + 1  # |r~| < 2^(b - 1)
    bnd = (2.0 ** (c - 56)) * rt.sum() + (2.0 ** (b - 57)) * (np.abs(M) * np.where(live, 2.0 ** -c, 0.0)).sum(1) \
        + 2.0 ** (c + b - 61)
    return np.where(live, bnd, 0.0)


def split_bound(om, r, sym=False):
    """The bound above summed over the levels (every level's product is split the
    same way), prolongated to the nodes, for r of shape (nrhs, V, 3)."""
    lv, N = om.levels, om.levels.N
    V = lv.coarse[0].size
    nrhs = r.shape[0]
    out = np.zeros((nrhs, V, 3))
    for l, inv in enumerate(om.invs):
        C = om.C[l]  # items (padded) x nodes, 0/1
        nd = inv.shape[0]
        bnd_items = np.zeros((nrhs, nd * N, 3))
        for k in range(nrhs):
            rl = (C @ r[k]).reshape(nd, 3 * N)  # restricted r of every domain of the level
            for d in range(nd):
                M = inv[d]
                rk = rl[d]
                if not np.any(M) or not np.any(rk):
                    continue
                if sym:
                    bnd = sym_terms(M, rk)
                else:
                    a = exps(M, 1)
                    b = exps(rk, 0)
                    bnd = (2.0 ** (a - 57)) * np.abs(rk).sum() + (2.0 ** (b - 57)) * np.abs(M).sum(1) \
                        + 2.0 ** (a + b - 56)
                bnd_items[k, d * N : d * N + N] = bnd.reshape(N, 3)
        for k in range(nrhs):
            out[k] += C.T @ bnd_items[k]
    return out.reshape(nrhs, -1)


def _build(B, ctx, s, N, L, tc):
    """Matrix and preconditioner; the digit storage follows GS_TUNE_F64_TC at build time."""
    B.gs_tune_set(ctx, B.GS_TUNE_F64_TC, tc)
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, N)
    M = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32),
                       dev(s.contacts, torch.int32), domain_size=N, max_levels=L)
    return mat, M, mp


@pytest.mark.parametrize("n,N,L,nrhs", [(11, 32, 3, 1), (11, 32, 3, 3), (11, 32, 3, 8), (9, 16, 2, 5),
                                        (7, 32, 1, 8), (12, 16, 3, 8)])
def test_digit_split_apply_matches_fp64(B, ctx, n, N, L, nrhs):
    s = make_tet_system(n, E=1e8, n_contacts=60, contact_mode="near", seed=70 + n)
    V = s.n_vertices
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    r = np.random.default_rng(nrhs).normal(size=(nrhs, 3 * V)) * np.logspace(-2, 2, 3 * V)
    z = torch.empty((nrhs, 3 * V), dtype=torch.float64, device="cuda")
    out, invs = {}, {}
    # symmetric digit bytes; BF16 digit matrices (one CTA per domain, then the
    # persistent schedule and 256-thread CTAs on the same storage); FP64 cores.  Each build's own
    # inverses are exported: builds may differ in the last bits of the coarse
    # level matrices (their sums are not ordered), amplified by the condition.
    for built, tcs in ((3, (3,)), (1, (1, 2, 4)), (0, (0,))):
        mat, M, mp = _build(B, ctx, s, N, L, built)
        L_, items = B.gs_mas_info(M)
        inv = [B.gs_mas_export_inverse(ctx, M, l, -(-items[l] // N), N).cpu().numpy() for l in range(L_)]
        for tc in tcs:
            B.gs_tune_set(ctx, B.GS_TUNE_F64_TC, tc)
            B.gs_mas_apply(ctx, M, dev(r, torch.float64), z, nrhs=nrhs)
            out[tc] = z.cpu().numpy()
            invs[tc] = inv
        B.gs_mas_destroy(M)
        B.gs_mat_destroy(mat)
    B.gs_tune_set(ctx, B.GS_TUNE_F64_TC, 4)  # the default
    om = mas.build_mas(mp, N, L, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    ref = {}
    for tc in (3, 1, 2, 4, 0):
        # the library's own FP64 inverses (they match the oracle's to ~cond * 1e-16,
        # checked by the parity tests) through the oracle's Eq. 6 apply
        z0 = mas.apply(om.levels, invs[tc], r, om.C)
        absz = mas.apply(om.levels, [np.abs(v) for v in invs[tc]], np.abs(r), om.C)
        ref[tc] = (z0, absz)
    z0, absz = ref[0]
    assert np.all(np.abs(out[0] - z0) <= 3e-14 * absz + 1e-300)  # FP64 cores: reordered FP64 sums (<= 99 terms)
    # the BF16-digit schedules compute the same integers and round them the same
    # way; they differ only through the order of the FP64 coarse sums (the two
    # per-domain forms, 128 or 256 threads, not at all)
    assert np.all(np.abs(out[1] - out[2]) <= 1e-14 * ref[1][1] + 1e-300)
    assert np.array_equal(out[1], out[4])
    for tc, sym in ((1, False), (2, False), (4, False), (3, True)):
        z0, absz = ref[tc]
        om.invs = invs[tc]
        bound = split_bound(om, r.reshape(nrhs, V, 3), sym=sym) + 3e-14 * absz
        assert np.all(np.abs(out[tc] - z0) <= bound + 1e-300), (tc, np.max(np.abs(out[tc] - z0) / (bound + 1e-300)))
        print(f"F64_TC={tc}: max |tc - FP64 product| / (|M||r|):", float(np.max(np.abs(out[tc] - z0) / (absz + 1e-300))))


def test_fp64_pcg_with_digit_split_apply_follows_the_oracle(B, ctx):
    s = make_tet_system(12, E=1e7, n_contacts=100, contact_mode="near", seed=91)
    V, N, L, nrhs = s.n_vertices, 32, 3, 4
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    A = pcg.SymmetricMatrix(V, rid, cid, au)
    b = rhs(3 * V, nrhs)
    its = {}
    for tc in (3, 1, 2, 4, 0):
        mat, M, mp = _build(B, ctx, s, N, L, tc)
        if tc == 3:
            om = mas.build_mas(mp, N, L, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
            xo, it_o, _ = pcg.pcg(A, om, b, tol=1e-6)
        x = torch.zeros((nrhs, 3 * V), dtype=torch.float64, device="cuda")
        it, _, _ = B.gs_pcg_solve(ctx, mat, M, dev(b, torch.float64), x, nrhs=nrhs, tol=1e-6)
        xg = x.cpu().numpy()
        for k in range(nrhs):
            assert abs(int(it[k]) - int(it_o[k])) <= 1, (tc, list(it), list(it_o))
            assert np.linalg.norm(b[k] - A(xg[k])) <= 1.05e-6 * np.linalg.norm(b[k])
            assert np.linalg.norm(xg[k] - xo[k]) <= 1e-5 * np.linalg.norm(xo[k])
        its[tc] = list(it)
        B.gs_mas_destroy(M)
        B.gs_mat_destroy(mat)
    B.gs_tune_set(ctx, B.GS_TUNE_F64_TC, 4)  # the default
    print("iterations sym bytes / bf16 digits / persistent / fp64 cores / oracle:", its[3], its[1], its[2], its[0],
          list(it_o))
