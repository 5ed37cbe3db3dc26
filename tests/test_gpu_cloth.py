"""Stiff-cloth element Hessians on the device (gs_cloth_*: membrane with the
cubic strain limit of Sec. 4, hinge bending, lumped masses) against the
oracle (oracle/cloth.py), triplet by triplet in the emission order, on a small
sheet in full and on the 512 x 512 sheet by sampled elements; the assembled
matrix against the independent input generator; bad inputs rejected."""

import numpy as np
import pytest
import torch

from oracle import assembly, cloth
from synth.cloth import hinges, make_cloth_system, sheet

pytestmark = pytest.mark.gpu

PARAMS = dict(E=1e8, lam=0.05e6, thickness=1e-3, rho=200.0, dt=0.01)


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


def deformed(n, seed=1003):
    """The generator's deformation of the n x n sheet (same draws)."""
    X, tris = sheet(n)
    rng = np.random.default_rng(seed)
    h = 1.0 / (n - 1)
    sh = rng.uniform(0.0, 0.1)
    x = X @ np.array([[1.02, sh, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]).T + rng.normal(0.0, 0.01 * h, X.shape)
    return X, x, tris, hinges(tris)


def block_close(got, ref, rtol=1e-11):
    """Per block: |got - ref| <= rtol * max|ref block| (entries of one block share its scale)."""
    scale = np.abs(ref).reshape(ref.shape[0], -1).max(axis=1)[:, None, None]
    return np.abs(got - ref) <= rtol * scale + 1e-300


def device_triplets(B, ctx, X, x, tris, hg, params=PARAMS):
    c = B.gs_cloth_create(ctx, dev(X, torch.float64), dev(tris, torch.int32), dev(hg, torch.int32), **params)
    try:
        r, cc, b = B.gs_cloth_triplets(ctx, c, dev(x, torch.float64))
        return r.cpu().numpy(), cc.cpu().numpy(), b.cpu().numpy()
    finally:
        B.gs_cloth_destroy(c)


@pytest.mark.parametrize("n,stretch", [(24, 1.02), (17, 1.15), (9, 0.9)])
def test_cloth_triplets_match_the_oracle_one_by_one(B, ctx, n, stretch):
    # stretch 1.15: every membrane direction past the strain limit; 0.9: the
    # stretching Hessian's clamp active and the strain limit off
    X, x, tris, hg = deformed(n)
    x = x.copy()
    x[:, 0] *= stretch / 1.02
    r, c, b = device_triplets(B, ctx, X, x, tris, hg)
    r0, c0, b0 = cloth.cloth_triplets(X, x, tris, hg, **PARAMS)
    assert np.array_equal(r, r0) and np.array_equal(c, c0)
    ok = block_close(b, b0)
    assert ok.all(), np.argwhere(~ok)[:5]


def test_stiffness_contrast_keeps_every_block_accurate(B, ctx):
    # E / lam = 2e5 with only the x direction past the strain limit: a vertex
    # block mixing mostly the soft direction is tiny next to the stiff ones,
    # and must still carry its own relative accuracy (a block formed as the
    # difference of two large ones would not)
    X, x, tris, hg = deformed(17)
    x = x.copy()
    x[:, 0] *= 1.3 / 1.02
    params = dict(PARAMS, E=1e10)
    r, c, b = device_triplets(B, ctx, X, x, tris, hg, params)
    r0, c0, b0 = cloth.cloth_triplets(X, x, tris, hg, **params)
    assert np.array_equal(r, r0) and np.array_equal(c, c0)
    m = 6 * len(tris)  # the membrane blocks, then bending and masses at the usual bound
    ok = block_close(b[:m], b0[:m], rtol=1e-12)
    assert ok.all(), np.argwhere(~ok)[:5]
    assert block_close(b[m:], b0[m:]).all()


def test_full_sheet_sampled_elements_and_masses(B, ctx):
    n = 512
    X, x, tris, hg = deformed(n)
    T, H, V = len(tris), len(hg), X.shape[0]
    r, c, b = device_triplets(B, ctx, X, x, tris, hg)
    assert r.size == 6 * T + 10 * H + V
    rng = np.random.default_rng(9)
    ts = np.sort(rng.choice(T, 2000, replace=False))
    hs = np.sort(rng.choice(H, 2000, replace=False))
    # the oracle on the sampled elements alone (its masses are not compared here)
    r0, c0, b0 = cloth.cloth_triplets(X, x, tris[ts], hg[hs], **PARAMS)
    mi = (6 * ts[:, None] + np.arange(6)).ravel()
    bi = (6 * T + 10 * hs[:, None] + np.arange(10)).ravel()
    for got, k0 in ((mi, slice(0, 6 * len(ts))), (bi, slice(6 * len(ts), 6 * len(ts) + 10 * len(hs)))):
        assert np.array_equal(r[got], r0[k0]) and np.array_equal(c[got], c0[k0])
        assert block_close(b[got], b0[k0]).all()
    w, A = cloth.rest_data(X, tris)
    m = cloth.lumped_masses(V, tris, A, PARAMS["rho"], PARAMS["thickness"]) / PARAMS["dt"] ** 2
    mb = b[6 * T + 10 * H :]
    assert np.array_equal(r[6 * T + 10 * H :], np.arange(V))
    assert np.all(np.abs(mb[:, 0, 0] - m) <= 1e-14 * m) and np.all(mb[:, 0, 1] == 0)


def test_assembled_matrix_equals_the_generators(B, ctx):
    # the device triplets and the independent torch generator's assemble to the
    # same matrix through the library's hash assembly
    n = 64
    s = make_cloth_system(n=n)
    X, x, tris, hg = deformed(n)
    cl = B.gs_cloth_create(ctx, dev(X, torch.float64), dev(tris, torch.int32), dev(hg, torch.int32), **PARAMS)
    V = X.shape[0]
    try:
        r, c, b = B.gs_cloth_triplets(ctx, cl, dev(x, torch.float64))
        m1 = B.gs_assemble(ctx, V, r, c, b)
        m2 = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
        r1, c1, a1 = (t.cpu().numpy() for t in B.gs_mat_export(ctx, m1))
        r2, c2, a2 = (t.cpu().numpy() for t in B.gs_mat_export(ctx, m2))
        assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
        assert np.abs(a1 - a2).max() <= 1e-11 * np.abs(a2).max()
        B.gs_mat_destroy(m1)
        B.gs_mat_destroy(m2)
    finally:
        B.gs_cloth_destroy(cl)


def test_bad_meshes_are_rejected(B, ctx):
    X, x, tris, hg = deformed(6)
    bad = tris.copy()
    bad[3, 1] = X.shape[0]  # out of range
    with pytest.raises(B.GsError) as e:
        B.gs_cloth_create(ctx, dev(X, torch.float64), dev(bad, torch.int32), dev(hg, torch.int32), **PARAMS)
    assert e.value.status == B.GS_ERR_INVALID
    Xd = X.copy()
    Xd[tris[5, 2]] = Xd[tris[5, 0]]  # a rest triangle of zero area
    with pytest.raises(B.GsError) as e:
        B.gs_cloth_create(ctx, dev(Xd, torch.float64), dev(tris, torch.int32), dev(hg, torch.int32), **PARAMS)
    assert e.value.status == B.GS_ERR_NONFINITE
    # the context is still usable
    r, c, b = device_triplets(B, ctx, X, x, tris, hg)
    assert np.isfinite(b).all()
