"""Device elastic bodies against the oracle: rest shapes and masses, the
PSD-projected stable Neo-Hookean element Hessians (Sec. 3.1) emitted as
triplets, the energy and gradient, assembly through the fixed pattern with
springs merged in (Sec. 5.1-5.2), the numeric MAS refresh, and the Newton
loop on the incremental potential (Fig. framework; supplement Eq. 1).

Tolerances.  The device projects with the analytic eigensystem (SVD of F),
the oracle with a numeric 9x9 eigendecomposition; both are backward stable,
and the projection onto the PSD cone is 1-Lipschitz in the Frobenius norm,
so an element's blocks agree to a few hundred ulps of its largest entry:
1e-11 relative leaves margin for near-degenerate singular values.  Sums
(masses, gradients, assembled blocks) differ from the oracle's only in
their order: 1e-13 relative to the sum of the absolute terms."""

import numpy as np
import pytest
import torch

from oracle import assembly, elastic, newton
from synth.workloads import make_elastic_scene

pytestmark = pytest.mark.gpu

E, NU, RHO, DT = 1e5, 0.4, 1000.0, 0.01


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


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def springs_of(s):
    return (s.pairs, s.K, s.rest)


def make_fem(B, ctx, s, E_=E):
    f = B.gs_fem_create(ctx, dev(s.X), dev(s.tets, torch.int32), E_, NU, RHO, DT)
    if len(s.pairs):
        B.gs_fem_set_springs(ctx, f, dev(s.pairs, torch.int32), dev(s.K), dev(s.rest))
    return f


def test_rest_shape_and_lumped_mass(B, ctx):
    s = make_elastic_scene(6, seed=11)
    f = make_fem(B, ctx, s)
    w, vol, mass = B.gs_fem_export_rest(ctx, f, len(s.tets), s.n_vertices)
    vol_o, w_o = elastic.rest_shape(s.X, s.tets)
    m_o = elastic.lumped_mass(s.X, s.tets, RHO)
    assert np.allclose(vol.cpu().numpy(), vol_o, rtol=1e-13, atol=0)
    # w = rows of Dm^-1: entries of size 1/h, each within the inverse's rounding
    assert np.abs(w.cpu().numpy() - w_o).max() <= 1e-12 * np.abs(w_o).max()
    assert np.allclose(mass.cpu().numpy(), m_o, rtol=1e-13, atol=0)
    _, _, mu, lam = B.gs_fem_info(f)
    assert (mu, lam) == pytest.approx(elastic.lame(E, NU), rel=1e-15)
    B.gs_fem_destroy(f)


@pytest.mark.parametrize("flip", [0, 5])
def test_triplets_match_the_oracle_element_by_element(B, ctx, flip):
    s = make_elastic_scene(7, n_springs=40, flip=flip, seed=12 + flip)
    f = make_fem(B, ctx, s)
    T, V, P = len(s.tets), s.n_vertices, len(s.pairs)
    r, c, b = B.gs_fem_triplets(ctx, f, dev(s.x), 10 * T + V + 3 * P)
    ro, co, bo = newton.hessian_triplets(s.X, s.x, s.tets, E, NU, RHO, DT, springs_of(s))
    # the oracle lists the springs' (i, i), (j, j), (min, max) blocks as three runs; the library pair by pair
    n0 = 10 * T + V
    per_pair = lambda a: np.concatenate([a[:n0], a[n0:].reshape(3, P, *a.shape[1:]).swapaxes(0, 1).reshape(-1, *a.shape[1:])])
    ro, co, bo = per_pair(ro), per_pair(co), per_pair(bo)
    assert np.array_equal(r.cpu().numpy(), ro) and np.array_equal(c.cpu().numpy(), co)
    b = b.cpu().numpy()
    be, beo = b[: 10 * T].reshape(T, 10, 9), bo[: 10 * T].reshape(T, 10, 9)
    scale = np.abs(beo).reshape(T, -1).max(axis=1)
    err = np.abs(be - beo).reshape(T, -1).max(axis=1)
    assert np.all(err <= 1e-11 * scale), (err / scale).max()
    # the projection is active: some element Hessians lost negative modes
    He_raw = elastic.element_hessians(s.X, s.x, s.tets, E, NU, project=False)
    assert np.linalg.eigvalsh(He_raw).min() < 0
    assert np.allclose(b[10 * T: 10 * T + V], bo[10 * T: 10 * T + V], rtol=1e-13, atol=0)
    assert np.array_equal(b[10 * T + V:], bo[10 * T + V:])  # spring blocks: copies of K
    B.gs_fem_destroy(f)


def test_energy_and_gradient_match_the_oracle(B, ctx):
    s = make_elastic_scene(8, n_springs=60, flip=9, seed=13)
    f = make_fem(B, ctx, s)
    g = torch.empty((s.n_vertices, 3), dtype=torch.float64, device="cuda")
    e = B.gs_fem_energy(ctx, f, dev(s.x), dev(s.xt), g)
    eo, go = newton.incremental_potential(s.X, s.x, s.tets, E, NU, RHO, DT, s.xt, springs_of(s))
    assert e == pytest.approx(eo, rel=1e-12)
    # element-wise, against the sum of absolute contributions per vertex
    _, gabs = elastic.energy_and_gradient(s.X, s.x, s.tets, E, NU)
    assert np.all(np.abs(g.cpu().numpy() - go) <= 1e-12 * (np.abs(go) + np.abs(gabs).max()))
    # repeatable bit for bit (fixed summation order)
    g2 = torch.empty_like(g)
    assert B.gs_fem_energy(ctx, f, dev(s.x), dev(s.xt), g2) == e and torch.equal(g, g2)
    B.gs_fem_destroy(f)


def _abs_assembled(rows, cols, blocks):
    return assembly.assemble(rows, cols, np.abs(blocks))[2]


def test_assembly_through_the_fixed_pattern_matches_the_oracle(B, ctx):
    s = make_elastic_scene(9, n_springs=300, flip=11, seed=14)
    # springs on element keys (mesh neighbours) and twice on one pair: duplicates across both parts
    extra = np.array([s.tets[0, :2], s.tets[5, 1:3], s.pairs[0]], dtype=np.int32)
    s.pairs = np.concatenate([s.pairs, extra])
    s.K = np.concatenate([s.K, s.K[:3] * 2.0])
    s.rest = np.concatenate([s.rest, s.X[extra[:, 0]] - s.X[extra[:, 1]]])
    f = make_fem(B, ctx, s)
    m = B.gs_fem_assemble(ctx, f, dev(s.x))
    n, U = B.gs_mat_info(m)
    ro, co, bo = newton.hessian_triplets(s.X, s.x, s.tets, E, NU, RHO, DT, springs_of(s))
    rid_o, cid_o, au_o = assembly.assemble(ro, co, bo)
    assert U == len(rid_o) and B.gs_fem_info(f)[0] == U
    rid, cid, au = B.gs_mat_export(ctx, m)
    assert np.array_equal(rid.cpu().numpy(), rid_o) and np.array_equal(cid.cpu().numpy(), cid_o)
    scale = _abs_assembled(ro, co, bo)
    assert np.all(np.abs(au.cpu().numpy().reshape(-1, 3, 3) - au_o) <= 1e-11 * scale + 1e-300)
    B.gs_mat_destroy(m)
    B.gs_fem_destroy(f)


def test_refill_equals_a_fresh_assembly_and_the_sorting_assembly(B, ctx):
    s = make_elastic_scene(8, seed=15)
    f = make_fem(B, ctx, s)
    m = B.gs_fem_assemble(ctx, f, dev(s.X))  # pattern made at rest, values replaced below
    B.gs_fem_refill(ctx, f, dev(s.x), m)
    m2 = B.gs_fem_assemble(ctx, f, dev(s.x))
    a1, a2 = B.gs_mat_export(ctx, m)[2], B.gs_mat_export(ctx, m2)[2]
    assert torch.equal(a1, a2)
    # the library's sorting assembly of the same triplets: same order, same sums
    T, V = len(s.tets), s.n_vertices
    r, c, b = B.gs_fem_triplets(ctx, f, dev(s.x), 10 * T + V)
    m3 = B.gs_assemble(ctx, V, r, c, b)
    assert torch.equal(B.gs_mat_export(ctx, m3)[2], a1)
    # the refilled matrix solves like the fresh one
    y1, y2 = torch.empty(3 * V, dtype=torch.float64, device="cuda"), torch.empty(3 * V, dtype=torch.float64,
                                                                                  device="cuda")
    xv = dev(np.random.default_rng(0).normal(size=3 * V))
    B.gs_spmv(ctx, m, xv, y1)
    B.gs_spmv(ctx, m2, xv, y2)
    assert torch.equal(y1, y2)
    for h in (m, m2, m3):
        B.gs_mat_destroy(h)
    B.gs_fem_destroy(f)


def test_changing_springs_resorts_only_them_and_retires_old_matrices(B, ctx):
    s = make_elastic_scene(7, n_springs=50, seed=16)
    f = make_fem(B, ctx, s)
    m = B.gs_fem_assemble(ctx, f, dev(s.x))
    s2 = make_elastic_scene(7, n_springs=80, seed=17)  # same mesh size, other pairs
    B.gs_fem_set_springs(ctx, f, dev(s2.pairs, torch.int32), dev(s2.K), dev(s2.rest))
    with pytest.raises(B.GsError) as e:
        B.gs_fem_refill(ctx, f, dev(s.x), m)
    assert e.value.status == B.GS_ERR_INVALID
    m2 = B.gs_fem_assemble(ctx, f, dev(s.x))
    ro, co, bo = newton.hessian_triplets(s.X, s.x, s.tets, E, NU, RHO, DT, springs_of(s2))
    rid_o, cid_o, au_o = assembly.assemble(ro, co, bo)
    rid, cid, au = B.gs_mat_export(ctx, m2)
    assert np.array_equal(rid.cpu().numpy(), rid_o) and np.array_equal(cid.cpu().numpy(), cid_o)
    assert np.all(np.abs(au.cpu().numpy().reshape(-1, 3, 3) - au_o) <= 1e-11 * _abs_assembled(ro, co, bo))
    B.gs_fem_set_springs(ctx, f, None, None, None)  # removed: the element pattern alone
    assert B.gs_fem_info(f)[0] == B.gs_fem_info(f)[1]
    B.gs_mat_destroy(m)
    B.gs_mat_destroy(m2)
    B.gs_fem_destroy(f)


def test_mas_refresh_equals_a_fresh_build(B, ctx):
    s = make_elastic_scene(11, n_springs=100, seed=18)
    f = make_fem(B, ctx, s)
    V = s.n_vertices
    args = (dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32), dev(s.pairs, torch.int32))
    m = B.gs_fem_assemble(ctx, f, dev(s.X))
    mas = B.gs_build_mas_mesh(ctx, m, dev(s.X), *args, domain_size=16, max_levels=3)
    B.gs_fem_refill(ctx, f, dev(s.x), m)
    B.gs_mas_refresh(ctx, mas, m)
    mas2 = B.gs_build_mas_mesh(ctx, m, dev(s.X), *args, domain_size=16, max_levels=3)
    r = dev(np.random.default_rng(1).normal(size=(2, 3 * V)))
    z1, z2 = torch.empty_like(r), torch.empty_like(r)
    B.gs_mas_apply(ctx, mas, r, z1, nrhs=2)
    B.gs_mas_apply(ctx, mas2, r, z2, nrhs=2)
    # coarse level matrices sum cross-domain blocks with atomics: equal up to rounding
    assert torch.all((z1 - z2).abs() <= 1e-12 * z2.abs().amax()).item()
    for lvl in range(B.gs_mas_info(mas)[0]):
        assert torch.equal(B.gs_mas_export_coarse(ctx, mas, lvl, V), B.gs_mas_export_coarse(ctx, mas2, lvl, V))
    B.gs_mas_destroy(mas)
    B.gs_mas_destroy(mas2)
    B.gs_mat_destroy(m)
    B.gs_fem_destroy(f)


@pytest.mark.parametrize("n,springs,omega", [(5, 12, 3.0), (6, 30, 10.0)])
def test_newton_follows_the_oracle_iterates(B, ctx, n, springs, omega):
    # a tight linear solve makes the device direction the oracle's to ~1e-10,
    # so both take the same steps and line-search decisions
    s = make_elastic_scene(n, n_springs=springs, omega=omega, seed=19 + n)
    tol = 1e-6
    xo, hist = newton.newton(s.X, s.x, s.tets, E, NU, RHO, DT, s.xt, springs_of(s), tol=tol)
    f = make_fem(B, ctx, s)
    x = dev(s.x)
    st, en, _ = B.gs_fem_newton(ctx, f, dev(s.xt), x, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32), tol=tol,
                                pcg_tol=1e-12, domain_size=16, max_levels=3)
    assert st["converged"] and hist[-1]["converged"]
    assert st["iterations"] == len(hist) - 1
    assert st["halvings"] == sum(h["halvings"] for h in hist)
    e_o = np.array([h["energy"] for h in hist])
    assert np.allclose(en, e_o, rtol=1e-10, atol=0)
    assert np.all(np.diff(en) < 0)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9
    B.gs_fem_destroy(f)


def test_newton_with_the_default_linear_tolerance_reaches_the_same_minimiser(B, ctx):
    s = make_elastic_scene(12, n_springs=200, omega=10.0, seed=31)
    tol = 1e-4
    xo, hist = newton.newton(s.X, s.x, s.tets, E, NU, RHO, DT, s.xt, springs_of(s), tol=tol)
    f = make_fem(B, ctx, s)
    x = dev(s.x)
    st, en, _ = B.gs_fem_newton(ctx, f, dev(s.xt), x, dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32), tol=tol,
                                pcg_tol=1e-6, domain_size=32, max_levels=3)
    assert st["converged"]
    assert abs(st["iterations"] - (len(hist) - 1)) <= 2
    # both stop within one small step of the unique minimiser near the start
    assert np.abs(x.cpu().numpy() - xo).max() <= 4 * tol * DT
    assert st["energy"] <= en[0] and st["energy"] == pytest.approx(hist[-1]["energy"], rel=1e-8)
    B.gs_fem_destroy(f)


def test_invalid_bodies_are_refused(B, ctx):
    s = make_elastic_scene(3, seed=40)
    bad = s.tets.copy()
    bad[3, 1] = bad[3, 0]  # repeated vertex
    with pytest.raises(B.GsError) as e:
        B.gs_fem_create(ctx, dev(s.X), dev(bad, torch.int32), E, NU, RHO, DT)
    assert e.value.status == B.GS_ERR_INVALID
    flat = s.X.copy()
    flat[:, 2] = 0.0  # every tet flat
    with pytest.raises(B.GsError) as e:
        B.gs_fem_create(ctx, dev(flat), dev(s.tets, torch.int32), E, NU, RHO, DT)
    assert e.value.status == B.GS_ERR_NONFINITE
    f = make_fem(B, ctx, s)
    with pytest.raises(B.GsError):
        B.gs_fem_set_springs(ctx, f, dev(np.array([[2, 2]]), torch.int32), dev(np.eye(3)[None]), dev(np.zeros((1, 3))))
    other = B.gs_assemble(ctx, s.n_vertices, dev([0], torch.int32), dev([0], torch.int32), dev(np.eye(3)[None]))
    with pytest.raises(B.GsError):
        B.gs_fem_refill(ctx, f, dev(s.x), other)
    B.gs_mat_destroy(other)
    B.gs_fem_destroy(f)
