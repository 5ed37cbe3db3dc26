"""The seeded input generators produce what their recipes state: symmetric PSD
element Hessians, the paper's strain-limiting Hessian (checked against the
oracle's restatement), and batches whose blocks never join two systems."""

import numpy as np

from oracle import assembly
from oracle import strain_limit as sl
from synth.cloth import make_cloth_system, strain_limit_F_hessian
from synth.hessians import _psd_project, snh_energy_grad_hess_F
from synth.workloads import make_tet_system, uneven_batch


def test_snh_gradient_by_differences_and_projection_psd():
    rng = np.random.default_rng(0)
    F = np.eye(3) + 0.2 * rng.normal(size=(3, 3))
    psi, g, H = snh_energy_grad_hess_F(F[None], 1e5, 0.4)
    f = F.T.reshape(9)
    E = lambda v: snh_energy_grad_hess_F(v.reshape(3, 3).T[None], 1e5, 0.4)[0][0]
    h = 1e-6
    g_fd = np.array([(E(f + h * e) - E(f - h * e)) / (2 * h) for e in np.eye(9)])
    np.testing.assert_allclose(g[0], g_fd, rtol=1e-6, atol=1e-3)
    P = _psd_project(H)
    assert np.linalg.eigvalsh(P[0]).min() > -1e-9 * np.abs(P).max()


def test_tet_system_matrix_is_symmetric_positive_definite():
    s = make_tet_system(4, E=1e7, n_contacts=4, seed=3)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    A = assembly.to_dense(s.n_vertices, rid, cid, au)
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0


def test_cloth_strain_limit_term_equals_oracle():
    rng = np.random.default_rng(1)
    F = rng.normal(size=(64, 3, 2)) * 0.2 + np.array([[1.05, 0.1], [0.0, 1.02], [0.0, 0.0]])
    got = strain_limit_F_hessian(F, E=3.0)
    ref = np.stack([sl.hessian(f, sl.N_U, 3.0) + sl.hessian(f, sl.N_V, 3.0) for f in F])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_cloth_system_is_spd():
    c = make_cloth_system(8, device="cpu")
    rid, cid, au = assembly.assemble(c.rows, c.cols, c.blocks)
    A = assembly.to_dense(c.n_vertices, rid, cid, au)
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0


def test_batch_blocks_stay_inside_their_system():
    b = uneven_batch(n_sys=5, v_range=(100, 600), seed=9)
    sys_of = np.searchsorted(b.node_off, np.arange(b.n_vertices), side="right") - 1
    assert np.all(sys_of[b.rows] == sys_of[b.cols])
    src = np.repeat(np.arange(b.n_vertices), np.diff(b.adj_ptr))
    assert np.all(sys_of[src] == sys_of[b.adj])
    assert np.all(sys_of[b.contacts[:, 0]] == sys_of[b.contacts[:, 1]])


def test_unique_sorted_is_numpys_unique():
    from synth.mesh import unique_sorted

    rng = np.random.default_rng(8)
    for n, hi in ((0, 5), (1, 5), (1000, 10), (100_000, 1 << 40)):
        a = rng.integers(0, hi, n)
        assert np.array_equal(unique_sorted(a), np.unique(a))


def test_coupled_scene_without_fem_blocks_keeps_every_other_input():
    from synth.abd import make_abd_scene

    a = make_abd_scene(n=8, n_bodies=9, n_contacts=400, seed=31)
    b = make_abd_scene(n=8, n_bodies=9, n_contacts=400, seed=31, fem_blocks=False)
    for f in ("X", "adj_ptr", "adj", "contacts", "body_of_node", "xbar"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    # the inputs that remain are the full scene's minus the FEM element and mass blocks
    fem = (a.rows < a.n_fem) & (a.cols < a.n_fem)
    key = lambda r, c, blk: sorted(zip(r.tolist(), c.tolist(), np.round(blk.reshape(len(r), -1), 6).tolist()))
    contacts_fem = (b.rows < b.n_fem) & (b.cols < b.n_fem)  # FEM-FEM contact pairs only
    assert key(a.rows[~fem], a.cols[~fem], a.blocks[~fem]) == key(b.rows[~contacts_fem], b.cols[~contacts_fem],
                                                                  b.blocks[~contacts_fem])
    assert b.fem_x.shape == (a.n_fem, 3) and b.fem_tets.shape[1] == 4
