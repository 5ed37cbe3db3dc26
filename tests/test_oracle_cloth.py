"""Pins of the cloth element-Hessian oracle (oracle/cloth.py) against what the
mathematics fixes: finite differences where the Hessian is exact, the PSD
projection of the exact Hessian where it is clamped, the dihedral-angle
gradient by central differences, closed-form masses, a brute-force dense
scatter of the triplets, the independent input generator, and the
invariances every element Hessian has (rigid translations in its null space,
blocks that rotate with the sheet, a dihedral gradient with no net force or
torque), also where the clamp or the strain limit is active."""

import numpy as np
import pytest

from oracle import assembly, cloth
from synth.cloth import hinges, make_cloth_system, sheet


def _fd_hessian(f, x, h):
    n = x.size
    H = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            xpp, xpm, xmp, xmm = (x.copy() for _ in range(4))
            xpp[i] += h; xpp[j] += h
            xpm[i] += h; xpm[j] -= h
            xmp[i] -= h; xmp[j] += h
            xmm[i] -= h; xmm[j] -= h
            H[i, j] = (f(xpp) - f(xpm) - f(xmp) + f(xmm)) / (4 * h * h)
    return H


def _element_dense(w, He):
    """9 x 9 element Hessian from the 3 x 3 vertex blocks He[a, b]."""
    return np.block([[He[a, b] for b in range(3)] for a in range(3)])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_membrane_hessian_is_the_exact_hessian_where_no_term_is_clamped(seed):
    # orthogonal columns stretched past 1: the stretch Hessian is unclamped,
    # the shear Gauss-Newton term is exact (f_0 . f_1 = 0) and the strain
    # limit is active, so the pulled-back Hessian equals the energy's own
    rng = np.random.default_rng(seed)
    X = np.zeros((3, 3))
    X[:, :2] = rng.normal(size=(3, 2))
    R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    s = rng.uniform(1.02, 1.2, 2)
    tris = np.array([[0, 1, 2]])
    w, A = cloth.rest_data(X, tris)
    # x with F = R[:, :2] diag(s): x_a = F X_a (in-plane rest coordinates) + a shift
    F = R[:, :2] * s[None, :]
    x = X[:, :2] @ F.T + rng.normal(size=3)
    assert np.allclose(cloth.deformation(x, tris, w)[0], F, atol=1e-12)
    lam, E, t = 0.05e6, 1e8, 1e-3
    He = cloth.pullback(w, cloth.membrane_F_hessian(cloth.deformation(x, tris, w), A * t, lam, E))[0]
    energy = lambda v: cloth.membrane_energy(cloth.deformation(v.reshape(3, 3), tris, w), A * t, lam, E)[0]
    H_fd = _fd_hessian(energy, x.ravel(), 1e-5)
    H = _element_dense(w[0], He)
    assert np.abs(H - H_fd).max() <= 1e-5 * np.abs(H).max()


@pytest.mark.parametrize("s0", [0.7, 0.95, 1.0, 1.3])
def test_stretch_block_is_the_psd_projection_of_the_exact_hessian(s0):
    # one direction's stretch term lam (|f| - 1)^2 (E = 0; the second column a
    # unit vector orthogonal to f, whose shear Gauss-Newton part in this block,
    # 2 (0.3 lam) f_1 f_1^T, is taken off): its F-Hessian block equals the
    # exact Hessian with negative eigenvalues clamped to zero
    rng = np.random.default_rng(7)
    f = rng.normal(size=3)
    f *= s0 / np.linalg.norm(f)
    f1 = np.cross(f, rng.normal(size=3))
    f1 /= np.linalg.norm(f1)
    F = np.zeros((1, 3, 2))
    F[0, :, 0] = f
    F[0, :, 1] = f1
    lam = 2.5
    H = cloth.membrane_F_hessian(F, np.ones(1), lam, 0.0)[0][:3, :3] - 2 * cloth.SHEAR * lam * np.outer(f1, f1)
    e = lambda v: lam * (np.linalg.norm(v) - 1.0) ** 2
    Hx = _fd_hessian(e, f.copy(), 1e-5)
    ev, V = np.linalg.eigh(0.5 * (Hx + Hx.T))
    Hp = (V * np.maximum(ev, 0.0)) @ V.T
    assert np.abs(H - Hp).max() <= 1e-6 * lam


def test_dihedral_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    P = rng.normal(size=(50, 4, 3))
    g = cloth.dihedral_gradient(P)
    h = 1e-6
    for a in range(4):
        for c in range(3):
            Pp, Pm = P.copy(), P.copy()
            Pp[:, a, c] += h
            Pm[:, a, c] -= h
            fd = (cloth.dihedral_angle(Pp) - cloth.dihedral_angle(Pm)) / (2 * h)
            assert np.abs(g[:, a, c] - fd).max() <= 1e-6 * (1 + np.abs(fd).max())
    # translation invariance: the four gradients sum to zero
    assert np.abs(g.sum(axis=1)).max() <= 1e-12 * np.abs(g).max()


def test_bending_gauss_newton_is_the_exact_hessian_at_the_rest_angle():
    rng = np.random.default_rng(4)
    P0 = rng.normal(size=(1, 4, 3))
    theta0 = cloth.dihedral_angle(P0)[0]
    kb = 3.0
    g = cloth.dihedral_gradient(P0)[0].ravel()
    energy = lambda v: kb * (cloth.dihedral_angle(v.reshape(1, 4, 3))[0] - theta0) ** 2
    H_fd = _fd_hessian(energy, P0.ravel(), 1e-5)
    assert np.abs(2 * kb * np.outer(g, g) - H_fd).max() <= 1e-5 * np.abs(H_fd).max()


def test_masses_and_bending_stiffness_closed_forms():
    n = 9
    X, tris = sheet(n)
    h = 1.0 / (n - 1)
    w, A = cloth.rest_data(X, tris)
    assert np.allclose(A, h * h / 2)
    rho, t = 200.0, 1e-3
    m = cloth.lumped_masses(X.shape[0], tris, A, rho, t)
    assert np.isclose(m.sum(), rho * t * 1.0)  # unit square sheet
    interior = (np.arange(n * n) % n > 0) & (np.arange(n * n) % n < n - 1) & (np.arange(n * n) // n > 0) \
        & (np.arange(n * n) // n < n - 1)
    assert np.allclose(m[interior], rho * t * h * h)  # six triangles of area h^2 / 2, a third each
    hg = hinges(tris)
    kb = cloth.bending_stiffness(X, hg, 1e8, t)
    e2 = np.sum((X[hg[:, 1]] - X[hg[:, 0]]) ** 2, axis=1)
    assert np.allclose(kb, 1e8 * t ** 3 / 12 * e2 / (h * h))  # two triangles of area h^2 / 2


def test_triplets_scatter_to_the_dense_element_sum():
    n = 4
    X, tris = sheet(n)
    rng = np.random.default_rng(5)
    x = X @ np.array([[1.05, 0.03, 0], [0, 1.01, 0], [0, 0, 1]]).T + rng.normal(0, 0.01, X.shape)
    hg = hinges(tris)
    E, lam, t, rho, dt = 1e8, 0.05e6, 1e-3, 200.0, 0.01
    r, c, b = cloth.cloth_triplets(X, x, tris, hg, E, lam, t, rho, dt)
    V = X.shape[0]
    assert r.size == 6 * len(tris) + 10 * len(hg) + V and np.all(r <= c)
    D = np.zeros((3 * V, 3 * V))  # dense scatter: upper blocks and their transposes
    for k in range(r.size):
        D[3 * r[k] : 3 * r[k] + 3, 3 * c[k] : 3 * c[k] + 3] += b[k]
        if r[k] != c[k]:
            D[3 * c[k] : 3 * c[k] + 3, 3 * r[k] : 3 * r[k] + 3] += b[k].T
    # brute force: element matrices summed into the dense matrix by vertex index
    w, A = cloth.rest_data(X, tris)
    He = cloth.pullback(w, cloth.membrane_F_hessian(cloth.deformation(x, tris, w), A * t, lam, E))
    D0 = np.zeros_like(D)
    for e, tri in enumerate(tris):
        for a in range(3):
            for bb in range(3):
                D0[3 * tri[a] : 3 * tri[a] + 3, 3 * tri[bb] : 3 * tri[bb] + 3] += He[e, a, bb]
    g = cloth.dihedral_gradient(x[hg])
    kb = cloth.bending_stiffness(X, hg, E, t)
    for e, hh in enumerate(hg):
        for a in range(4):
            for bb in range(4):
                D0[3 * hh[a] : 3 * hh[a] + 3, 3 * hh[bb] : 3 * hh[bb] + 3] += 2 * kb[e] * np.outer(g[e, a], g[e, bb])
    m = cloth.lumped_masses(V, tris, A, rho, t)
    D0 += np.kron(np.diag(m / dt ** 2), np.eye(3))
    assert np.abs(D - D0).max() <= 1e-12 * np.abs(D0).max()
    assert np.abs(D - D.T).max() <= 1e-12 * np.abs(D).max()
    assert np.linalg.eigvalsh(D).min() > 0  # PSD elements plus positive masses


def test_oracle_matches_the_independent_generator():
    # synth.cloth builds the same Hessian in torch (autograd dihedral gradient,
    # its own membrane formulas); both assemble to the same matrix
    n = 12
    s = make_cloth_system(n=n, device="cpu")
    X, tris = sheet(n)
    rng = np.random.default_rng(1003)
    h = 1.0 / (n - 1)
    sh = rng.uniform(0.0, 0.1)
    x = X @ np.array([[1.02, sh, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]).T + rng.normal(0.0, 0.01 * h, X.shape)
    r, c, b = cloth.cloth_triplets(X, x, tris, hinges(tris), 1e8, 0.05e6, 1e-3, 200.0, 0.01)
    R0, C0, B0 = assembly.assemble(r, c, b)
    R1, C1, B1 = assembly.assemble(s.rows, s.cols, s.blocks)
    assert np.array_equal(R0, R1) and np.array_equal(C0, C1)
    assert np.abs(B0 - B1).max() <= 1e-12 * np.abs(B1).max()


@pytest.mark.parametrize("stretch", [0.9, 1.02, 1.3])
def test_element_hessians_are_frame_indifferent_and_translation_free(stretch):
    # the energies depend on x only through edge vectors and their lengths and
    # angles, so (i) every element Hessian annihilates a rigid translation
    # (sum_b H_ab = 0), (ii) rotating the deformed sheet rotates every block
    # (H_ab(R x) = R H_ab(x) R^T), and (iii) the dihedral gradient sums to zero
    # and carries no torque (sum_a g_a = 0, sum_a p_a x g_a = 0); this holds
    # with the stretch clamp (0.9) and the strain limit (1.3) active as well
    n = 6
    X, tris = sheet(n)
    hg = hinges(tris)
    rng = np.random.default_rng(7)
    x = X @ np.array([[stretch, 0.04, 0], [0, 1.0, 0], [0, 0, 1]]).T + rng.normal(0, 0.02 / (n - 1), X.shape)
    E, lam, t = 1e8, 0.05e6, 1e-3
    w, A = cloth.rest_data(X, tris)
    He = lambda v: cloth.pullback(w, cloth.membrane_F_hessian(cloth.deformation(v, tris, w), A * t, lam, E))
    H0 = He(x)
    scale = np.abs(H0).max()
    assert np.abs(H0.sum(axis=2)).max() <= 1e-12 * scale  # (i), every row block a
    R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    HR = He(x @ R.T + rng.normal(size=3))
    assert np.abs(HR - np.einsum("xp,tabpq,yq->tabxy", R, H0, R)).max() <= 1e-11 * scale  # (ii)
    P = x[hg]
    g = cloth.dihedral_gradient(P)
    gs = np.abs(g).max()
    assert np.abs(g.sum(axis=1)).max() <= 1e-12 * gs * np.abs(P).max()  # (iii) force balance
    assert np.abs(np.cross(P, g).sum(axis=1)).max() <= 1e-11 * gs * np.abs(P).max()  # (iii) torque
    gR = cloth.dihedral_gradient(P @ R.T)
    assert np.abs(gR - g @ R.T).max() <= 1e-11 * gs
