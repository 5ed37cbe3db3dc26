"""Element Hessians of the implicit-Euler elastic energy, restated for the oracle
(test infrastructure; the library computes them on the device from positions).

The paper assembles the Hessian of the incremental potential from local
element Hessians (Sec. 3.1: elastic energies plus barriers; Fig. framework),
each projected to positive semi-definite (PSD) so that the system stays SPD.
The elastic energy is the stable Neo-Hookean form the paper cites (Sec. 3.1),
here the variant without the log term (Smith, de Goes and Kim 2018):

  Psi(F) = mu/2 (I_C - 3) + lam/2 (J - alpha)^2,  alpha = 1 + mu / lam,

with the Lame parameters re-parameterised from Young's modulus E and
Poisson's ratio nu as mu = 4/3 mu_L, lam = lam_L + 5/6 mu_L.  With vec(F) the
stacked columns f0, f1, f2 and g0 = f1 x f2, g1 = f2 x f0, g2 = f0 x f1
(so J = f0 . g0 and dJ/dvec(F) = [g0; g1; g2]):

  dPsi/dvec(F)    = mu vec(F) + lam (J - alpha) dJ/dvec(F)
  d2Psi/dvec(F)^2 = mu I9 + lam dJ dJ^T + lam (J - alpha) H_J,

H_J the 9 x 9 matrix of cross-product blocks d2J/df_i df_j.  The F-Hessian
is projected to PSD by clamping its negative eigenvalues to 0 (a symmetric
eigendecomposition), then pulled back.  For a tet (x_0, x_1, x_2, x_3) with
rest edge matrix Dm (columns X_a - X_0, a = 1..3) and B = Dm^-1,
F = sum_a x_a w_a^T with w_a = row a - 1 of B for a >= 1 and w_0 = -(w_1 +
w_2 + w_3); so dvec(F)/dx_a = [w_a0 I3; w_a1 I3; w_a2 I3] and the 12 x 12
element Hessian is vol * dF/dx^T H_F+ dF/dx, vol = |det Dm| / 6.  Implicit Euler scales the
system as K + M / dt^2 with lumped masses m_v = rho * (sum of adjacent tet
volumes) / 4.

Every quantity is float64.
"""

import numpy as np


def lame(E, nu):
    mu_l = E / (2.0 * (1.0 + nu))
    lam_l = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return 4.0 / 3.0 * mu_l, lam_l + 5.0 / 6.0 * mu_l


def cross_matrix(v):
    """[v]_x with [v]_x u = v x u, for (..., 3) v."""
    z = np.zeros(v.shape[:-1])
    return np.stack([np.stack([z, -v[..., 2], v[..., 1]], -1),
                     np.stack([v[..., 2], z, -v[..., 0]], -1),
                     np.stack([-v[..., 1], v[..., 0], z], -1)], -2)


def snh(F, mu, lam):
    """(Psi, dPsi/dvec(F) (..., 9), d2Psi/dvec(F)^2 (..., 9, 9)) of F (..., 3, 3)."""
    F = np.asarray(F, dtype=np.float64)
    alpha = 1.0 + mu / lam
    f = [F[..., :, j] for j in range(3)]
    g = [np.cross(f[1], f[2]), np.cross(f[2], f[0]), np.cross(f[0], f[1])]
    J = np.einsum("...i,...i->...", f[0], g[0])
    Ic = np.einsum("...ij,...ij->...", F, F)
    psi = 0.5 * mu * (Ic - 3.0) + 0.5 * lam * (J - alpha) ** 2
    vecF = np.concatenate(f, -1)
    dJ = np.concatenate(g, -1)
    grad = mu * vecF + lam * (J - alpha)[..., None] * dJ
    HJ = np.zeros(F.shape[:-2] + (9, 9))
    # d2J/(df_i df_j): J = f0 . (f1 x f2) is trilinear in the columns
    HJ[..., 0:3, 3:6] = -cross_matrix(f[2])
    HJ[..., 0:3, 6:9] = cross_matrix(f[1])
    HJ[..., 3:6, 0:3] = cross_matrix(f[2])
    HJ[..., 3:6, 6:9] = -cross_matrix(f[0])
    HJ[..., 6:9, 0:3] = -cross_matrix(f[1])
    HJ[..., 6:9, 3:6] = cross_matrix(f[0])
    H = mu * np.eye(9) + lam * dJ[..., :, None] * dJ[..., None, :] + lam * (J - alpha)[..., None, None] * HJ
    return psi, grad, H


def psd_project(H):
    """Symmetric H with its negative eigenvalues set to 0."""
    w, Q = np.linalg.eigh(0.5 * (H + np.swapaxes(H, -1, -2)))
    return np.einsum("...ik,...k,...jk->...ij", Q, np.maximum(w, 0.0), Q)


def rest_shape(X, tets):
    """Rest volume (T,) and the weights w (T, 4, 3) with F = sum_a x_a w_a^T."""
    X = np.asarray(X, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    Dm = np.stack([X[tets[:, a]] - X[tets[:, 0]] for a in (1, 2, 3)], -1)  # edge vectors as columns
    Bm = np.linalg.inv(Dm)
    vol = np.abs(np.linalg.det(Dm)) / 6.0
    w = np.empty((tets.shape[0], 4, 3))
    w[:, 1:, :] = Bm
    w[:, 0, :] = -Bm.sum(axis=1)
    return vol, w


def deformation(x, tets, w):
    x = np.asarray(x, dtype=np.float64)
    return np.einsum("tax,taj->txj", x[np.asarray(tets, dtype=np.int64)], w)


def element_hessians(X, x, tets, E, nu, project=True):
    """12 x 12 element Hessians (T, 12, 12): vol * dF/dx^T H_F(+) dF/dx, node-major
    rows (node a's three coordinates at 3a .. 3a + 2)."""
    mu, lam = lame(E, nu)
    vol, w = rest_shape(X, tets)
    F = deformation(x, tets, w)
    _, _, H = snh(F, mu, lam)
    if project:
        H = psd_project(H)
    T = w.shape[0]
    D = np.zeros((T, 9, 12))  # dvec(F)/dx: row 3j + i, column 3a + i = w[a, j]
    for a in range(4):
        for j in range(3):
            for i in range(3):
                D[:, 3 * j + i, 3 * a + i] = w[:, a, j]
    return vol[:, None, None] * np.einsum("tki,tkl,tlj->tij", D, H, D)


def energy_and_gradient(X, x, tets, E, nu):
    """Total elastic energy and its gradient (V, 3) at positions x."""
    mu, lam = lame(E, nu)
    vol, w = rest_shape(X, tets)
    F = deformation(x, tets, w)
    psi, gF, _ = snh(F, mu, lam)
    tets = np.asarray(tets, dtype=np.int64)
    g = np.zeros_like(np.asarray(x, dtype=np.float64))
    for a in range(4):
        # dPsi/dx_a = sum_j w[a, j] dPsi/df_j
        ga = sum(w[:, a, j, None] * gF[:, 3 * j: 3 * j + 3] for j in range(3))
        np.add.at(g, tets[:, a], vol[:, None] * ga)
    return float((vol * psi).sum()), g


def lumped_mass(X, tets, rho):
    vol, _ = rest_shape(X, tets)
    m = np.zeros(np.asarray(X).shape[0])
    for a in range(4):
        np.add.at(m, np.asarray(tets, dtype=np.int64)[:, a], rho * vol / 4.0)
    return m


def system_triplets(X, x, tets, E, nu, rho, dt):
    """Upper-triangle (r <= c) triplets of K + M / dt^2: ten blocks per tet in
    the pair order (0,0),(0,1),(0,2),(0,3),(1,1),(1,2),(1,3),(2,2),(2,3),(3,3),
    each stored for (min, max) of its two nodes (the block transposed when
    the first node is the larger), then one mass block per vertex."""
    He = element_hessians(X, x, tets, E, nu)
    tets = np.asarray(tets, dtype=np.int64)
    rows, cols, blocks = [], [], []
    for a in range(4):
        for b in range(a, 4):
            ra, cb = tets[:, a], tets[:, b]
            blk = He[:, 3 * a: 3 * a + 3, 3 * b: 3 * b + 3]
            swap = ra > cb
            rows.append(np.where(swap, cb, ra))
            cols.append(np.where(swap, ra, cb))
            blocks.append(np.where(swap[:, None, None], np.swapaxes(blk, 1, 2), blk))
    pair_rows = np.stack(rows, 1).reshape(-1)
    pair_cols = np.stack(cols, 1).reshape(-1)
    pair_blocks = np.stack(blocks, 1).reshape(-1, 3, 3)
    m = lumped_mass(X, tets, rho)
    V = m.size
    vi = np.arange(V)
    return (np.concatenate([pair_rows, vi]), np.concatenate([pair_cols, vi]),
            np.concatenate([pair_blocks, (m / dt ** 2)[:, None, None] * np.eye(3)]))
