"""Element Hessians of the stiff-cloth system, restated for the oracle (test
infrastructure; the library computes them on the device from positions).

A triangle sheet with rest positions X (z = 0) and deformed positions x.
Per triangle (vertices 0, 1, 2) the rest edge matrix Dm (2 x 2, columns
X_1 - X_0 and X_2 - X_0 in the plane), its area A = |det Dm| / 2 and
B = Dm^-1 give F = sum_a x_a w_a^T (3 x 2) with w_a = row a - 1 of B for
a >= 1 and w_0 = -(w_1 + w_2), evaluated from the edges (x_1 - x_0) and
(x_2 - x_0); f_0, f_1 are the columns of F and vec(F) = [f_0; f_1].  With a_t = A * thickness the membrane energy is

  stretching     lam a_t sum_d (|f_d| - 1)^2,
  strain limit   E a_t sum_d max(|f_d| - 1, 0)^3            (Sec. 4, Eq. memb_u),
  shearing       0.3 lam a_t (f_0 . f_1)^2,

and its 6 x 6 F-Hessian, per direction d with s = |f_d| and P = f_d f_d^T / s^2:
  stretching     2 lam (P + max(1 - 1/s, 0) (I - P))    (the exact Hessian with
                 the negative eigenvalue 2 lam (1 - 1/s), s < 1, clamped to 0),
  strain limit   the analytic PSD Hessian of Sec. 4 (Eq. Stretch_Hessian,
                 ``strain_limit.hessian``): 3 E ((1 - 1/s)(s - 1) I
                 + (s^2 - 1) / s^3 f_d f_d^T) for s > 1, else 0,
  shearing       Gauss-Newton 2 (0.3 lam) g g^T, g = [f_1; f_0],
all times a_t.  The element Hessian is dvec(F)/dx^T H_F dvec(F)/dx, block
(a, b) = sum_{i,j} w_a[i] w_b[j] H_F[i, j] (H_F[i, j] the 3 x 3 block of
directions i, j).

Bending, per interior edge (hinge) with shared vertices e_0, e_1 and the
opposite vertices o_1, o_2 of its two triangles: the dihedral angle theta =
atan2(((n_1 x n_2) . e/|e|), n_1 . n_2) with e = e_1 - e_0, n_1 = e x (o_1 -
e_0), n_2 = (o_2 - e_0) x e, stiffness k_b = E t^3 / 12 * |e_rest|^2 /
(A_1 + A_2) (rest edge length and rest triangle areas), and the Gauss-Newton
Hessian 2 k_b grad(theta) grad(theta)^T.  With q_i = n_i / |n_i|^2:
  dtheta/do_1 = -|e| q_1,  dtheta/do_2 = -|e| q_2,
  dtheta/de_0 = -((o_1 - e_1) . e / |e|) q_1 - ((o_2 - e_1) . e / |e|) q_2,
  dtheta/de_1 =  ((o_1 - e_0) . e / |e|) q_1 + ((o_2 - e_0) . e / |e|) q_2.

Masses: rho t A / 3 per triangle corner, on the diagonal as m / dt^2 I3.

The triplets come in the library's emission order: per triangle the 6 vertex
pairs (0,0) (0,1) (0,2) (1,1) (1,2) (2,2), per hinge the 10 pairs of
(e_0, e_1, o_1, o_2) with a <= b in that order, each at (min, max) of its
two vertices (transposed when the first is the larger), then one mass block
per vertex.  Every quantity is float64.
"""

import numpy as np

from . import strain_limit

SHEAR = 0.3  # shear stiffness relative to lam


def rest_data(X, tris):
    """w (T, 3, 2) and rest areas A (T,) of the triangles (in-plane rest coordinates)."""
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(tris)
    Dm = np.stack([X[t[:, 1], :2] - X[t[:, 0], :2], X[t[:, 2], :2] - X[t[:, 0], :2]], axis=2)  # columns
    A = 0.5 * np.abs(np.linalg.det(Dm))
    B = np.linalg.inv(Dm)
    w = np.zeros((t.shape[0], 3, 2))
    w[:, 1, :] = B[:, 0, :]
    w[:, 2, :] = B[:, 1, :]
    w[:, 0, :] = -(w[:, 1, :] + w[:, 2, :])
    return w, A


def deformation(x, tris, w):
    """F (T, 3, 2) = sum_a x_a w_a^T, evaluated from the edge vectors as
    (x_1 - x_0) w_1^T + (x_2 - x_0) w_2^T (the same value, as w_0 = -(w_1 + w_2),
    without the cancellation of absolute coordinates against 1/h weights)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(tris)
    e1 = x[t[:, 1]] - x[t[:, 0]]
    e2 = x[t[:, 2]] - x[t[:, 0]]
    return e1[:, :, None] * w[:, 1, None, :] + e2[:, :, None] * w[:, 2, None, :]


def membrane_energy(F, a_t, lam, E):
    """Per-triangle membrane energy (stretching + strain limit + shearing)."""
    s = np.linalg.norm(F, axis=1)  # (T, 2): |f_0|, |f_1|
    stretch = lam * np.sum((s - 1.0) ** 2, axis=1)
    sl = E * np.sum(np.maximum(s - 1.0, 0.0) ** 3, axis=1)
    shear = SHEAR * lam * np.sum(F[:, :, 0] * F[:, :, 1], axis=1) ** 2
    return a_t * (stretch + sl + shear)


def membrane_F_hessian(F, a_t, lam, E):
    """(T, 6, 6) PSD F-Hessians of the membrane energy (rows/columns [f_0; f_1])."""
    T = F.shape[0]
    H = np.zeros((T, 6, 6))
    I3 = np.eye(3)
    for d in range(2):
        f = F[:, :, d]
        s = np.linalg.norm(f, axis=1)
        P = f[:, :, None] * f[:, None, :] / (s * s)[:, None, None]
        across = np.maximum(1.0 - 1.0 / s, 0.0)
        H[:, 3 * d : 3 * d + 3, 3 * d : 3 * d + 3] += 2.0 * lam * (P + across[:, None, None] * (I3 - P))
        n = np.eye(2)[d]
        for t in range(T):  # the strain-limiting part through the pinned single-element form
            if s[t] > 1.0:
                H[t] += strain_limit.hessian(F[t], n, E)
    g = np.concatenate([F[:, :, 1], F[:, :, 0]], axis=1)
    H += 2.0 * SHEAR * lam * g[:, :, None] * g[:, None, :]
    return H * a_t[:, None, None]


def pullback(w, HF):
    """Element blocks He[t, a, b] (3 x 3) = sum_{i,j} w_a[i] w_b[j] HF[t, i, j]."""
    HFb = HF.reshape(-1, 2, 3, 2, 3)  # [t, i, x, j, y]
    return np.einsum("tai,tbj,tixjy->tabxy", w, w, HFb)


def dihedral_angle(P):
    """theta per hinge for P (H, 4, 3) = (e_0, e_1, o_1, o_2)."""
    e0, e1, o1, o2 = P[:, 0], P[:, 1], P[:, 2], P[:, 3]
    e = e1 - e0
    n1 = np.cross(e, o1 - e0)
    n2 = np.cross(o2 - e0, e)
    en = e / np.linalg.norm(e, axis=1, keepdims=True)
    return np.arctan2(np.sum(np.cross(n1, n2) * en, axis=1), np.sum(n1 * n2, axis=1))


def dihedral_gradient(P):
    """dtheta/dP (H, 4, 3), the closed form in the module docstring."""
    e0, e1, o1, o2 = P[:, 0], P[:, 1], P[:, 2], P[:, 3]
    e = e1 - e0
    le = np.linalg.norm(e, axis=1)
    n1 = np.cross(e, o1 - e0)
    n2 = np.cross(o2 - e0, e)
    q1 = n1 / np.sum(n1 * n1, axis=1)[:, None]
    q2 = n2 / np.sum(n2 * n2, axis=1)[:, None]
    dot = lambda a, b: np.sum(a * b, axis=1)[:, None]
    g_e0 = -dot(o1 - e1, e) / le[:, None] * q1 - dot(o2 - e1, e) / le[:, None] * q2
    g_e1 = dot(o1 - e0, e) / le[:, None] * q1 + dot(o2 - e0, e) / le[:, None] * q2
    return np.stack([g_e0, g_e1, -le[:, None] * q1, -le[:, None] * q2], axis=1)


def bending_stiffness(X, hinges, E, thickness):
    """k_b = E t^3 / 12 |e_rest|^2 / (A_1 + A_2) per hinge."""
    X = np.asarray(X, dtype=np.float64)
    h = np.asarray(hinges)
    e = X[h[:, 1]] - X[h[:, 0]]
    a1 = 0.5 * np.linalg.norm(np.cross(e, X[h[:, 2]] - X[h[:, 0]]), axis=1)
    a2 = 0.5 * np.linalg.norm(np.cross(e, X[h[:, 3]] - X[h[:, 0]]), axis=1)
    return E * thickness ** 3 / 12.0 * np.sum(e * e, axis=1) / (a1 + a2)


def lumped_masses(V, tris, A, rho, thickness):
    m = np.zeros(V)
    np.add.at(m, np.asarray(tris).ravel(), np.repeat(rho * thickness * A / 3.0, 3))
    return m


def _emit(idx, blocks, pairs):
    """(rows, cols, blocks) of element blocks[e, a, b] for the listed (a, b) pairs, element-major."""
    rows, cols, out = [], [], []
    for a, b in pairs:
        ra, cb = idx[:, a], idx[:, b]
        swap = ra > cb
        rows.append(np.where(swap, cb, ra))
        cols.append(np.where(swap, ra, cb))
        blk = blocks[:, a, b]
        out.append(np.where(swap[:, None, None], np.swapaxes(blk, 1, 2), blk))
    rows = np.stack(rows, 1).reshape(-1)
    cols = np.stack(cols, 1).reshape(-1)
    out = np.stack(out, 1).reshape(-1, 3, 3)
    return rows, cols, out


def cloth_triplets(X, x, tris, hinges, E, lam, thickness, rho, dt):
    """The whole Hessian as triplets in the library's emission order (module docstring)."""
    tris = np.asarray(tris)
    hinges = np.asarray(hinges)
    w, A = rest_data(X, tris)
    F = deformation(x, tris, w)
    He = pullback(w, membrane_F_hessian(F, A * thickness, lam, E))
    r1, c1, b1 = _emit(tris, He, [(a, b) for a in range(3) for b in range(a, 3)])
    x = np.asarray(x, dtype=np.float64)
    g = dihedral_gradient(x[hinges])
    kb = bending_stiffness(X, hinges, E, thickness)
    Hb = 2.0 * kb[:, None, None, None, None] * g[:, :, None, :, None] * g[:, None, :, None, :]  # [h, a, b, x, y]
    r2, c2, b2 = _emit(hinges, Hb, [(a, b) for a in range(4) for b in range(a, 4)])
    V = np.asarray(X).shape[0]
    m = lumped_masses(V, tris, A, rho, thickness)
    r3 = np.arange(V)
    b3 = (m / dt ** 2)[:, None, None] * np.eye(3)
    return (np.concatenate([r1, r2, r3]).astype(np.int32), np.concatenate([c1, c2, r3]).astype(np.int32),
            np.concatenate([b1, b2, b3]))
