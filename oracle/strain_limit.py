"""Cubic inexact strain-limiting energy and its analytic eigensystem (Sec. 4).

For a triangle with deformation gradient F = [f0 | f1] (3 x 2) and a material
direction n (n_u = [1, 0], n_v = [0, 1]), I5 = n^T F^T F n and s = sqrt(I5):

  Psi_SL^n = lambda' a_t max(s - 1, 0)^3                       (Eq. memb_u)

summed over n_u and n_v.  With respect to vec(F) (the 6-vector [f0; f1]) the
direction-n part has, for s > 1, the eigenvalues (dropping lambda' a_t)
  e_1 = 6 (s - 1)  along f_n = F n,  e_{2,3} = 3 (1/s + s - 2)  across it
(Eq. e1, e23_0), and the PSD Hessian
  H = 3 (1 - 1/s)(s - 1) H_n + 3 (I5 - 1) / I5^{3/2} f f^T      (Eq. Stretch_Hessian)
with H_n = L_n (x) I3, L_n = n n^T, f = vec(F L_n).  The paper's 1_{3x3} in
H_n is read as the 3 x 3 identity.  For s <= 1 the energy and its
derivatives vanish.

Test infrastructure only (see the package docstring).
"""

import numpy as np

N_U = np.array([1.0, 0.0])
N_V = np.array([0.0, 1.0])


def _parts(F, n):
    F = np.asarray(F, dtype=np.float64).reshape(3, 2)
    fn = F @ n
    I5 = float(fn @ fn)
    return F, fn, I5, np.sqrt(I5)


def energy(F, n, stiffness=1.0):
    _, _, _, s = _parts(F, n)
    return stiffness * max(s - 1.0, 0.0) ** 3


def gradient(F, n, stiffness=1.0):
    """dPsi/dvec(F), vec stacking the columns of F."""
    F, fn, I5, s = _parts(F, n)
    g = np.zeros(6)
    if s > 1.0:
        # dPsi/dfn = 3 (s-1)^2 fn / s, and fn = F n
        dfn = 3.0 * (s - 1.0) ** 2 / s * fn
        g = np.concatenate([dfn * n[0], dfn * n[1]])
    return stiffness * g


def hessian(F, n, stiffness=1.0):
    """The analytic PSD Hessian of Eq. Stretch_Hessian, 6 x 6."""
    F, fn, I5, s = _parts(F, n)
    if s <= 1.0:
        return np.zeros((6, 6))
    L = np.outer(n, n)
    Hn = np.kron(L, np.eye(3))
    f = (F @ L).T.reshape(6)  # vec(F L): columns stacked
    return stiffness * (3.0 * (1.0 - 1.0 / s) * (s - 1.0) * Hn + 3.0 * (I5 - 1.0) / I5 ** 1.5 * np.outer(f, f))


def eigenvalues(F, n):
    """(e_1, e_2, e_3) of Eq. e1 / e23_0 for the direction-n part (s > 1)."""
    _, _, _, s = _parts(F, n)
    return 6.0 * (s - 1.0), 3.0 * (1.0 / s + s - 2.0), 3.0 * (1.0 / s + s - 2.0)
