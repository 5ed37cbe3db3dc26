"""Newton's method on the implicit-Euler incremental potential, restated for
the oracle (test infrastructure only; the library runs the loop on the device).

The paper's simulation step (Fig. framework; supplement Eq. 1) repeats:
assemble the gradient and the PSD-projected Hessian of the incremental
potential, solve H d = -g with MAS-PCG, and move along d.  The oracle takes
the same steps on a smooth potential without contact barriers or CCD:

  E(x) = sum_tets vol Psi_SNH(F)                       (elastic.py)
       + sum_v m_v / (2 dt^2) |x_v - xt_v|^2           (inertia; xt the predicted positions)
       + sum_springs 1/2 (x_i - x_j - r)^T K (x_i - x_j - r)

with K symmetric positive semi-definite per spring (the stiffness form of
the synthetic contact pairs).  Its Hessian is the elastic K_e (projected) +
M / dt^2 + the spring blocks [K, -K; -K, K].

Loop (the reading of the paper's framework used here):
  1. g = grad E(x); H = projected Hessian at x;
  2. d = -H^-1 g, by a direct sparse solve (the definition of the Newton
     direction; the library reaches it by MAS-PCG);
  3. stop when max_i |d_i| <= tol * dt (the step's velocity is small);
  4. backtracking line search: alpha = 1, halved while
     E(x + alpha d) > E(x) + c alpha g.d (Armijo, c = 1e-4), at most
     max_halvings times;
  5. x <- x + alpha d.
"""

import numpy as np

from . import assembly, elastic


def spring_terms(x, springs):
    """Energy, gradient (V, 3) and (rows, cols, blocks) of the springs.

    springs: (pairs (P, 2) int, K (P, 3, 3), rest (P, 3)) or None."""
    x = np.asarray(x, dtype=np.float64)
    g = np.zeros_like(x)
    if springs is None or len(springs[0]) == 0:
        return 0.0, g, (np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((0, 3, 3)))
    pairs, K, rest = (np.asarray(springs[0], dtype=np.int64), np.asarray(springs[1], dtype=np.float64),
                      np.asarray(springs[2], dtype=np.float64))
    i, j = pairs[:, 0], pairs[:, 1]
    d = x[i] - x[j] - rest
    Kd = np.einsum("pab,pb->pa", K, d)
    energy = 0.5 * float(np.einsum("pa,pa->", d, Kd))
    np.add.at(g, i, Kd)
    np.add.at(g, j, -Kd)
    swap = i > j
    off = np.where(swap[:, None, None], -np.swapaxes(K, 1, 2), -K)
    rows = np.concatenate([i, j, np.minimum(i, j)])
    cols = np.concatenate([i, j, np.maximum(i, j)])
    return energy, g, (rows, cols, np.concatenate([K, K, off]))


def incremental_potential(X, x, tets, E, nu, rho, dt, xt, springs=None):
    """E(x) and grad E(x) (V, 3)."""
    e_el, g_el = elastic.energy_and_gradient(X, x, tets, E, nu)
    m = elastic.lumped_mass(X, tets, rho)
    dx = np.asarray(x, dtype=np.float64) - np.asarray(xt, dtype=np.float64)
    e_in = float((m * (dx * dx).sum(axis=1)).sum()) / (2.0 * dt * dt)
    g_in = (m / (dt * dt))[:, None] * dx
    e_sp, g_sp, _ = spring_terms(x, springs)
    return e_el + e_in + e_sp, g_el + g_in + g_sp


def hessian_triplets(X, x, tets, E, nu, rho, dt, springs=None):
    """Upper triplets of the projected Hessian: the elastic and mass triplets
    in elastic.system_triplets' order, then three blocks per spring."""
    r, c, b = elastic.system_triplets(X, x, tets, E, nu, rho, dt)
    _, _, (rs, cs, bs) = spring_terms(x, springs)
    return np.concatenate([r, rs]), np.concatenate([c, cs]), np.concatenate([b, bs])


def newton_direction(V, rows, cols, blocks, g):
    """d = -H^-1 g by a sparse direct solve of the assembled symmetric H."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    rid, cid, au = assembly.assemble(rows, cols, blocks)
    a = np.arange(3)
    ii = (3 * rid[:, None, None] + a[None, :, None]) + 0 * a[None, None, :]
    jj = (3 * cid[:, None, None] + a[None, None, :]) + 0 * a[None, :, None]
    off = rid != cid  # the stored block's transpose sits at (c, r)
    ii, jj, vv = (np.concatenate([ii.ravel(), jj[off].ravel()]), np.concatenate([jj.ravel(), ii[off].ravel()]),
                  np.concatenate([au.ravel(), au[off].ravel()]))
    H = sp.csc_matrix((vv, (ii, jj)), shape=(3 * V, 3 * V))
    return -spla.spsolve(H, np.asarray(g, dtype=np.float64).reshape(-1)).reshape(V, 3)


def newton(X, x0, tets, E, nu, rho, dt, xt, springs=None, tol=1e-3, max_newton=50, armijo=1e-4,
           max_halvings=30):
    """The loop in the module docstring.  Returns (x, history) with history a
    list of dicts per step: energy before the step, max |d|, alpha, halvings."""
    x = np.array(x0, dtype=np.float64)
    V = x.shape[0]
    hist = []
    for _ in range(max_newton):
        e, g = incremental_potential(X, x, tets, E, nu, rho, dt, xt, springs)
        rows, cols, blocks = hessian_triplets(X, x, tets, E, nu, rho, dt, springs)
        d = newton_direction(V, rows, cols, blocks, g)
        dinf = float(np.abs(d).max()) if d.size else 0.0
        if dinf <= tol * dt:
            hist.append(dict(energy=e, dinf=dinf, alpha=0.0, halvings=0, converged=True))
            return x, hist
        gd = float((g * d).sum())
        alpha, halvings = 1.0, 0
        while True:
            e_try, _ = incremental_potential(X, x + alpha * d, tets, E, nu, rho, dt, xt, springs)
            if e_try <= e + armijo * alpha * gd or halvings >= max_halvings:
                break
            alpha *= 0.5
            halvings += 1
        hist.append(dict(energy=e, dinf=dinf, alpha=alpha, halvings=halvings, converged=False))
        x = x + alpha * d
    return x, hist
