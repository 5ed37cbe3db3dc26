"""Test helper: per-entry error bounds for FP64 results that pass through the
MAS preconditioner (supplement Eq. 4-6), built from the oracle's levels.

z = sum_l C_l^T M_l^{-1} C_l r.  Two implementations of it differ by
  (i)  the rounding of their sums, at most about m * eps * (|M^{-1}| |r|) per
       entry, with m <= 3N terms per domain row plus the levels' additions;
  (ii) the difference of their domain inverses.  A backward-stable Cholesky
       inverse of domain d has ||dM_d^{-1}||_2 <= c * 3N * eps * kappa_d *
       ||M_d^{-1}||_2, so every entry of dM_d^{-1} r_d is bounded by
       c * 3N * eps * kappa_d * ||M_d^{-1}||_2 * ||r_d||_2, the same for all
       entries of that domain (||A v||_inf <= ||A||_2 ||v||_2).
apply_bound() returns (i) + (ii) per entry, prolongated to the nodes the way z
is.  A wrong coarse item or domain changes its entries by O(|z|), far above
both terms, so the bound is checked entry by entry."""

import numpy as np

from oracle import mas

C_DOMAIN = 1e-12  # c * 3N * eps with c ~ 100 and 3N <= 96
C_SUM = 1e-13


def domain_scales(om):
    """Per level: kappa_d * ||M_d^{-1}||_2 for every domain (0 for empty ones)."""
    lv = om.levels
    N = lv.N
    out = []
    for l in range(lv.n_levels):
        nd = lv.n_domains(l)
        real = np.zeros(nd * N, dtype=bool)
        real[: lv.n_items[l]] = lv.real[l]
        sc = np.zeros(nd)
        for d in range(nd):
            lanes = np.nonzero(real[d * N : d * N + N])[0]
            if lanes.size == 0:
                continue
            idx = (3 * lanes[:, None] + np.arange(3)).ravel()
            ev = np.linalg.eigvalsh(om.invs[l][d][np.ix_(idx, idx)])
            sc[d] = (ev[-1] / ev[0]) * ev[-1]
        out.append(sc)
    return out


def apply_bound(om, r, scales=None):
    """Per-entry bound on |z_1 - z_2| for two FP64 applies of r (shape (K, 3V))."""
    lv = om.levels
    N = lv.N
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    K = r.shape[0]
    V = lv.coarse[0].size
    if scales is None:
        scales = domain_scales(om)
    absz = mas.apply(lv, [np.abs(v) for v in om.invs], np.abs(r), om.C)
    R = r.reshape(K, V, 3).transpose(1, 0, 2).reshape(V, 3 * K)  # node-major
    dom_term = np.zeros((K, V))
    for l in range(lv.n_levels):
        nd = lv.n_domains(l)
        rl = (om.C[l] @ R).reshape(nd, N, K, 3)
        rn = np.sqrt((rl ** 2).sum(axis=(1, 3)))  # (nd, K): ||r_{l,d}||_2 per RHS
        per_dom = scales[l][:, None] * rn  # (nd, K)
        dom_of_node = lv.coarse[l] // N
        dom_term += per_dom[dom_of_node].T
    bound = C_SUM * absz.reshape(K, V, 3) + C_DOMAIN * dom_term[:, :, None]
    return bound.reshape(K, 3 * V)
