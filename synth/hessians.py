"""Local Hessian blocks emitted as (row, col, 3x3) triplets.

Only blocks with row <= col are emitted: the matrix is symmetric and its
lower triangle is implied by the upper one.  Every block is row-major.

* Stable Neo-Hookean volume energy (Smith, de Goes, Kim 2018, the form
  without the log term): Psi = mu/2 (I_C - 3) + lam/2 (J - alpha)^2 with
  alpha = 1 + mu/lam and the Lame parameters re-parameterised as
  mu = 4/3 mu_L, lam = lam_L + 5/6 mu_L.  Its 9x9 Hessian with respect to
  vec(F) (column-major) is projected to PSD by clamping negative
  eigenvalues, then pulled back to the 12x12 element Hessian
  vol * dF/dx^T H_F dF/dx.  The system is scaled as K + M / dt^2 (the
  paper's M + dt^2 K of Eq. E_s divided by dt^2), so contact blocks keep
  their own stiffness.
* Lumped mass m_v / dt^2 * I3 on the diagonal blocks.
* Contact stand-ins: a PSD block K = k n n^T on a vertex pair (i, j),
  added as [[K, -K], [-K, K]].
"""

import numpy as np
import torch


def _hat(v):
    """Cross-product matrices of (..., 3) vectors -> (..., 3, 3)."""
    z = np.zeros(v.shape[:-1])
    return np.stack(
        [
            np.stack([z, -v[..., 2], v[..., 1]], -1),
            np.stack([v[..., 2], z, -v[..., 0]], -1),
            np.stack([-v[..., 1], v[..., 0], z], -1),
        ],
        -2,
    )


def _lame(E, nu):
    mu_l = E / (2.0 * (1.0 + nu))
    lam_l = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return 4.0 / 3.0 * mu_l, lam_l + 5.0 / 6.0 * mu_l


def snh_energy_grad_hess_F(F, E, nu):
    """Energy density, dPsi/dvec(F) (.., 9) and d2Psi/dvec(F)^2 (.., 9, 9).

    vec(F) stacks the columns f0, f1, f2 of F.  Works on numpy arrays or
    torch tensors (float64).
    """
    xp = torch if isinstance(F, torch.Tensor) else np
    mu, lam = _lame(E, nu)
    alpha = 1.0 + mu / lam
    f0, f1, f2 = F[..., :, 0], F[..., :, 1], F[..., :, 2]
    cross = (lambda a, b: torch.linalg.cross(a, b, dim=-1)) if xp is torch else np.cross
    g0, g1, g2 = cross(f1, f2), cross(f2, f0), cross(f0, f1)
    J = (f0 * g0).sum(-1)
    gJ = xp.concatenate([g0, g1, g2], -1) if xp is np else torch.cat([g0, g1, g2], -1)
    Ic = (F * F).sum((-1, -2)) if xp is torch else np.einsum("...ij,...ij->...", F, F)
    psi = 0.5 * mu * (Ic - 3.0) + 0.5 * lam * (J - alpha) ** 2
    vecF = torch.cat([f0, f1, f2], -1) if xp is torch else np.concatenate([f0, f1, f2], -1)
    grad = mu * vecF + lam * (J - alpha)[..., None] * gJ
    if xp is torch:
        HJ = torch.zeros(F.shape[:-2] + (9, 9), dtype=F.dtype, device=F.device)
        h0, h1, h2 = _hat_t(f0), _hat_t(f1), _hat_t(f2)
        eye9 = torch.eye(9, dtype=F.dtype, device=F.device)
    else:
        HJ = np.zeros(F.shape[:-2] + (9, 9))
        h0, h1, h2 = _hat(f0), _hat(f1), _hat(f2)
        eye9 = np.eye(9)
    HJ[..., 0:3, 3:6], HJ[..., 0:3, 6:9] = -h2, h1
    HJ[..., 3:6, 0:3], HJ[..., 3:6, 6:9] = h2, -h0
    HJ[..., 6:9, 0:3], HJ[..., 6:9, 3:6] = -h1, h0
    H = mu * eye9 + lam * gJ[..., :, None] * gJ[..., None, :] + lam * (J - alpha)[..., None, None] * HJ
    return psi, grad, H


def _hat_t(v):
    z = torch.zeros_like(v[..., 0])
    return torch.stack(
        [
            torch.stack([z, -v[..., 2], v[..., 1]], -1),
            torch.stack([v[..., 2], z, -v[..., 0]], -1),
            torch.stack([-v[..., 1], v[..., 0], z], -1),
        ],
        -2,
    )


def _psd_project(H):
    if isinstance(H, torch.Tensor):
        w, Q = torch.linalg.eigh(0.5 * (H + H.transpose(-1, -2)))
        return (Q * w.clamp_min(0.0)[..., None, :]) @ Q.transpose(-1, -2)
    w, Q = np.linalg.eigh(0.5 * (H + np.swapaxes(H, -1, -2)))
    w = np.maximum(w, 0.0)
    return np.einsum("...ik,...k,...jk->...ij", Q, w, Q)


def _shape_weights(X, tets):
    """Rest volume (T,) and w (T, 4, 3): dF[:, j]/dx_a = w[a, j] * I3."""
    Dm = np.stack([X[tets[:, a]] - X[tets[:, 0]] for a in (1, 2, 3)], -1)  # columns
    B = np.linalg.inv(Dm)
    vol = np.abs(np.linalg.det(Dm)) / 6.0
    w = np.empty((tets.shape[0], 4, 3))
    w[:, 1:, :] = B
    w[:, 0, :] = -B.sum(axis=1)
    return vol, w


def deformation_gradient(X, x, tets):
    vol, w = _shape_weights(X, tets)
    xs = x[tets]  # (T, 4, 3)
    F = np.einsum("tax,taj->txj", xs, w)
    return F, vol, w


_PAIRS = [(a, b) for a in range(4) for b in range(a, 4)]


def _generator_device():
    return "cuda" if torch.cuda.is_available() else "cpu"


def _element_chunk(X, x, t, swap, E, nu, pa, pb, device):
    F, vol, w = deformation_gradient(X, x, t)
    Ft = torch.from_numpy(F).to(device)
    _, _, HF = snh_energy_grad_hess_F(Ft, E, nu)
    P = _psd_project(HF).reshape(-1, 3, 3, 3, 3)  # [t, i, x, j, y] (F column i, comp x)
    wt = torch.from_numpy(w).to(device)
    He = torch.einsum("tai,tixjy->taxjy", wt, P)
    He = torch.einsum("tbj,taxjy->tabxy", wt, He)
    He = He * torch.from_numpy(vol).to(device)[:, None, None, None, None]
    blk = He[:, pa, pb]  # (t, 10, 3, 3)
    sw = torch.from_numpy(swap).to(device)
    blk = torch.where(sw[:, :, None, None], blk.transpose(-1, -2), blk)
    return blk.cpu().numpy()


def snh_element_blocks(X, x, tets, E, nu, chunk=None, device=None):
    """Upper-triangle 3x3 blocks of the PSD-projected SNH Hessian per tet.

    Returns rows (K,), cols (K,), blocks (K, 3, 3) with K = 10 * T, in
    tet-major order.  The batched 9x9 eigendecompositions run through torch
    (on the GPU when one is present); only the inputs depend on this.
    """
    device = device or _generator_device()
    if chunk is None:
        chunk = 32_768 if device == "cuda" else 400_000  # batched eigh sizes the solver accepts
    T = tets.shape[0]
    pa = np.array([p[0] for p in _PAIRS])
    pb = np.array([p[1] for p in _PAIRS])
    ra = tets[:, pa]
    cb = tets[:, pb]
    swap = ra > cb
    rows = np.where(swap, cb, ra).astype(np.int32).ravel()
    cols = np.where(swap, ra, cb).astype(np.int32).ravel()
    blocks = np.empty((T, 10, 3, 3))
    s = 0
    while s < T:
        try:
            blocks[s : s + chunk] = _element_chunk(X, x, tets[s : s + chunk], swap[s : s + chunk], E, nu, pa, pb,
                                                   device)
        except RuntimeError:
            if device == "cpu":
                raise
            device, chunk = "cpu", 400_000  # the GPU solver is unavailable here: finish on the host
            continue
        s += chunk
    return rows, cols, blocks.reshape(-1, 3, 3)


def lumped_mass_blocks(X, tets, rho, dt):
    """Diagonal blocks m_v / dt^2 * I3, m_v = rho * (quarter of incident tet volumes)."""
    V = X.shape[0]
    vol, _ = _shape_weights(X, tets)
    m = np.zeros(V)
    np.add.at(m, tets.ravel(), np.repeat(rho * vol / 4.0, 4))
    idx = np.arange(V, dtype=np.int32)
    blocks = (m / (dt * dt))[:, None, None] * np.eye(3)[None]
    return idx, idx.copy(), blocks


def random_pairs(rng, n_vertices, n_pairs):
    """Distinct unordered vertex pairs (i < j), drawn uniformly."""
    out = set()
    while len(out) < n_pairs:
        i, j = rng.integers(0, n_vertices, 2)
        if i != j:
            out.add((min(i, j), max(i, j)))
    p = np.array(sorted(out), dtype=np.int64)
    return p[rng.permutation(len(p))].astype(np.int32)


def near_pairs(rng, X, n_grid, n_pairs, radius):
    """Random vertex pairs (i < j) of an n_grid^3 cube grid with |X_i - X_j| < radius.

    Partners are drawn from the +-2 grid-cell neighbourhood of a uniformly
    drawn vertex and kept when closer than ``radius``; pairs may repeat and
    may coincide with mesh edges (they then become duplicate keys).
    """
    V = X.shape[0]
    n = n_grid
    out = []
    need = n_pairs
    while need > 0:
        i = rng.integers(0, V, 4 * need)
        off = rng.integers(-2, 3, (4 * need, 3))
        ijk = np.stack([i % n, (i // n) % n, i // (n * n)], -1) + off
        ok = np.all((ijk >= 0) & (ijk < n), axis=1)
        j = ijk[:, 0] + n * ijk[:, 1] + n * n * ijk[:, 2]
        i, j = i[ok], j[ok]
        d = np.linalg.norm(X[i] - X[j], axis=1)
        sel = (i != j) & (d < radius)
        i, j = i[sel], j[sel]
        take = min(need, i.size)
        out.append(np.stack([np.minimum(i, j), np.maximum(i, j)], -1)[:take])
        need -= take
    return np.concatenate(out).astype(np.int32)


def contact_blocks(rng, pairs, k_lo, k_hi):
    """Upper triplets of k n n^T couplings: (i,i,K), (j,j,K), (i,j,-K) per pair."""
    P = pairs.shape[0]
    nvec = rng.normal(size=(P, 3))
    nvec /= np.linalg.norm(nvec, axis=1, keepdims=True)
    k = np.exp(rng.uniform(np.log(k_lo), np.log(k_hi), P))
    K = k[:, None, None] * nvec[:, :, None] * nvec[:, None, :]
    i, j = pairs[:, 0].astype(np.int32), pairs[:, 1].astype(np.int32)
    rows = np.concatenate([i, j, np.minimum(i, j)])
    cols = np.concatenate([i, j, np.maximum(i, j)])
    blocks = np.concatenate([K, K, -K])
    return rows, cols, blocks
