"""Seeded stiff-cloth systems (inputs): a triangle sheet with a membrane
Hessian that includes the cubic strain-limiting term, plus hinge bending.

Recipe (unit square sheet, n x n vertices, h = 1/(n-1), two triangles per
quad, thickness t = 1e-3 m, rho = 200 kg/m^3, dt = 0.01 s):
  * deformed positions: in-plane x' = [[1 + eps, s], [0, 1]] x with
    eps = 0.02 and s ~ U(0, 0.1), plus N(0, 0.01 h) noise on all three
    coordinates (the out-of-plane part gives the hinges bending);
  * stretching (Baraff-Witkin in I5 form): lam a_t (sqrt(I5) - 1)^2 per
    direction, lam = 0.05 MPa, Hessian clamped to PSD along its eigenvectors;
  * shearing: 0.3 lam a_t (f0 . f1)^2, Gauss-Newton Hessian;
  * strain limiting: E a_t max(sqrt(I5) - 1, 0)^3 per direction with E = 1e8
    and the analytic PSD Hessian of Sec. 4;
  * bending: k_b (theta - theta_0)^2 per interior edge with the Gauss-Newton
    Hessian 2 k_b grad(theta) grad(theta)^T, k_b = E t^3 / 12 * |e|^2 / (A_1 + A_2);
  * lumped mass rho t A / 3 per triangle corner, divided by dt^2.
a_t is the rest area times the thickness.  Everything here produces inputs
(triplets); none of it is solver arithmetic.
"""

import numpy as np
import torch

from .mesh import adjacency_csr
from .workloads import TetSystem


def sheet(n):
    """Rest positions (V, 3) with z = 0 and triangles (T, 3); vertex index = i + n j."""
    h = 1.0 / (n - 1)
    g = np.arange(n) * h
    X = np.stack(np.meshgrid(g, g, indexing="xy"), -1).reshape(-1, 2)
    X = np.concatenate([X, np.zeros((X.shape[0], 1))], 1)
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="xy")
    a = (i + n * j).ravel()
    b, c, d = a + 1, a + n, a + n + 1
    tris = np.concatenate([np.stack([a, b, d], 1), np.stack([a, d, c], 1)]).astype(np.int32)
    return X, tris


def hinges(tris):
    """Interior edges as (e0, e1, opposite in tri 1, opposite in tri 2)."""
    T = tris.shape[0]
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    opp = np.concatenate([tris[:, 2], tris[:, 0], tris[:, 1]])
    key = np.minimum(e[:, 0], e[:, 1]).astype(np.int64) * (tris.max() + 1) + np.maximum(e[:, 0], e[:, 1])
    order = np.argsort(key, kind="stable")
    k = key[order]
    same = np.nonzero(k[1:] == k[:-1])[0]
    i0, i1 = order[same], order[same + 1]
    return np.stack([e[i0, 0], e[i0, 1], opp[i0], opp[i1]], 1).astype(np.int32)


def _membrane_F_hessians(Fm, area_t, lam, E):
    """Per-triangle 6 x 6 PSD Hessians in vec(F) = [f0; f1] (torch, float64)."""
    f0, f1 = Fm[:, :, 0], Fm[:, :, 1]
    T = Fm.shape[0]
    eye3 = torch.eye(3, dtype=Fm.dtype, device=Fm.device)
    H = torch.zeros((T, 6, 6), dtype=Fm.dtype, device=Fm.device)
    for d, f in ((0, f0), (1, f1)):
        sl = slice(3 * d, 3 * d + 3)
        s = f.norm(dim=1).clamp_min(1e-12)
        ff = f[:, :, None] * f[:, None, :] / (s * s)[:, None, None]
        # stretching lam (s - 1)^2: 2 lam along f, 2 lam (1 - 1/s) across, clamped at 0
        Hs = 2 * lam * (ff + (1 - 1 / s).clamp_min(0.0)[:, None, None] * (eye3 - ff))
        # strain limit E max(s - 1, 0)^3: 3 E (1 - 1/s)(s - 1) I + 3 E (s^2 - 1)/s^3 f f^T for s > 1
        act = (s > 1.0).to(Fm.dtype)
        Hsl = 3 * E * act[:, None, None] * (((1 - 1 / s) * (s - 1))[:, None, None] * eye3
                                            + ((s * s - 1) / s ** 3)[:, None, None] * f[:, :, None] * f[:, None, :])
        H[:, sl, sl] += Hs + Hsl
    # shearing 0.3 lam (f0 . f1)^2, Gauss-Newton: 2 mu g g^T, g = [f1; f0]
    g = torch.cat([f1, f0], 1)
    H += 2 * 0.3 * lam * g[:, :, None] * g[:, None, :]
    return H * area_t[:, None, None]


def strain_limit_F_hessian(F, E=1.0):
    """The strain-limiting part alone for F (T, 3, 2), used to check the generator."""
    f0, f1 = F[..., 0], F[..., 1]
    eye3 = np.eye(3)
    H = np.zeros(F.shape[:-2] + (6, 6))
    for d, f in ((0, f0), (1, f1)):
        s = np.linalg.norm(f, axis=-1)
        act = (s > 1.0).astype(float)
        H[..., 3 * d : 3 * d + 3, 3 * d : 3 * d + 3] = 3 * E * act[..., None, None] * (
            ((1 - 1 / s) * (s - 1))[..., None, None] * eye3
            + ((s * s - 1) / s ** 3)[..., None, None] * f[..., :, None] * f[..., None, :]
        )
    return H


def _dihedral_grad(P):
    """theta and d theta / d P for hinges P (H, 4, 3) = (e0, e1, o1, o2)."""
    P = P.clone().requires_grad_(True)
    e0, e1, o1, o2 = P[:, 0], P[:, 1], P[:, 2], P[:, 3]
    e = e1 - e0
    n1 = torch.linalg.cross(e, o1 - e0, dim=1)
    n2 = torch.linalg.cross(o2 - e0, e, dim=1)
    en = e / e.norm(dim=1, keepdim=True)
    theta = torch.atan2((torch.linalg.cross(n1, n2, dim=1) * en).sum(1), (n1 * n2).sum(1))
    (g,) = torch.autograd.grad(theta.sum(), P)
    return theta.detach(), g


def make_cloth_system(n=512, E=1e8, lam=0.05e6, thickness=1e-3, rho=200.0, dt=0.01, eps=0.02, seed=1003,
                      device=None):
    device = device or ("cuda" if torch.cuda.is_available() else "cpu")
    rng = np.random.default_rng(seed)
    h = 1.0 / (n - 1)
    X, tris = sheet(n)
    s = rng.uniform(0.0, 0.1)
    A = np.array([[1 + eps, s, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    x = X @ A.T + rng.normal(0.0, 0.01 * h, X.shape)
    # membrane
    Xt = torch.as_tensor(X, device=device)
    xt = torch.as_tensor(x, device=device)
    tt = torch.as_tensor(tris.astype(np.int64), device=device)
    Dm = torch.stack([Xt[tt[:, 1], :2] - Xt[tt[:, 0], :2], Xt[tt[:, 2], :2] - Xt[tt[:, 0], :2]], 2)  # (T, 2, 2)
    area = 0.5 * torch.abs(torch.linalg.det(Dm))
    Bm = torch.linalg.inv(Dm)
    w = torch.zeros((tris.shape[0], 3, 2), dtype=torch.float64, device=device)
    w[:, 1:, :] = Bm
    w[:, 0, :] = -Bm.sum(1)
    Fm = torch.einsum("tax,taj->txj", xt[tt], w)  # (T, 3, 2)
    HF = _membrane_F_hessians(Fm, area * thickness, lam, E).reshape(-1, 2, 3, 2, 3)  # [t, i, x, j, y]
    He = torch.einsum("tai,tbj,tixjy->tabxy", w, w, HF)  # (T, 3, 3, 3, 3)
    pairs = [(a, b) for a in range(3) for b in range(a, 3)]
    rows, cols, blocks = [], [], []
    for a, b in pairs:
        ra, cb = tt[:, a], tt[:, b]
        swap = ra > cb
        rows.append(torch.where(swap, cb, ra))
        cols.append(torch.where(swap, ra, cb))
        blk = He[:, a, b]
        blocks.append(torch.where(swap[:, None, None], blk.transpose(1, 2), blk))
    # bending
    hg = hinges(tris)
    hgt = torch.as_tensor(hg.astype(np.int64), device=device)
    theta, grad = _dihedral_grad(xt[hgt])
    e_len = (Xt[hgt[:, 1]] - Xt[hgt[:, 0]]).norm(dim=1)
    a1 = 0.5 * torch.linalg.cross(Xt[hgt[:, 1]] - Xt[hgt[:, 0]], Xt[hgt[:, 2]] - Xt[hgt[:, 0]], dim=1).norm(dim=1)
    a2 = 0.5 * torch.linalg.cross(Xt[hgt[:, 1]] - Xt[hgt[:, 0]], Xt[hgt[:, 3]] - Xt[hgt[:, 0]], dim=1).norm(dim=1)
    kb = E * thickness ** 3 / 12.0 * e_len ** 2 / (a1 + a2)
    Hb = 2 * kb[:, None, None, None, None] * grad[:, :, None, :, None] * grad[:, None, :, None, :]  # [h, a, b, x, y]
    for a in range(4):
        for b in range(a, 4):
            ra, cb = hgt[:, a], hgt[:, b]
            swap = ra > cb
            rows.append(torch.where(swap, cb, ra))
            cols.append(torch.where(swap, ra, cb))
            blk = Hb[:, a, b]
            blocks.append(torch.where(swap[:, None, None], blk.transpose(1, 2), blk))
    # lumped mass
    m = torch.zeros(X.shape[0], dtype=torch.float64, device=device)
    m.index_add_(0, tt.reshape(-1), (rho * thickness * area / 3.0).repeat_interleave(3))
    idx = torch.arange(X.shape[0], device=device)
    rows.append(idx)
    cols.append(idx)
    blocks.append((m / dt ** 2)[:, None, None] * torch.eye(3, dtype=torch.float64, device=device))
    rows = torch.cat(rows).cpu().numpy().astype(np.int32)
    cols = torch.cat(cols).cpu().numpy().astype(np.int32)
    blocks = torch.cat(blocks).cpu().numpy()
    perm = np.random.default_rng(seed + 7919).permutation(rows.size)
    # coupling graph: triangle edges and hinge pairs (all element-internal pairs)
    ep = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [0, 2]], hg[:, [2, 3]]]).astype(np.int64)
    ep.sort(axis=1)
    ptr, adj = adjacency_csr(X.shape[0], ep)
    return TetSystem(
        n_grid=n, X=X, rows=rows[perm], cols=cols[perm], blocks=np.ascontiguousarray(blocks[perm]),
        adj_ptr=ptr, adj=adj, contacts=np.zeros((0, 2), np.int32),
        params=dict(n=n, E=E, lam=lam, thickness=thickness, rho=rho, dt=dt, shear=s, seed=seed, kind="cloth"),
    )
