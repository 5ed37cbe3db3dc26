"""Seeded coupled FEM / affine-body scenes (inputs of the two-level assembly).

Recipe (stand-in for the paper's FEM + ABD coupling scenes):
  * FEM part: the n^3 tet cube of synth.workloads (stable Neo-Hookean,
    E = 1e6, nu = 0.4, lumped mass rho = 1000, dt = 0.01);
  * n_bodies affine bodies: 2 cm cubes on a square grid resting on the
    cube's top face (centres at z = 1 + 1.2 cm), each with its 8 corners as
    contact nodes; xbar = corner rest position relative to the body centre;
  * body inertia: corner masses m = rho vol / 8 given as node blocks
    (m / dt^2) I, so that the Jacobian map yields sum_i m_i J_i^T J_i;
  * orthogonality potential kappa vol ||A^T A - I||_F^2, kappa = 1e11,
    at A = I + N(0, 0.01): its 9 x 9 Hessian in (a_1, a_2, a_3),
    PSD-projected, given on the body's own reduced rows 1..3;
  * contact pairs: 50% FEM-ABD (a body corner and one of the four top-face
    FEM vertices nearest below it), 25% ABD-ABD (corners of two bodies that
    are neighbours on the grid), 25% FEM-FEM (vertices closer than 2h);
    each pair a PSD block k n n^T with k log-uniform in [1e2, 1e6], added
    as [[K, -K], [-K, K]].  Pairs may repeat (duplicate keys).

Numbering: FEM vertices 0..V-1, body corner nodes V + 8b + c (full space);
reduced block rows: FEM vertices 0..V-1, body b at V + 4b + {0..3}.  The
reduced rows carry rest positions (a body's four rows at its centre) and a
coupling graph (mesh edges, the body's own rows, contact couplings mapped to
reduced rows) for the partition and the MAS levels.  Everything here makes
inputs; none of it is solver arithmetic.
"""

from dataclasses import dataclass
from types import SimpleNamespace

import numpy as np

from .hessians import contact_blocks, near_pairs
from .mesh import adjacency_csr, unique_sorted
from .workloads import make_tet_system, tet_geometry


@dataclass
class AbdScene:
    n_nodes: int          # full-space nodes: FEM vertices + 8 corners per body
    n_fem: int
    n_bodies: int
    body_of_node: np.ndarray  # int32 (n_nodes,), -1 for FEM vertices
    xbar: np.ndarray      # (n_nodes, 3) body-frame rest coordinates (0 for FEM)
    rows: np.ndarray      # int32 (K,) full-space / body-row indices, row <= col
    cols: np.ndarray
    blocks: np.ndarray    # (K, 3, 3)
    X: np.ndarray         # (n_red, 3) rest positions of the reduced rows
    adj_ptr: np.ndarray   # reduced-row coupling graph (CSR)
    adj: np.ndarray
    contacts: np.ndarray  # int32 (P, 2) contact couplings on reduced rows
    params: dict
    fem_x: np.ndarray = None     # with fem_blocks=False: the FEM part's deformed positions,
    fem_tets: np.ndarray = None  # and its tets (its Hessian blocks are left to the caller)

    @property
    def n_red(self):
        return self.n_fem + 4 * self.n_bodies


def _orthogonality_hessian(A, kv):
    """9 x 9 Hessian of kv sum_ij (a_i . a_j - delta_ij)^2 in (a_1, a_2, a_3), PSD-projected.

    H_kl = 4 kv [delta_kl sum_j a_j a_j^T + a_l a_k^T + G_kl I], G = A^T A - I."""
    a = [A[:, k] for k in range(3)]
    G = A.T @ A - np.eye(3)
    S = sum(np.outer(v, v) for v in a)
    H = np.zeros((9, 9))
    for k in range(3):
        for l in range(3):
            blk = np.outer(a[l], a[k]) + G[k, l] * np.eye(3)
            if k == l:
                blk = blk + S
            H[3 * k : 3 * k + 3, 3 * l : 3 * l + 3] = 4.0 * kv * blk
    H = 0.5 * (H + H.T)
    w, V = np.linalg.eigh(H)
    return (V * np.maximum(w, 0.0)) @ V.T


def make_abd_scene(n=100, n_bodies=2000, n_contacts=500_000, E=1e6, rho=1000.0, dt=0.01, kappa=1e11,
                   size=0.02, seed=1005, fem_blocks=True):
    """The scene of the recipe above.  fem_blocks=False leaves out the FEM
    part's element and mass blocks (same geometry, same draws for the rest)
    and returns its deformed positions and tets instead, for a caller that
    computes those blocks itself."""
    rng = np.random.default_rng(seed)
    if fem_blocks:
        fem = make_tet_system(n, E=E, rho=rho, dt=dt, n_contacts=0, seed=seed)
    else:
        X_, x_, tets_, ptr_, adj_ = tet_geometry(n, seed=seed)
        fem = SimpleNamespace(n_vertices=X_.shape[0], X=X_, x=x_, tets=tets_, adj_ptr=ptr_, adj=adj_,
                              rows=np.zeros(0, np.int32), cols=np.zeros(0, np.int32), blocks=np.zeros((0, 3, 3)))
    V = fem.n_vertices
    h = 1.0 / (n - 1)
    g = int(np.ceil(np.sqrt(n_bodies)))
    bi = np.arange(n_bodies)
    centre = np.stack([(bi % g + 0.5) / g, (bi // g + 0.5) / g, np.full(n_bodies, 1.0 + 0.6 * size)], -1)
    corner = np.array([[(c & 1) - 0.5, ((c >> 1) & 1) - 0.5, ((c >> 2) & 1) - 0.5] for c in range(8)]) * size
    n_nodes = V + 8 * n_bodies
    body_of_node = np.concatenate([np.full(V, -1), np.repeat(bi, 8)]).astype(np.int32)
    xbar = np.zeros((n_nodes, 3))
    xbar[V:] = np.tile(corner, (n_bodies, 1))
    Xfull = np.concatenate([fem.X, (centre[:, None, :] + corner[None]).reshape(-1, 3)])

    rows, cols, blocks = [fem.rows], [fem.cols], [fem.blocks]
    # body inertia as node blocks on the corners
    m = rho * size ** 3 / 8.0
    cn = np.arange(V, n_nodes, dtype=np.int32)
    rows.append(cn), cols.append(cn), blocks.append(np.broadcast_to(m / dt ** 2 * np.eye(3), (cn.size, 3, 3)))
    # orthogonality Hessians on the bodies' own rows 1..3 (indices n_nodes + 4b + a)
    kv = kappa * size ** 3
    for b in range(n_bodies):
        H = _orthogonality_hessian(np.eye(3) + rng.normal(0.0, 0.01, (3, 3)), kv)
        for k in range(3):
            for l in range(k, 3):
                rows.append(np.array([n_nodes + 4 * b + 1 + k], np.int32))
                cols.append(np.array([n_nodes + 4 * b + 1 + l], np.int32))
                blocks.append(H[None, 3 * k : 3 * k + 3, 3 * l : 3 * l + 3])
    # contacts
    n_fa, n_aa = n_contacts // 2, n_contacts // 4
    n_ff = n_contacts - n_fa - n_aa
    # FEM-ABD: a body corner and one of the four top-face vertices nearest below it
    c_fa = rng.integers(V, n_nodes, n_fa)
    ij = np.floor(Xfull[c_fa, :2] / h).astype(np.int64)
    di, dj = rng.integers(0, 2, n_fa), rng.integers(0, 2, n_fa)
    fi = np.clip(ij[:, 0] + di, 0, n - 1)
    fj = np.clip(ij[:, 1] + dj, 0, n - 1)
    v_fa = fi + n * fj + n * n * (n - 1)
    p_fa = np.stack([v_fa, c_fa], -1)
    # ABD-ABD: a corner of a body and a corner of a grid neighbour
    b0 = rng.integers(0, n_bodies, n_aa)
    step = np.array([1, -1, g, -g])[rng.integers(0, 4, n_aa)]
    b1 = b0 + step
    bad = (b1 < 0) | (b1 >= n_bodies) | ((np.abs(step) == 1) & (b0 // g != b1 // g))
    b1[bad] = np.where(b0[bad] + 1 < n_bodies, b0[bad] + 1, b0[bad] - 1)
    c0 = V + 8 * b0 + rng.integers(0, 8, n_aa)
    c1 = V + 8 * b1 + rng.integers(0, 8, n_aa)
    p_aa = np.stack([np.minimum(c0, c1), np.maximum(c0, c1)], -1)
    # FEM-FEM: near pairs
    p_ff = near_pairs(rng, fem.X, n, n_ff, 2.0 * h).astype(np.int64)
    pairs = np.concatenate([p_fa, p_aa, p_ff]).astype(np.int32)
    cr, cc, cb = contact_blocks(rng, pairs, 1e2, 1e6)
    rows.append(cr), cols.append(cc), blocks.append(cb)

    rows = np.concatenate(rows).astype(np.int32)
    cols = np.concatenate(cols).astype(np.int32)
    blocks = np.concatenate([np.asarray(b, dtype=np.float64).reshape(-1, 3, 3) for b in blocks])
    perm = np.random.default_rng(seed + 7919).permutation(rows.size)

    # reduced rows: positions, coupling graph and contact couplings
    red_of = lambda node: np.where(node < V, node, V + 4 * ((node - V) // 8))  # first row of a body
    Xr = np.concatenate([fem.X, np.repeat(centre, 4, axis=0)])
    src = np.repeat(np.arange(V), np.diff(fem.adj_ptr))
    e_mesh = np.stack([src, fem.adj], -1)
    e_mesh = e_mesh[e_mesh[:, 0] < e_mesh[:, 1]]
    base = V + 4 * bi
    e_body = np.concatenate([np.stack([base + a, base + c], -1) for a in range(4) for c in range(a + 1, 4)])
    ptr, adj = adjacency_csr(V + 4 * n_bodies, np.concatenate([e_mesh, e_body]))
    ra, rb = red_of(pairs[:, 0].astype(np.int64)), red_of(pairs[:, 1].astype(np.int64))
    cpl = []
    for a in range(4):  # a coupling reaches every reduced row of a body
        for c in range(4):
            x = ra + np.where(pairs[:, 0] >= V, a, 0)
            y = rb + np.where(pairs[:, 1] >= V, c, 0)
            cpl.append(np.stack([np.minimum(x, y), np.maximum(x, y)], -1))
    cpl = np.concatenate(cpl).astype(np.int64)
    nr = V + 4 * n_bodies
    key = unique_sorted(cpl[:, 0] * nr + cpl[:, 1])  # distinct pairs in (first, second) order
    cpl = np.stack([key // nr, key % nr], -1)
    cpl = cpl[cpl[:, 0] != cpl[:, 1]].astype(np.int32)
    return AbdScene(
        n_nodes=n_nodes, n_fem=V, n_bodies=n_bodies, body_of_node=body_of_node, xbar=xbar,
        rows=rows[perm], cols=cols[perm], blocks=np.ascontiguousarray(blocks[perm]),
        X=Xr, adj_ptr=ptr, adj=adj, contacts=cpl,
        params=dict(n=n, n_bodies=n_bodies, n_contacts=n_contacts, E=E, rho=rho, dt=dt, kappa=kappa, size=size,
                    seed=seed),
        fem_x=None if fem_blocks else fem.x, fem_tets=None if fem_blocks else fem.tets,
    )
