"""Tet-cube meshes and their vertex adjacency graph (seeded, numpy only)."""

import numpy as np

# The two mirror-image 5-tet splits of a hex cell.  Local corner c encodes
# (i, j, k) offsets as c = i + 2 j + 4 k.  Split A has the central tet
# {1, 2, 4, 7}; split B has {0, 3, 5, 6}.  Alternating them with the parity
# of the cell index makes the face diagonals of neighbouring cells agree.
_SPLIT_A = np.array([[1, 2, 4, 7], [0, 1, 2, 4], [3, 1, 7, 2], [5, 1, 4, 7], [6, 2, 7, 4]])
_SPLIT_B = np.array([[0, 3, 5, 6], [1, 0, 5, 3], [2, 0, 3, 6], [4, 0, 6, 5], [7, 3, 6, 5]])


def tet_cube(n, rng=None, jitter=0.05):
    """Unit cube with n^3 vertices, (n-1)^3 cells, 5 tets per cell.

    Returns (X, tets): rest positions (V, 3) float64, with every coordinate
    jittered by N(0, jitter * h) when ``rng`` is given, and tets (T, 4)
    int32 with positive rest volume.  Vertex index = i + n j + n^2 k.
    """
    h = 1.0 / (n - 1)
    g = np.arange(n, dtype=np.float64) * h
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1)  # [i, j, k, xyz]
    X = X.transpose(2, 1, 0, 3).reshape(-1, 3)  # index i + n j + n^2 k
    if rng is not None and jitter > 0:
        X = X + rng.normal(0.0, jitter * h, X.shape)
    c = np.arange(n - 1)
    ci, cj, ck = np.meshgrid(c, c, c, indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    corners = np.empty((ci.size, 8), dtype=np.int64)
    for cc in range(8):
        di, dj, dk = cc & 1, (cc >> 1) & 1, (cc >> 2) & 1
        corners[:, cc] = (ci + di) + n * (cj + dj) + n * n * (ck + dk)
    parity = (ci + cj + ck) & 1
    tets = np.where(parity[:, None, None] == 0, corners[:, _SPLIT_A], corners[:, _SPLIT_B])
    tets = tets.reshape(-1, 4)
    # orient every tet positively at rest
    d = X[tets[:, 1:]] - X[tets[:, :1]]
    vol = np.einsum("ij,ij->i", d[:, 0], np.cross(d[:, 1], d[:, 2]))
    neg = vol < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    return X, tets.astype(np.int32)


def unique_sorted(a):
    """Sorted distinct values of a 1-D integer array (a sort and a neighbour
    test: some numpy releases take a far slower hashing path in np.unique)."""
    s = np.sort(np.asarray(a).ravel())
    if s.size == 0:
        return s
    return s[np.concatenate([[True], s[1:] != s[:-1]])]


def tet_edges(tets):
    """Unique undirected vertex pairs (a < b) of a tet mesh, sorted, (E, 2) int64."""
    t = tets.astype(np.int64)
    pairs = np.concatenate([t[:, [a, b]] for a in range(4) for b in range(a + 1, 4)])
    pairs.sort(axis=1)
    V = int(t.max()) + 1 if t.size else 1
    key = unique_sorted(pairs[:, 0] * V + pairs[:, 1])
    return np.stack([key // V, key % V], -1)


def adjacency_csr(n_vertices, edges):
    """Symmetric CSR (ptr, adj) int32 of an undirected edge list, neighbours ascending."""
    e = np.asarray(edges, dtype=np.int64)
    src = np.concatenate([e[:, 0], e[:, 1]])
    dst = np.concatenate([e[:, 1], e[:, 0]])
    keep = src != dst
    src, dst = src[keep], dst[keep]
    key = unique_sorted(src * n_vertices + dst)
    src, dst = key // n_vertices, key % n_vertices
    ptr = np.zeros(n_vertices + 1, dtype=np.int64)
    np.add.at(ptr, src + 1, 1)
    return np.cumsum(ptr).astype(np.int32), dst.astype(np.int32)
