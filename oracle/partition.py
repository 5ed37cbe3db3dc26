"""Level-0 domain partition with padding (Sec. 3.2; supplement Algorithm 1).

The paper partitions the mesh with METIS into M = ceil(V / (N - N_o)) parts
of at most N nodes each (Eq. num_subdomains), then assigns part p to MAS
subdomain p: node v gets slot N*p + (its rank inside the part), and empty
slots are padding (remap = -1).  METIS is not available and is not
reproducible by an independent implementation, so the partition is
specified as a deterministic rule that the oracle and the library
implement independently.

Recursive coordinate bisection of the rest positions (supplement
Algorithm 1 takes the node positions as input).  For a vertex set S with
P = ceil(|S| / N) > 1 parts to make:

  1. axis = the coordinate with the largest extent max - min over S
     (ties: the lower axis, x before y before z);
  2. order S by (coordinate along that axis, vertex index);
  3. the first N * ceil(P / 2) vertices form the left set, the rest the
     right set; recurse on both.

Leaves (|S| <= N) are parts, numbered left to right.  Every part but the
last holds exactly N vertices, so M = ceil(V / N) (N_o = 0).  On a
volumetric mesh the parts are compact boxes, hence densely connected --
what the paper obtains from METIS -- and numbering leaves left to right
puts neighbouring parts at consecutive indices, which is what the coarser
MAS levels group together.

Inside a part, vertices take slots in ascending vertex index (the paper's
stable sort by part index).

Two further rules: component_bisection runs the same bisection inside each
connected component of the mesh graph, so no part mixes two bodies; and
morton_partition groups N consecutive vertices in Morton order, the level-0
subdomains of the earlier MAS the paper compares against.

Test infrastructure only (see the package docstring).
"""

import numpy as np


def recursive_bisection(X, N, label0=None):
    """Part label (int32) of every vertex of positions X (V, 3), rule in the docstring.

    label0: initial sets (int, 0 .. S-1, every value used), each bisected on
    its own and numbered in that order; default one set of all vertices."""
    X = np.asarray(X, dtype=np.float64)
    V = X.shape[0]
    idx = np.arange(V)
    label = np.zeros(V, dtype=np.int64) if label0 is None else np.asarray(label0, dtype=np.int64).copy()
    n_sets = (int(label.max()) + 1 if label0 is not None else 1) if V else 0
    while n_sets:
        size = np.bincount(label, minlength=n_sets)
        parts = -(-size // N)
        split = parts > 1
        if not split.any():
            break
        lo = np.full((n_sets, 3), np.inf)
        hi = np.full((n_sets, 3), -np.inf)
        np.minimum.at(lo, label, X)
        np.maximum.at(hi, label, X)
        axis = np.argmax(hi - lo, axis=1)  # first maximum -> lower axis on ties
        coord = X[idx, axis[label]]
        order = np.lexsort((idx, coord, label))
        lab_o = label[order]
        start = np.concatenate([[0], np.cumsum(size)])[:-1]
        rank = np.arange(V) - start[lab_o]
        left = N * (-(-parts // 2))
        go_right = split[lab_o] & (rank >= left[lab_o])
        width = np.where(split, 2, 1)
        first_new = np.cumsum(width) - width
        label[order] = first_new[lab_o] + go_right
        n_sets = int(width.sum())
    return label.astype(np.int32)


def components(V, adj_ptr, adj):
    """Connected components of the mesh graph (CSR), numbered in the order of
    their smallest vertex index (component 0 holds vertex 0)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    adj_ptr = np.asarray(adj_ptr, dtype=np.int64)
    A = sp.csr_matrix((np.ones(len(adj)), np.asarray(adj, dtype=np.int64), adj_ptr), shape=(V, V))
    _, lab = connected_components(A, directed=False)
    first = np.full(lab.max() + 1 if V else 0, V, dtype=np.int64)
    np.minimum.at(first, lab, np.arange(V))
    rank = np.empty_like(first)
    rank[np.argsort(first, kind="stable")] = np.arange(first.size)
    return rank[lab]


def component_bisection(X, N, adj_ptr, adj):
    """Recursive coordinate bisection inside each connected component of the
    mesh graph (components numbered by their smallest vertex index): a part
    never mixes two bodies, which plain coordinate bisection does where
    separate bodies interleave in space.  The paper's connectivity-enhanced
    MAS gets connected subdomains from METIS (Sec. 3.2); on a single
    connected mesh this rule equals recursive_bisection."""
    return recursive_bisection(X, N, label0=components(np.asarray(X).shape[0], adj_ptr, adj))


MORTON_BITS = 10


def morton_codes(X, bits=MORTON_BITS):
    """Morton (Z-order) code of every vertex: each coordinate quantised to
    `bits` bits over the bounding box, q = min(floor((x - lo) / (hi - lo) *
    2^bits), 2^bits - 1) (0 on a flat axis), bits interleaved x, y, z from
    the least significant bit of x upward."""
    X = np.asarray(X, dtype=np.float64)
    lo, hi = X.min(axis=0), X.max(axis=0)
    code = np.zeros(X.shape[0], dtype=np.int64)
    for a in range(3):
        ext = hi[a] - lo[a]
        if ext > 0:
            q = np.floor((X[:, a] - lo[a]) / ext * float(1 << bits)).astype(np.int64)
            q = np.minimum(q, (1 << bits) - 1)
        else:
            q = np.zeros(X.shape[0], dtype=np.int64)
        for b in range(bits):
            code |= ((q >> b) & 1) << (3 * b + a)
    return code


def morton_partition(X, N):
    """Parts of N consecutive vertices in Morton order (ties by vertex index):
    the level-0 subdomains of the MAS of Wu et al. that the paper compares
    against (Sec. 3.1)."""
    code = morton_codes(X)
    order = np.lexsort((np.arange(code.size), code))
    part = np.empty(code.size, dtype=np.int64)
    part[order] = np.arange(code.size) // N
    return part.astype(np.int32)


def map_remap(part, N):
    """map[v] = slot of vertex v; remap[slot] = vertex or -1 (supplement Algorithm 1).

    Slot = N * part + rank of v among the vertices of its part, ascending
    vertex index.  remap has N * M entries, M = number of parts.
    """
    part = np.asarray(part)
    M = int(part.max()) + 1 if part.size else 0
    order = np.lexsort((np.arange(part.size), part))  # by part, then vertex
    remap = np.full(N * M, -1, dtype=np.int32)
    mp = np.empty(part.size, dtype=np.int32)
    s = 0
    for i, v in enumerate(order.tolist()):
        if i > 0 and part[v] != part[order[i - 1]]:
            s = 0
        if s >= N:
            raise ValueError("part larger than the domain size")
        slot = N * int(part[v]) + s
        remap[slot] = v
        mp[v] = slot
        s += 1
    return mp, remap
