"""Connectivity-enhanced MAS preconditioner (Sec. 3; supplement Sec. 2, Eq. 4-6).

Definitions restated from the paper, in the order the paper gives them:

Levels (supplement Algorithms 2-5).  Items of level 0 are the N*M slots of
the padded partition (fine node u sits at slot map[u]); items of level
l >= 1 are supernodes, numbered consecutively.  coarse[l][u] is the item
holding fine node u at level l (coarse[0] = map).  Level-l domain d is the
item range [d*N, d*N + N).

  * Connectivity (Alg. 2 initial hash, Alg. 3 contact handling): items a != b
    of the same level-l domain are adjacent iff some fine pair (u, v) of the
    mesh graph or of the contact list has coarse[l][u] = a and
    coarse[l][v] = b.  In bit form, item a's 32-bit mask holds its own lane
    bit (a mod N) and the lane bits of its in-domain neighbours.
  * Expansion (Alg. 4): the supernodes of level l+1 are the connected
    components of that adjacency inside each domain.
  * Numbering (Alg. 5): components are numbered domain by domain and, inside
    a domain, by the smallest lane among their items (the "elected" lane).
  * A level is added while the level count is below ``max_levels``, the
    current level has more than one domain, and at least one merge happened
    (fewer supernodes than real items).

Level matrices (Alg. 1): M_{l,d} = S_d C_l A C_l^T S_d^T, i.e. block (i, j)
of domain d sums every block A_uv of the full symmetric matrix with
coarse[l][u] = d*N + i and coarse[l][v] = d*N + j.

Inverses (Alg. 1, "invert unpadded parts"): each domain's matrix restricted
to its real items is inverted (Cholesky-based, FP64); padded rows and
columns of the inverse stay zero.  A non-positive pivot is reported.

Apply (supplement Eq. 4-6): z = sum_l C_l^T M_l^{-1} C_l r, where C_l sums
the fine 3-vectors of every item and M_l^{-1} is block-diagonal over
domains.  Level 0 alone is block-Jacobi over the domains (Eq. 4).

Test infrastructure only (see the package docstring).
"""

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


class NotSPDError(ValueError):
    pass


@dataclass
class Levels:
    N: int
    coarse: list  # per level: int64 (V,) item of every fine node
    n_items: list  # per level: item count (level 0: N*M slots incl. padding)
    real: list = field(default_factory=list)  # per level: bool (n_items,) item has a fine node

    @property
    def n_levels(self):
        return len(self.coarse)

    def n_domains(self, l):
        return -(-self.n_items[l] // self.N)


def fine_edges(adj_ptr, adj, contacts):
    """Undirected fine pairs (u, v), u != v: mesh graph edges plus contact pairs."""
    adj_ptr = np.asarray(adj_ptr, dtype=np.int64)
    src = np.repeat(np.arange(adj_ptr.size - 1), np.diff(adj_ptr))
    e = np.stack([src, np.asarray(adj, dtype=np.int64)], -1)
    if contacts is not None and len(contacts):
        e = np.concatenate([e, np.asarray(contacts, dtype=np.int64).reshape(-1, 2)])
    e = e[e[:, 0] != e[:, 1]]
    return e


def in_domain_masks(item_of_u, N, n_items, edges):
    """Alg. 2 + Alg. 3 masks: own lane bit plus lane bits of in-domain neighbours.

    Items that hold no fine node (padding) keep mask 0.
    """
    masks = np.zeros(n_items, dtype=np.int64)
    items = np.unique(item_of_u)
    masks[items] = np.left_shift(1, items % N)
    a = item_of_u[edges[:, 0]]
    b = item_of_u[edges[:, 1]]
    same = (a != b) & (a // N == b // N)
    np.bitwise_or.at(masks, a[same], np.left_shift(1, b[same] % N))
    np.bitwise_or.at(masks, b[same], np.left_shift(1, a[same] % N))
    return masks


def next_level(item_of_u, N, n_items, real, edges):
    """Supernode id of every level-l item (Alg. 4-5); returns (next_of_item, n_next).

    Components are found by breadth-first search over the in-domain
    adjacency; scanning lanes in ascending order makes the first item seen
    of each component its smallest lane, which fixes the numbering.
    """
    masks = in_domain_masks(item_of_u, N, n_items, edges)
    next_of_item = np.full(n_items, -1, dtype=np.int64)
    nid = 0
    for d in range(-(-n_items // N)):
        for lane in range(N):
            a = d * N + lane
            if a >= n_items or not real[a] or next_of_item[a] >= 0:
                continue
            stack = [a]
            next_of_item[a] = nid
            while stack:
                s = stack.pop()
                m = int(masks[s])
                for bl in range(N):
                    if (m >> bl) & 1:
                        b = d * N + bl
                        if next_of_item[b] < 0 and real[b]:
                            next_of_item[b] = nid
                            stack.append(b)
            nid += 1
    return next_of_item, nid


def build_levels(map_, N, max_levels, adj_ptr, adj, contacts=None):
    """All MAS levels under the rules in the module docstring."""
    map_ = np.asarray(map_, dtype=np.int64)
    V = map_.size
    M = int(map_.max()) // N + 1 if V else 0
    n0 = M * N
    real0 = np.zeros(n0, dtype=bool)
    real0[map_] = True
    lv = Levels(N=N, coarse=[map_], n_items=[n0], real=[real0])
    edges = fine_edges(adj_ptr, adj, contacts)
    while lv.n_levels < max_levels:
        l = lv.n_levels - 1
        if lv.n_items[l] <= N:
            break
        nxt, n_next = next_level(lv.coarse[l], N, lv.n_items[l], lv.real[l], edges)
        if n_next >= int(lv.real[l].sum()):
            break
        lv.coarse.append(nxt[lv.coarse[l]])
        lv.n_items.append(n_next)
        lv.real.append(np.ones(n_next, dtype=bool))
    return lv


def level_matrices(lv, rid, cid, au):
    """Dense domain matrices per level: list of (n_domains, 3N, 3N) float64 (Alg. 1)."""
    N = lv.N
    out = []
    rid = np.asarray(rid, dtype=np.int64)
    cid = np.asarray(cid, dtype=np.int64)
    for l in range(lv.n_levels):
        a = lv.coarse[l][rid]
        b = lv.coarse[l][cid]
        M = np.zeros((lv.n_domains(l), N, N, 3, 3))
        same = a // N == b // N
        np.add.at(M, (a[same] // N, a[same] % N, b[same] % N), au[same])
        off = same & (rid != cid)
        np.add.at(M, (b[off] // N, b[off] % N, a[off] % N), np.swapaxes(au[off], -1, -2))
        out.append(M.transpose(0, 1, 3, 2, 4).reshape(-1, 3 * N, 3 * N))
    return out


def invert_domains(lv, mats):
    """Per-domain inverses of the real items' part; padded rows/cols zero."""
    N = lv.N
    invs = []
    for l, Ms in enumerate(mats):
        real = np.zeros(lv.n_domains(l) * N, dtype=bool)
        real[: lv.n_items[l]] = lv.real[l]
        inv = np.zeros_like(Ms)
        for d in range(Ms.shape[0]):
            lanes = np.nonzero(real[d * N : d * N + N])[0]
            if lanes.size == 0:
                continue
            idx = (3 * lanes[:, None] + np.arange(3)[None]).ravel()
            sub = Ms[d][np.ix_(idx, idx)]
            try:
                L = np.linalg.cholesky(sub)
            except np.linalg.LinAlgError as e:
                raise NotSPDError(f"level {l} domain {d} is not SPD") from e
            Linv = np.linalg.inv(L)
            inv[d][np.ix_(idx, idx)] = Linv.T @ Linv
        invs.append(inv)
    return invs


def inverse_factors(lv, mats):
    """Per-domain inverse Cholesky factors W = L^{-1} (lower triangular) of the
    real items' part, M_d = L L^T, so that M_d^{-1} = W^T W; padded rows and
    columns zero.  The low-precision (BF16) preconditioner stores W instead of
    M_d^{-1}: any rounding of W keeps W^T W positive semi-definite."""
    N = lv.N
    facs = []
    for l, Ms in enumerate(mats):
        real = np.zeros(lv.n_domains(l) * N, dtype=bool)
        real[: lv.n_items[l]] = lv.real[l]
        fac = np.zeros_like(Ms)
        for d in range(Ms.shape[0]):
            lanes = np.nonzero(real[d * N : d * N + N])[0]
            if lanes.size == 0:
                continue
            idx = (3 * lanes[:, None] + np.arange(3)[None]).ravel()
            L = np.linalg.cholesky(Ms[d][np.ix_(idx, idx)])
            fac[d][np.ix_(idx, idx)] = np.linalg.inv(L)
        facs.append(fac)
    return facs


def coarsener(lv, l):
    """C_l of supplement Eq. 5-6 as a sparse 0/1 matrix acting on nodes:
    row a (an item of level l, padded domains included) sums the nodes u with
    coarse[l][u] = a.  Applied to (V, m) arrays it acts on each 3-vector."""
    V = lv.coarse[0].size
    n_pad = lv.n_domains(l) * lv.N
    return sp.csr_matrix((np.ones(V), (lv.coarse[l], np.arange(V))), shape=(n_pad, V))


def apply(lv, invs, r, C=None):
    """z = sum_l C_l^T M_l^{-1} C_l r for r of shape (..., V, 3) or (..., 3V)."""
    N = lv.N
    r = np.asarray(r, dtype=np.float64)
    shape = r.shape
    V = lv.coarse[0].size
    r3 = r.reshape(shape[:-1] + (V, 3)) if shape[-1] == 3 * V else r
    lead = r3.shape[:-2]
    r3 = r3.reshape((-1, V, 3))
    K = r3.shape[0]
    R = r3.transpose(1, 0, 2).reshape(V, 3 * K)  # node-major
    Z = np.zeros_like(R)
    for l in range(lv.n_levels):
        Cl = C[l] if C is not None else coarsener(lv, l)
        nd = lv.n_domains(l)
        rl = (Cl @ R).reshape(nd, N, K, 3).transpose(0, 1, 3, 2).reshape(nd, 3 * N, K)
        zl = np.matmul(invs[l], rl)  # block-diagonal M_l^{-1}, one dense product per domain
        Z += Cl.T @ zl.reshape(nd, N, 3, K).transpose(0, 1, 3, 2).reshape(nd * N, 3 * K)
    z = Z.reshape(V, K, 3).transpose(1, 0, 2)
    return z.reshape(lead + (V, 3)).reshape(shape)


@dataclass
class MAS:
    levels: Levels
    mats: list
    invs: list
    C: list = field(default_factory=list)

    def __post_init__(self):
        if not self.C:
            self.C = [coarsener(self.levels, l) for l in range(self.levels.n_levels)]

    def __call__(self, r):
        return apply(self.levels, self.invs, r, self.C)


def build_mas(map_, N, max_levels, adj_ptr, adj, contacts, rid, cid, au):
    lv = build_levels(map_, N, max_levels, adj_ptr, adj, contacts)
    mats = level_matrices(lv, rid, cid, au)
    return MAS(lv, mats, invert_domains(lv, mats))


def dense_preconditioner(lv, invs):
    """Explicit M^{-1} (3V x 3V) built from 0/1 coarsening matrices C_l (tiny meshes)."""
    V = lv.coarse[0].size
    N = lv.N
    Minv = np.zeros((3 * V, 3 * V))
    for l in range(lv.n_levels):
        n = lv.n_domains(l) * N
        C = np.zeros((3 * n, 3 * V))
        for u in range(V):
            a = int(lv.coarse[l][u])
            C[3 * a : 3 * a + 3, 3 * u : 3 * u + 3] = np.eye(3)
        B = np.zeros((3 * n, 3 * n))
        for d in range(lv.n_domains(l)):
            s = slice(3 * N * d, 3 * N * (d + 1))
            B[s, s] = invs[l][d]
        Minv += C.T @ B @ C
    return Minv
