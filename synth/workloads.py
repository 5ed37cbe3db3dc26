"""Named synthetic workloads: tet-cube systems shaped like the paper's FEM scenes.

Recipe (unit cube, side 1 m, h = 1/(n-1)):
  * n^3 vertices, 5 tets per cell; rest positions jittered N(0, 0.05 h);
  * deformed positions x = (I + G) X + N(0, 0.02 h), G_ij ~ U(-0.1, 0.1),
    so the PSD projection of the stable Neo-Hookean Hessian is active;
  * SNH Hessian with Young's modulus E, Poisson ratio nu, plus lumped
    mass m_v / dt^2 on the diagonal (the system K + M / dt^2);
  * contact stand-ins: PSD blocks k n n^T on vertex pairs, k log-uniform;
  * right-hand sides N(0, 1), seed 2000 + rhs index.

The stable Neo-Hookean F-space Hessian is linear in E at fixed nu (both
Lame parameters scale with E and alpha = 1 + mu/lam does not), and PSD
projection commutes with positive scaling, so systems that differ only in
E share one set of element blocks computed at E = 1.
"""

from dataclasses import dataclass, field

import numpy as np

from .hessians import (
    contact_blocks,
    lumped_mass_blocks,
    near_pairs,
    random_pairs,
    snh_element_blocks,
)
from .mesh import adjacency_csr, tet_cube, tet_edges


@dataclass
class TetSystem:
    n_grid: int
    X: np.ndarray  # rest positions (V, 3)
    rows: np.ndarray  # int32 (K,)  upper-triangle triplets, duplicates allowed
    cols: np.ndarray  # int32 (K,)
    blocks: np.ndarray  # float64 (K, 3, 3) row-major
    adj_ptr: np.ndarray  # int32 (V+1,) mesh vertex graph (contacts excluded)
    adj: np.ndarray  # int32
    contacts: np.ndarray  # int32 (P, 2) contact vertex pairs
    params: dict = field(default_factory=dict)

    @property
    def n_vertices(self):
        return self.X.shape[0]


@dataclass
class _Geometry:
    n: int
    X: np.ndarray
    tets: np.ndarray
    unit_rows: np.ndarray
    unit_cols: np.ndarray
    unit_blocks: np.ndarray  # element blocks at E = 1
    mass: tuple
    contacts: np.ndarray
    contact_trip: tuple
    adj_ptr: np.ndarray
    adj: np.ndarray
    shuffle_seed: int


def _geometry(n, nu, rho, dt, n_contacts, contact_mode, k_range, seed):
    rng = np.random.default_rng(seed)
    h = 1.0 / (n - 1)
    X, tets = tet_cube(n, rng, jitter=0.05)
    G = rng.uniform(-0.1, 0.1, (3, 3))
    x = X @ (np.eye(3) + G).T + rng.normal(0.0, 0.02 * h, X.shape)
    r_e, c_e, b_e = snh_element_blocks(X, x, tets, 1.0, nu)
    mass = lumped_mass_blocks(X, tets, rho, dt)
    V = X.shape[0]
    if n_contacts > 0:
        if contact_mode == "random":
            pairs = random_pairs(rng, V, n_contacts)
        else:
            pairs = near_pairs(rng, X, n, n_contacts, 2.0 * h)
        ctrip = contact_blocks(rng, pairs, *k_range)
    else:
        pairs = np.zeros((0, 2), np.int32)
        ctrip = (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros((0, 3, 3)))
    ptr, adj = adjacency_csr(V, tet_edges(tets))
    return _Geometry(n, X, tets, r_e, c_e, b_e, mass, pairs, ctrip, ptr, adj, seed + 7919)


def tet_geometry(n, seed=1000):
    """Rest positions X, deformed positions x, tets and the mesh graph of the n^3
    cube of the recipe above, from the same draws as make_tet_systems (no
    Hessian blocks): the inputs of a device element-Hessian kernel."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (n - 1)
    X, tets = tet_cube(n, rng, jitter=0.05)
    G = rng.uniform(-0.1, 0.1, (3, 3))
    x = X @ (np.eye(3) + G).T + rng.normal(0.0, 0.02 * h, X.shape)
    ptr, adj = adjacency_csr(X.shape[0], tet_edges(tets))
    return X, x, tets.astype(np.int32), ptr, adj


def _system(g, E, params):
    rows = np.concatenate([g.unit_rows, g.mass[0], g.contact_trip[0]]).astype(np.int32)
    cols = np.concatenate([g.unit_cols, g.mass[1], g.contact_trip[1]]).astype(np.int32)
    blocks = np.concatenate([E * g.unit_blocks, g.mass[2], g.contact_trip[2]])
    # shuffle so duplicates are not adjacent (as emitted by a parallel element loop)
    perm = np.random.default_rng(g.shuffle_seed).permutation(rows.size)
    return TetSystem(
        n_grid=g.n,
        X=g.X,
        rows=rows[perm],
        cols=cols[perm],
        blocks=np.ascontiguousarray(blocks[perm]),
        adj_ptr=g.adj_ptr,
        adj=g.adj,
        contacts=g.contacts,
        params=dict(params, E=E),
    )


def make_tet_systems(n, Es, nu=0.4, rho=1000.0, dt=0.01, n_contacts=0,
                     contact_mode="random", k_range=(1e2, 1e6), seed=1000):
    """Systems on one n^3 tet cube that differ only in Young's modulus (list, one per E).

    contact_mode "random" draws distinct uniform vertex pairs; "near" draws
    pairs closer than 2h at rest (which may repeat mesh edges).
    """
    g = _geometry(n, nu, rho, dt, n_contacts, contact_mode, k_range, seed)
    params = dict(n=n, nu=nu, rho=rho, dt=dt, n_contacts=n_contacts,
                  contact_mode=contact_mode, seed=seed)
    return [_system(g, E, params) for E in Es]


def make_tet_system(n, E=1e5, **kw):
    return make_tet_systems(n, [E], **kw)[0]


def rhs(n_dof, nrhs, seed0=2000):
    """nrhs right-hand sides N(0,1), each from seed seed0 + index; shape (nrhs, n_dof)."""
    return np.stack([np.random.default_rng(seed0 + k).normal(size=n_dof) for k in range(nrhs)])


def plain_small(seed=1001):
    """16^3 cube (4,096 verts), E=1e5, 2,000 random contact pairs (2-level MAS, N=32)."""
    return make_tet_system(16, E=1e5, n_contacts=2000, contact_mode="random", seed=seed)


def stiffness_sweep(Es=(1e5, 1e7, 1e9), n=64, seed=1002):
    """n^3 cube (64^3 = 262,144 verts), one system per E, 200k contact pairs within 2h
    (scaled with the vertex count for other n); 3-level MAS, N=32."""
    return make_tet_systems(n, Es, n_contacts=max(1, 200_000 * n ** 3 // 64 ** 3),
                            contact_mode="near", seed=seed)


@dataclass
class Batch:
    """Independent systems concatenated as the diagonal blocks of one matrix."""

    systems: list
    node_off: np.ndarray  # int32 (S + 1,)
    X: np.ndarray
    rows: np.ndarray
    cols: np.ndarray
    blocks: np.ndarray
    adj_ptr: np.ndarray
    adj: np.ndarray
    contacts: np.ndarray

    @property
    def n_vertices(self):
        return int(self.node_off[-1])


def concat_systems(systems):
    off = np.concatenate([[0], np.cumsum([s.n_vertices for s in systems])]).astype(np.int32)
    rows = np.concatenate([s.rows + o for s, o in zip(systems, off)]).astype(np.int32)
    cols = np.concatenate([s.cols + o for s, o in zip(systems, off)]).astype(np.int32)
    blocks = np.concatenate([s.blocks for s in systems])
    eoff = np.concatenate([[0], np.cumsum([s.adj.size for s in systems])])
    adj_ptr = np.concatenate([s.adj_ptr[:-1] + e for s, e in zip(systems, eoff)] + [[eoff[-1]]]).astype(np.int32)
    adj = np.concatenate([s.adj + o for s, o in zip(systems, off)]).astype(np.int32)
    contacts = np.concatenate([s.contacts.reshape(-1, 2) + o for s, o in zip(systems, off)]).astype(np.int32)
    X = np.concatenate([s.X for s in systems])
    return Batch(systems, off, X, rows, cols, blocks, adj_ptr, adj, contacts)


def uneven_batch(n_sys=64, v_range=(1_000, 50_000), e_range=(1e5, 1e9), contact_frac=0.05, seed=1004):
    """n_sys tet cubes with vertex counts log-uniform in v_range (n = round(V^(1/3))),
    E log-uniform in e_range and random contact pairs on contact_frac of the vertices."""
    rng = np.random.default_rng(seed)
    systems = []
    for s in range(n_sys):
        V = np.exp(rng.uniform(np.log(v_range[0]), np.log(v_range[1])))
        n = max(3, int(round(V ** (1.0 / 3.0))))
        E = float(np.exp(rng.uniform(np.log(e_range[0]), np.log(e_range[1]))))
        systems.append(make_tet_system(n, E=E, n_contacts=max(1, int(contact_frac * n ** 3)),
                                       contact_mode="random", seed=seed * 1000 + s))
    return concat_systems(systems)


@dataclass
class ElasticScene:
    """Inputs of one implicit-Euler step of a tet cube (positions, springs,
    graph); the element arithmetic is left to the solver under test."""

    n_grid: int
    X: np.ndarray  # rest positions (V, 3)
    tets: np.ndarray  # int32 (T, 4)
    x: np.ndarray  # deformed start positions (V, 3)
    xt: np.ndarray  # predicted positions x + dt v (V, 3)
    pairs: np.ndarray  # int32 (P, 2) spring vertex pairs
    K: np.ndarray  # (P, 3, 3) k n n^T
    rest: np.ndarray  # (P, 3) rest offsets X_i - X_j
    adj_ptr: np.ndarray
    adj: np.ndarray
    params: dict = field(default_factory=dict)

    @property
    def n_vertices(self):
        return self.X.shape[0]


def make_elastic_scene(n, E=1e5, nu=0.4, rho=1000.0, dt=0.01, n_springs=0, k_range=(1e2, 1e4), omega=1.0,
                       flip=0, seed=3000):
    """n^3 tet cube: rest X jittered N(0, 0.05 h); start x = (I + G) X + N(0, 0.02 h)
    with G_ij ~ U(-0.1, 0.1) (the stiffness-sweep recipe); velocity a rigid
    rotation with angular velocity N(0, omega^2) per axis about the centre, so
    xt = x + dt v; springs: random distinct vertex pairs with K = k n n^T (n
    uniform on the sphere, k log-uniform in k_range) at their rest offsets.
    flip > 0 reflects every flip-th vertex of x through the plane z = centre
    (inverted elements: the projection's hard case)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (n - 1)
    X, tets = tet_cube(n, rng, jitter=0.05)
    G = rng.uniform(-0.1, 0.1, (3, 3))
    x = X @ (np.eye(3) + G).T + rng.normal(0.0, 0.02 * h, X.shape)
    if flip:
        c = x[:, 2].mean()
        x[::flip, 2] = 2 * c - x[::flip, 2]
    w = rng.normal(0.0, omega, 3)
    xt = x + dt * np.cross(w, x - x.mean(axis=0))
    V = X.shape[0]
    if n_springs:
        pairs = random_pairs(rng, V, n_springs)
        nvec = rng.normal(size=(n_springs, 3))
        nvec /= np.linalg.norm(nvec, axis=1, keepdims=True)
        k = np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1]), n_springs))
        K = k[:, None, None] * nvec[:, :, None] * nvec[:, None, :]
        rest = X[pairs[:, 0]] - X[pairs[:, 1]]
    else:
        pairs, K, rest = np.zeros((0, 2), np.int32), np.zeros((0, 3, 3)), np.zeros((0, 3))
    ptr, adj = adjacency_csr(V, tet_edges(tets))
    return ElasticScene(n, X, tets.astype(np.int32), x, xt, pairs.astype(np.int32), K, rest, ptr, adj,
                        dict(n=n, E=E, nu=nu, rho=rho, dt=dt, n_springs=n_springs, seed=seed))
