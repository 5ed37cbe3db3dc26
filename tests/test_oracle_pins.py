"""Pins of the FP64 oracle against closed forms, worked examples, brute force and
dense linear algebra -- never against a retyping of the oracle's own formula."""

import json
import os

import numpy as np
import pytest

from oracle import assembly, mas, partition, pcg
from synth.workloads import make_tet_system, rhs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny_system(n=4, E=1e6, contacts=3, seed=7):
    return make_tet_system(n, E=E, n_contacts=contacts, contact_mode="random", seed=seed)


# ---------------------------------------------------------------- assembly (Sec. 5.2)


def test_hash_key_layout():
    # Sec. 5.2: first index in the high 32 bits, second in the low 32.
    assert int(assembly.hash_key(1, 2)) == (1 << 32) + 2
    assert int(assembly.hash_key(7, 0)) == 7 << 32


def test_assembly_matches_dict_bruteforce():
    rng = np.random.default_rng(0)
    n, K = 9, 400
    rows = rng.integers(0, n, K)
    cols = rng.integers(0, n, K)
    blocks = rng.normal(size=(K, 3, 3))
    r1, c1, a1 = assembly.assemble(rows, cols, blocks)
    r2, c2, a2 = assembly.assemble_dict(rows, cols, blocks)
    assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
    np.testing.assert_allclose(a1, a2, rtol=1e-13, atol=1e-13)
    assert np.all(r1 <= c1)
    k = assembly.hash_key(r1, c1)
    assert np.all(np.diff(k) > 0)  # sorted, unique


def test_assembly_recovers_split_matrix():
    # Split every block of a known upper pattern into random summands
    # (duplicates), add lower-triangle noise that must be ignored, shuffle:
    # the reduction must give back the original blocks.
    rng = np.random.default_rng(1)
    n = 12
    pat = sorted({(min(a, b), max(a, b)) for a, b in rng.integers(0, n, (60, 2))} | {(i, i) for i in range(n)})
    truth = {p: rng.normal(size=(3, 3)) for p in pat}
    rows, cols, blocks = [], [], []
    for (r, c), B in truth.items():
        k = int(rng.integers(1, 6))
        parts = rng.normal(size=(k, 3, 3))
        parts[-1] = B - parts[:-1].sum(0)
        for P in parts:
            rows.append(r), cols.append(c), blocks.append(P)
        if r != c:  # a lower-triangle copy that is ignored
            rows.append(c), cols.append(r), blocks.append(rng.normal(size=(3, 3)))
    perm = rng.permutation(len(rows))
    rid, cid, au = assembly.assemble(np.array(rows)[perm], np.array(cols)[perm], np.array(blocks)[perm])
    assert [(int(a), int(b)) for a, b in zip(rid, cid)] == pat
    for (r, c), B in zip(zip(rid.tolist(), cid.tolist()), au):
        np.testing.assert_allclose(B, truth[(r, c)], atol=1e-12)


def test_head_segmented_reduce_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "head_segmented_reduce.json")))
    out = assembly.head_segmented_reduce(g["values"], g["tags"], width=g["width"])
    assert out == g["output"]
    # A warp boundary always opens a segment (Alg. FastSegmentReduction: LaneId == 0).
    out2 = assembly.head_segmented_reduce([1] * 10, [1] + [0] * 9, width=4)
    assert out2 == [4, None, None, None, 4, None, None, None, 2, None]


def test_abd_two_level_equals_dense_jacobian_product():
    # Sec. 5.1: the reduced Hessian is J^T A J with J = [I, x1 I, x2 I, x3 I]
    # for body nodes and I for FEM nodes; compare with dense matrices.
    rng = np.random.default_rng(2)
    n_full, n_fem, n_bodies = 10, 4, 2
    body = np.array([-1] * n_fem + [0, 0, 0, 1, 1, 1])
    xbar = rng.normal(size=(n_full, 3))
    K = 80
    rows = rng.integers(0, n_full, K)
    cols = rng.integers(0, n_full, K)
    lo = np.minimum(rows, cols)
    hi = np.maximum(rows, cols)
    blocks = rng.normal(size=(K, 3, 3))
    blocks[lo == hi] = blocks[lo == hi] + np.swapaxes(blocks[lo == hi], 1, 2)
    rid, cid, au = assembly.assemble_abd(lo, hi, blocks, body, xbar, n_fem)
    n_red = n_fem + 4 * n_bodies
    got = assembly.to_dense(n_red, rid, cid, au)
    # dense route
    r0, c0, a0 = assembly.assemble_dict(lo, hi, blocks)
    A = assembly.to_dense(n_full, r0, c0, a0)
    J = np.zeros((3 * n_full, 3 * n_red))
    for i in range(n_full):
        if body[i] < 0:
            J[3 * i : 3 * i + 3, 3 * i : 3 * i + 3] = np.eye(3)
        else:
            w = [1.0, *xbar[i]]
            for a in range(4):
                R = n_fem + 4 * body[i] + a
                J[3 * i : 3 * i + 3, 3 * R : 3 * R + 3] = w[a] * np.eye(3)
    np.testing.assert_allclose(got, J.T @ A @ J, rtol=1e-12, atol=1e-12)


def test_abd_body_rows_take_a_bodys_own_hessian_unchanged():
    # Sec. 5.2: a 12 x 12 ABD-ABD block is 16 sub-blocks on the body's reduced
    # rows; given at indices n_full + 4b + a they add to J^T A J as they are.
    rng = np.random.default_rng(12)
    n_full, n_fem, n_bodies = 9, 3, 2
    body = np.array([-1] * n_fem + [0, 0, 0, 1, 1, 1])
    xbar = rng.normal(size=(n_full, 3))
    K = 60
    rows, cols = rng.integers(0, n_full, K), rng.integers(0, n_full, K)
    lo, hi = np.minimum(rows, cols), np.maximum(rows, cols)
    blocks = rng.normal(size=(K, 3, 3))
    H = [rng.normal(size=(12, 12)) for _ in range(n_bodies)]
    H = [h + h.T for h in H]
    br, bc, bb = [], [], []
    for b in range(n_bodies):
        for a in range(4):
            for c in range(a, 4):
                br.append(n_full + 4 * b + a)
                bc.append(n_full + 4 * b + c)
                bb.append(H[b][3 * a : 3 * a + 3, 3 * c : 3 * c + 3])
    rid, cid, au = assembly.assemble_abd(np.concatenate([lo, br]), np.concatenate([hi, bc]),
                                         np.concatenate([blocks, np.array(bb)]), body, xbar, n_fem)
    n_red = n_fem + 4 * n_bodies
    got = assembly.to_dense(n_red, rid, cid, au)
    r1, c1, a1 = assembly.assemble_abd(lo, hi, blocks, body, xbar, n_fem)
    want = assembly.to_dense(n_red, r1, c1, a1)
    for b in range(n_bodies):
        s = 3 * (n_fem + 4 * b)
        want[s : s + 12, s : s + 12] += H[b]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- SpMV (Sec. 5.3)


def test_symmetric_spmv_equals_dense_product():
    s = _tiny_system()
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    V = s.n_vertices
    A = assembly.to_dense(V, rid, cid, au)
    x = np.random.default_rng(3).normal(size=(2, V, 3))
    y = pcg.spmv(rid, cid, au, x)
    for k in range(2):
        np.testing.assert_allclose(y[k].ravel(), A @ x[k].ravel(), rtol=1e-12, atol=1e-9)
    assert np.allclose(A, A.T)


def test_symmetric_matrix_operator_worked_example():
    # Sec. 5.3: a stored off-diagonal block H = A_rc stands for A_rc = H and
    # A_cr = H^T.  One non-symmetric block between rows 0 and 2 of a 3-row
    # matrix, worked by hand: y_0 = H x_2, y_2 = H^T x_0, y_1 = D x_1.
    H = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 9.0]])
    D = np.diag([2.0, 3.0, 5.0])
    x = np.array([1.0, -1.0, 2.0, 0.5, 0.25, -2.0, 3.0, 0.0, -1.0])
    A = pcg.SymmetricMatrix(3, [0, 1], [2, 1], np.stack([H, D]))
    y = A(x)
    want = np.array([1 * 3 + 3 * -1, 4 * 3 + 6 * -1, 7 * 3 + 9 * -1,  # H x_2
                     2 * 0.5, 3 * 0.25, 5 * -2.0,  # D x_1
                     1 * 1 + 4 * -1 + 7 * 2, 2 * 1 + 5 * -1 + 8 * 2, 3 * 1 + 6 * -1 + 9 * 2])  # H^T x_0
    assert np.array_equal(y, want)


@pytest.mark.parametrize("seed", [0, 1])
def test_symmetric_matrix_operator_entrywise(seed):
    # The scipy BSR operator that checks the full-size SpMV and writes the
    # golden iteration counts, against an entry-by-entry dense matrix built
    # from the definition (A[3r+a, 3c+b] = H[a, b], A[3c+b, 3r+a] = H[a, b])
    # and against the loop-based pcg.spmv.  The off-diagonal blocks are not
    # symmetric, so a missing transpose or a swapped index fails; duplicate
    # stored keys are absent by construction (assembly output).
    s = _tiny_system(n=4, contacts=5, seed=seed + 3)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    rng = np.random.default_rng(seed)
    au = au + np.where((rid != cid)[:, None, None], rng.normal(size=au.shape), 0.0)
    V = s.n_vertices
    Ad = np.zeros((3 * V, 3 * V))
    for r, c, H in zip(rid.tolist(), cid.tolist(), au):
        for a in range(3):
            for b in range(3):
                Ad[3 * r + a, 3 * c + b] += H[a, b]
                if r != c:
                    Ad[3 * c + b, 3 * r + a] += H[a, b]
    Aop = pcg.SymmetricMatrix(V, rid, cid, au)
    X = rng.normal(size=(3 * V, 3))
    ref = Ad @ X
    scale = np.abs(Ad) @ np.abs(X)
    assert np.all(np.abs(Aop(X) - ref) <= 1e-12 * scale)  # (3n, k) operand
    for k in range(3):
        assert np.all(np.abs(Aop(X[:, k]) - ref[:, k]) <= 1e-12 * scale[:, k])
        y = pcg.spmv(rid, cid, au, X[:, k].reshape(V, 3)).ravel()
        assert np.all(np.abs(y - ref[:, k]) <= 1e-12 * scale[:, k])
    assert np.array_equal(Aop.A.toarray() != 0, Ad != 0)


# ---------------------------------------------------------------- partition (Sec. 3.2)


def test_partition_hand_worked_grid():
    # 4x4 grid, N = 4.  Extents tie -> x; left = 4*ceil(4/2) = 8 vertices
    # with x in {0, 1}; each half then splits along y: four 2x2 boxes,
    # numbered left to right.
    i, j = np.meshgrid(np.arange(4), np.arange(4), indexing="xy")
    X = np.stack([i.ravel(), j.ravel(), np.zeros(16)], -1).astype(float)  # index = x + 4 y
    part = partition.recursive_bisection(X, 4)
    expect = np.array([0, 0, 2, 2, 0, 0, 2, 2, 1, 1, 3, 3, 1, 1, 3, 3])
    assert np.array_equal(part, expect)
    mp, rm = partition.map_remap(part, 4)
    assert list(rm[:4]) == [0, 1, 4, 5] and list(rm[4:8]) == [8, 9, 12, 13]
    assert np.all(rm[mp] == np.arange(16))


@pytest.mark.parametrize("V,N", [(1, 32), (31, 32), (32, 32), (33, 32), (1000, 16), (4096, 32)])
def test_partition_invariants(V, N):
    X = np.random.default_rng(V).normal(size=(V, 3))
    part = partition.recursive_bisection(X, N)
    sizes = np.bincount(part)
    M = -(-V // N)
    assert part.max() + 1 == M  # Eq. num_subdomains with N_o = 0
    assert np.all(sizes[:-1] == N) and 1 <= sizes[-1] <= N
    mp, rm = partition.map_remap(part, N)
    assert rm.size == N * M
    assert np.array_equal(np.sort(mp), np.sort(np.nonzero(rm >= 0)[0]))
    assert np.all(rm[mp] == np.arange(V))
    assert np.all(mp // N == part)


def test_partition_boxes_are_connected_on_tet_cube():
    s = make_tet_system(16, n_contacts=0, seed=3)
    part = partition.recursive_bisection(s.X, 32)
    V = s.n_vertices
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    A = csr_matrix((np.ones(s.adj.size), s.adj, s.adj_ptr), shape=(V, V))
    ncomp = [connected_components(A[p][:, p])[0] for p in (np.nonzero(part == q)[0] for q in range(part.max() + 1))]
    assert max(ncomp) == 1


def _csr_from_edges(V, edges):
    nb = [[] for _ in range(V)]
    for a, b in edges:
        nb[a].append(b), nb[b].append(a)
    ptr = np.cumsum([0] + [len(x) for x in nb])
    adj = np.array([v for x in nb for v in sorted(x)], dtype=np.int64)
    return ptr, adj


def test_components_by_brute_force_search():
    # numbered by their smallest vertex: {0, 4, 7}, {1, 2}, {3}, {5, 6, 8}
    edges = [(0, 4), (4, 7), (2, 1), (5, 8), (8, 6)]
    ptr, adj = _csr_from_edges(9, edges)
    assert list(partition.components(9, ptr, adj)) == [0, 1, 1, 2, 0, 3, 3, 0, 3]
    # random graphs: same components as a depth-first search from each unseen vertex
    rng = np.random.default_rng(0)
    for V in (1, 17, 60):
        edges = [tuple(e) for e in rng.integers(0, V, (V // 2, 2)) if e[0] != e[1]]
        ptr, adj = _csr_from_edges(V, edges)
        comp = -np.ones(V, dtype=int)
        c = 0
        for s0 in range(V):
            if comp[s0] >= 0:
                continue
            stack = [s0]
            comp[s0] = c
            while stack:
                u = stack.pop()
                for w in adj[ptr[u]:ptr[u + 1]]:
                    if comp[w] < 0:
                        comp[w] = c
                        stack.append(w)
            c += 1
        assert np.array_equal(partition.components(V, ptr, adj), comp)


def test_component_bisection_never_mixes_bodies():
    # two interleaved combs of points on a line: plain bisection mixes them,
    # the component rule bisects each comb on its own, parts numbered comb by comb
    V, N = 40, 4
    X = np.stack([np.arange(V, dtype=float), np.zeros(V), np.zeros(V)], 1)
    edges = [(i, i + 2) for i in range(V - 2)]  # evens and odds: two chains
    ptr, adj = _csr_from_edges(V, edges)
    plain = partition.recursive_bisection(X, N)
    assert any(len(set(np.arange(V)[plain == q] % 2)) > 1 for q in range(plain.max() + 1))
    part = partition.component_bisection(X, N, ptr, adj)
    for q in range(part.max() + 1):
        assert len(set(np.arange(V)[part == q] % 2)) == 1
    # each comb's parts are the plain bisection of that comb alone, shifted
    evens, odds = np.arange(0, V, 2), np.arange(1, V, 2)
    pe = partition.recursive_bisection(X[evens], N)
    po = partition.recursive_bisection(X[odds], N)
    assert np.array_equal(part[evens], pe) and np.array_equal(part[odds], po + pe.max() + 1)
    # a connected mesh: the same as plain bisection
    s = make_tet_system(6, n_contacts=0, seed=2)
    assert np.array_equal(partition.component_bisection(s.X, 16, s.adj_ptr, s.adj),
                          partition.recursive_bisection(s.X, 16))


def test_morton_codes_hand_worked():
    # 2 bits per axis over the unit box: q = min(floor(4 x), 3); bit b of axis a
    # goes to position 3b + a
    X = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.75], [0.25, 0.3, 0.1]], dtype=float)
    X = np.vstack([X, [[1.0, 1.0, 1.0]]])
    codes = partition.morton_codes(X, bits=2)
    assert list(codes[:6]) == [0, 63, 8, 16, 2 ** 2 + 2 ** 5, 1 + 2]
    # a flat axis quantises to 0
    Y = np.array([[0.0, 0.0, 5.0], [1.0, 1.0, 5.0]])
    assert list(partition.morton_codes(Y, bits=1)) == [0, 3]


def test_morton_partition_by_sorting():
    rng = np.random.default_rng(4)
    X = rng.random((203, 3))
    X[10] = X[20]  # a tie: broken by vertex index
    N = 16
    codes = partition.morton_codes(X)
    order = sorted(range(203), key=lambda v: (int(codes[v]), v))
    part = partition.morton_partition(X, N)
    assert [int(part[v]) for v in order] == [i // N for i in range(203)]
    assert part[10] == part[20] or order.index(10) // N != order.index(20) // N


# ---------------------------------------------------------------- MAS levels (supp. Alg. 2-5)


def test_initial_hash_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "initial_hash_mask.json")))
    N = g["domain_size"]
    nodes = [g["node"]] + g["neighbours"]
    slots = [g["node_slot"]] + g["neighbour_slots"]
    item_of_u = np.full(max(nodes) + 1, 0, dtype=np.int64)
    for u, s_ in zip(nodes, slots):
        item_of_u[u] = s_
    # nodes not listed get distinct far slots (outside domain 0)
    unused = [u for u in range(item_of_u.size) if u not in nodes]
    item_of_u[unused] = 1000 + np.arange(len(unused))
    edges = np.array([[g["node"], v] for v in g["neighbours"]])
    masks = mas.in_domain_masks(item_of_u, N, 2000, edges)
    assert int(masks[g["node_slot"]]) == g["mask"]


def _graph_from_edges(V, edges):
    from synth.mesh import adjacency_csr

    return adjacency_csr(V, np.array(edges))


def test_case_study_morton_ordering_gives_three_levels():
    # Sec. 3.1 case study, domain size 4, nodes a..p = 0..15 in Morton order.
    # Level 0: only {b,d} connected in Omega_0; {f,h}, {i,j,k,l}, {m,o},
    # {n,p} merge; b+d is placed before c (lowest order of merged nodes).
    a, b, c, d, e, f, g, h, i, j, k, l, m, n, o, p = range(16)
    edges = [(b, d), (f, h), (i, j), (j, k), (k, l), (m, o), (n, p), (g, i), (c, n), (e, m)]
    ptr, adj = _graph_from_edges(16, edges)
    lv = mas.build_levels(np.arange(16), 4, 8, ptr, adj)
    assert lv.n_items[1] == 9  # a, bd, c | e, fh, g | ijkl | mo, np
    assert list(lv.coarse[1][[a, b, d, c]]) == [0, 1, 1, 2]
    assert lv.n_levels == 3  # the inefficient three-level hierarchy of the text


def test_case_study_connectivity_grouping_gives_two_levels():
    # Sec. 3.1: grouping by connectivity makes every level-0 domain one
    # supernode; level 1 then holds 4 supernodes in 1 domain and stops.
    edges = []
    for q in range(4):
        grp = [4 * q + t for t in range(4)]
        edges += [(u, v) for u in grp for v in grp if u < v]
    edges += [(3, 4), (7, 8), (11, 12), (0, 15)]
    ptr, adj = _graph_from_edges(16, edges)
    lv = mas.build_levels(np.arange(16), 4, 8, ptr, adj)
    assert lv.n_levels == 2 and lv.n_items == [16, 4]
    assert list(lv.coarse[1]) == [0] * 4 + [1] * 4 + [2] * 4 + [3] * 4


def test_contact_pairs_join_supernodes():
    # Alg. 3: a contact pair inside a domain connects its two nodes.
    ptr, adj = _graph_from_edges(8, [(0, 1), (2, 3)])
    lv = mas.build_levels(np.arange(8), 4, 2, ptr, adj)
    assert lv.n_items[1] == 6  # {0,1},{2,3} | 4,5,6,7
    lv2 = mas.build_levels(np.arange(8), 4, 2, ptr, adj, contacts=np.array([[1, 2], [5, 6]]))
    assert lv2.n_items[1] == 4  # {0,1,2,3} | 4,{5,6},7
    assert list(lv2.coarse[1]) == [0, 0, 0, 0, 1, 2, 2, 3]


def _component_invariants(lv, edges):
    N = lv.N
    for l in range(lv.n_levels - 1):
        item = lv.coarse[l]
        nxt_of_fine = lv.coarse[l + 1]
        a = item[edges[:, 0]]
        b = item[edges[:, 1]]
        same_dom = a // N == b // N
        # maximality: adjacent items in one domain share a supernode
        assert np.all(nxt_of_fine[edges[same_dom, 0]] == nxt_of_fine[edges[same_dom, 1]])
        # supernodes never span two domains; ids are domain-major
        dom_of_super = {}
        for u in range(item.size):
            s_ = int(nxt_of_fine[u])
            dom_of_super.setdefault(s_, set()).add(int(item[u]) // N)
        assert all(len(v) == 1 for v in dom_of_super.values())
        doms = [next(iter(dom_of_super[s_])) for s_ in sorted(dom_of_super)]
        assert doms == sorted(doms)
        assert lv.n_items[l + 1] <= int(lv.real[l].sum())


def test_level_invariants_on_tet_cube():
    s = _tiny_system(n=10, contacts=40, seed=11)
    part = partition.recursive_bisection(s.X, 8)
    mp, _ = partition.map_remap(part, 8)
    lv = mas.build_levels(mp, 8, 5, s.adj_ptr, s.adj, s.contacts)
    assert lv.n_levels >= 3
    _component_invariants(lv, mas.fine_edges(s.adj_ptr, s.adj, s.contacts))


# ---------------------------------------------------------------- MAS matrices / apply (Alg. 1, Eq. 4-6)


def _system_and_partition(n=5, N=8, E=1e6, contacts=6, seed=5):
    s = _tiny_system(n=n, E=E, contacts=contacts, seed=seed)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    part = partition.recursive_bisection(s.X, N)
    mp, rm = partition.map_remap(part, N)
    A = assembly.to_dense(s.n_vertices, rid, cid, au)
    return s, rid, cid, au, mp, rm, A


def test_single_domain_preconditioner_is_exact_inverse():
    s, rid, cid, au, mp, rm, A = _system_and_partition(n=4, N=64)
    M = mas.build_mas(mp, 64, 4, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    assert M.levels.n_levels == 1
    r = np.random.default_rng(0).normal(size=3 * s.n_vertices)
    np.testing.assert_allclose(M(r), np.linalg.solve(A, r), rtol=1e-9, atol=1e-12)
    b = rhs(3 * s.n_vertices, 1)
    mv = lambda v: pcg.spmv(rid, cid, au, v.reshape(-1, 3)).ravel()
    _, it, rel = pcg.pcg(mv, lambda v: M(v), b, tol=1e-8)
    assert it[0] == 1 and rel[0] <= 1e-8


def test_one_level_is_block_jacobi():
    # supplement Eq. 4: non-overlapping domains -> block-diagonal preconditioner.
    s, rid, cid, au, mp, rm, A = _system_and_partition()
    N = 8
    M = mas.build_mas(mp, N, 1, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    r = np.random.default_rng(1).normal(size=3 * s.n_vertices)
    z = np.zeros_like(r)
    part = mp // N
    for q in range(part.max() + 1):
        nodes = np.nonzero(part == q)[0]
        idx = (3 * nodes[:, None] + np.arange(3)).ravel()
        z[idx] = np.linalg.solve(A[np.ix_(idx, idx)], r[idx])
    np.testing.assert_allclose(M(r), z, rtol=1e-10, atol=1e-14)


def test_domain_size_one_is_3x3_block_jacobi():
    s, rid, cid, au, mp, rm, A = _system_and_partition()
    part1 = partition.recursive_bisection(s.X, 1)
    mp1, _ = partition.map_remap(part1, 1)
    M = mas.build_mas(mp1, 1, 1, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    r = np.random.default_rng(2).normal(size=(s.n_vertices, 3))
    z = np.stack([np.linalg.solve(A[3 * v : 3 * v + 3, 3 * v : 3 * v + 3], r[v]) for v in range(s.n_vertices)])
    np.testing.assert_allclose(M(r), z, rtol=1e-10, atol=1e-14)


def test_two_node_supernode_block_by_hand():
    # Level-1 block of a supernode {0, 1} is A00 + A01 + A10 + A11 (Alg. 1).
    rng = np.random.default_rng(3)
    B = [rng.normal(size=(3, 3)) for _ in range(4)]
    A00 = B[0] @ B[0].T + 5 * np.eye(3)
    A11 = B[1] @ B[1].T + 5 * np.eye(3)
    A22 = B[2] @ B[2].T + 5 * np.eye(3)
    A01 = 0.3 * B[3]
    rid = np.array([0, 0, 1, 2])
    cid = np.array([0, 1, 1, 2])
    au = np.stack([A00, A01, A11, A22])
    ptr, adj = _graph_from_edges(3, [(0, 1)])
    lv = mas.build_levels(np.array([0, 1, 2]), 2, 2, ptr, adj)
    assert lv.n_items == [4, 2] and list(lv.coarse[1]) == [0, 0, 1]
    mats = mas.level_matrices(lv, rid, cid, au)
    np.testing.assert_allclose(mats[1][0][:3, :3], A00 + A01 + A01.T + A11, atol=1e-14)
    np.testing.assert_allclose(mats[1][0][3:, 3:], A22, atol=1e-14)
    np.testing.assert_allclose(mats[1][0][:3, 3:], 0.0)


def test_level_matrices_equal_galerkin_products():
    # Alg. 1's scatter equals S_d C_l A C_l^T S_d^T computed with dense 0/1 matrices.
    s, rid, cid, au, mp, rm, A = _system_and_partition()
    N = 8
    lv = mas.build_levels(mp, N, 4, s.adj_ptr, s.adj, s.contacts)
    assert lv.n_levels >= 2
    mats = mas.level_matrices(lv, rid, cid, au)
    V = s.n_vertices
    for l in range(lv.n_levels):
        n = lv.n_domains(l) * N
        C = np.zeros((3 * n, 3 * V))
        for u in range(V):
            a = int(lv.coarse[l][u])
            C[3 * a : 3 * a + 3, 3 * u : 3 * u + 3] = np.eye(3)
        G = C @ A @ C.T
        for d in range(lv.n_domains(l)):
            sl = slice(3 * N * d, 3 * N * (d + 1))
            np.testing.assert_allclose(mats[l][d], G[sl, sl], rtol=1e-12, atol=1e-9)


def test_apply_equals_explicit_coarsener_sum_and_is_spd():
    s, rid, cid, au, mp, rm, A = _system_and_partition()
    M = mas.build_mas(mp, 8, 4, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    D = mas.dense_preconditioner(M.levels, M.invs)
    rng = np.random.default_rng(4)
    r1, r2 = rng.normal(size=(2, 3 * s.n_vertices))
    np.testing.assert_allclose(M(r1), D @ r1, rtol=1e-10, atol=1e-14)
    assert abs(r1 @ M(r2) - r2 @ M(r1)) <= 1e-12 * np.linalg.norm(r1) * np.linalg.norm(M(r2))
    w = np.linalg.eigvalsh(0.5 * (D + D.T))
    assert w.min() > 0
    # MAS adds coarse corrections to block-Jacobi: r.M r >= r.M0 r
    M0 = mas.build_mas(mp, 8, 1, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    assert r1 @ M(r1) >= r1 @ M0(r1)


def test_not_spd_domain_is_reported():
    rid = np.array([0, 0, 1])
    cid = np.array([0, 1, 1])
    au = np.stack([np.eye(3), 2 * np.eye(3), np.eye(3)])  # [[I, 2I], [2I, I]] indefinite
    ptr, adj = _graph_from_edges(2, [(0, 1)])
    with pytest.raises(mas.NotSPDError):
        mas.build_mas(np.array([0, 1]), 2, 1, ptr, adj, None, rid, cid, au)


# ---------------------------------------------------------------- PCG (Sec. 3.2)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_pcg_matches_dense_solve(levels):
    s, rid, cid, au, mp, rm, A = _system_and_partition(n=5, N=8, E=1e7)
    M = mas.build_mas(mp, 8, levels, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    b = rhs(3 * s.n_vertices, 2)
    mv = lambda v: pcg.spmv(rid, cid, au, v.reshape(-1, 3)).ravel()
    x, it, rel = pcg.pcg(mv, lambda v: M(v), b, tol=1e-12)
    for k in range(2):
        xs = np.linalg.solve(A, b[k])
        assert np.linalg.norm(x[k] - xs) <= 1e-9 * np.linalg.norm(xs)
        assert np.linalg.norm(b[k] - A @ x[k]) <= 1e-11 * np.linalg.norm(b[k])
        assert rel[k] <= 1e-12 and 1 <= it[k] <= 3 * s.n_vertices


def test_pcg_fixed_iterations_and_zero_rhs():
    s, rid, cid, au, mp, rm, A = _system_and_partition(n=4, N=8)
    M = mas.build_mas(mp, 8, 2, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    mv = lambda v: pcg.spmv(rid, cid, au, v.reshape(-1, 3)).ravel()
    b = np.zeros((2, 3 * s.n_vertices))
    b[1] = rhs(3 * s.n_vertices, 1)[0]
    x, it, rel = pcg.pcg(mv, lambda v: M(v), b, fixed_iters=3)
    assert it[0] == 0 and np.all(x[0] == 0)
    assert it[1] == 3
    # after 3 steps the residual is smaller than at the start
    assert np.linalg.norm(b[1] - A @ x[1]) < np.linalg.norm(b[1])


# ---------------------------------------------------------------- adjoint (gradients through the solve)
def test_adjoint_gradients_match_central_differences():
    from oracle import adjoint

    s = _tiny_system(n=4, E=1e5, contacts=5, seed=9)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    n = s.n_vertices
    rng = np.random.default_rng(10)
    b = rng.normal(size=(2, 3 * n))
    xt = rng.normal(size=(2, 3 * n)) * 1e-3

    def L_of(bb, aa):
        x = adjoint.solve_dense(n, rid, cid, aa, bb)
        return adjoint.loss_and_grad(x, xt)[0]

    x = adjoint.solve_dense(n, rid, cid, au, b)
    _, g = adjoint.loss_and_grad(x, xt)
    lam = adjoint.solve_dense(n, rid, cid, au, g)
    G = adjoint.block_gradients(rid, cid, x, lam)
    # along b
    db = rng.normal(size=b.shape)
    eps = 1e-6 * np.linalg.norm(b) / np.linalg.norm(db)
    fd = (L_of(b + eps * db, au) - L_of(b - eps * db, au)) / (2 * eps)
    assert abs(fd - np.sum(lam * db)) <= 1e-6 * abs(fd)
    # along the stored blocks (each perturbation symmetric through the storage)
    dH = rng.normal(size=au.shape)
    eps = 1e-6 * np.linalg.norm(au) / np.linalg.norm(dH)
    fd = (L_of(b, au + eps * dH) - L_of(b, au - eps * dH)) / (2 * eps)
    assert abs(fd - np.sum(G * dH)) <= 1e-5 * abs(fd)


# ---------------------------------------------------------------- cubic strain-limiting energy (Sec. 4)
def _random_F(rng, stretch):
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    S = np.array([[stretch[0], rng.uniform(-0.05, 0.05)], [0.0, stretch[1]]])
    return Q[:, :2] @ S


@pytest.mark.parametrize("stretch", [(1.08, 0.97), (1.3, 1.2), (0.9, 1.15)])
def test_strain_limit_gradient_and_hessian_by_differences(stretch):
    from oracle import strain_limit as sl

    rng = np.random.default_rng(int(100 * stretch[0]))
    F = _random_F(rng, stretch)
    for n in (sl.N_U, sl.N_V):
        f = F.T.reshape(6)  # vec(F), columns stacked
        E = lambda v: sl.energy(v.reshape(2, 3).T, n)
        G = lambda v: sl.gradient(v.reshape(2, 3).T, n)
        h = 1e-6
        g_fd = np.array([(E(f + h * e) - E(f - h * e)) / (2 * h) for e in np.eye(6)])
        np.testing.assert_allclose(sl.gradient(F, n), g_fd, rtol=1e-6, atol=1e-9)
        H_fd = np.stack([(G(f + h * e) - G(f - h * e)) / (2 * h) for e in np.eye(6)], 1)
        np.testing.assert_allclose(sl.hessian(F, n), H_fd, rtol=1e-5, atol=1e-7)


def test_strain_limit_eigensystem_closed_forms():
    from oracle import strain_limit as sl

    rng = np.random.default_rng(5)
    for _ in range(20):
        F = _random_F(rng, rng.uniform(1.01, 1.5, 2))
        for n in (sl.N_U, sl.N_V):
            w = np.sort(np.linalg.eigvalsh(sl.hessian(F, n)))
            e1, e2, e3 = sl.eigenvalues(F, n)
            # the direction-n block has e1, e2, e3; the other direction's block is zero
            np.testing.assert_allclose(w[-3:], np.sort([e1, e2, e3]), rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(w[:3], 0.0, atol=1e-12)
            assert min(e1, e2) > 0  # convex when stretched


def test_strain_limit_is_c2_at_the_limit():
    from oracle import strain_limit as sl

    F = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    for eps in (1e-3, 1e-5):
        Fe = F * (1.0 + eps)
        assert sl.energy(Fe, sl.N_U) < 2 * eps ** 3
        assert np.abs(sl.gradient(Fe, sl.N_U)).max() < 4 * eps ** 2
        assert np.abs(sl.hessian(Fe, sl.N_U)).max() < 20 * eps
    assert sl.energy(F * 0.9, sl.N_U) == 0.0 and not sl.hessian(F * 0.9, sl.N_U).any()


def test_inverse_factors_reproduce_the_inverses():
    # M_d^{-1} = W^T W with W = L^{-1} lower triangular (the BF16 storage form)
    s = _tiny_system(n=5, E=1e6, contacts=6, seed=21)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    part = partition.recursive_bisection(s.X, 8)
    mp, _ = partition.map_remap(part, 8)
    lv = mas.build_levels(mp, 8, 3, s.adj_ptr, s.adj, s.contacts)
    mats = mas.level_matrices(lv, rid, cid, au)
    invs = mas.invert_domains(lv, mats)
    facs = mas.inverse_factors(lv, mats)
    for l, (inv, fac) in enumerate(zip(invs, facs)):
        for d in range(inv.shape[0]):
            assert np.allclose(np.triu(fac[d], 1), 0.0)
            np.testing.assert_allclose(fac[d].T @ fac[d], inv[d], rtol=1e-10, atol=1e-12 * np.abs(inv[d]).max())
            # W M_d W^T = I on the real part (and 0 on the padding)
            real = np.any(fac[d] != 0, axis=1)
            if not real.any():
                continue
            WMW = fac[d] @ mats[l][d] @ fac[d].T
            np.testing.assert_allclose(WMW[np.ix_(real, real)], np.eye(real.sum()), atol=1e-9)


# ---------------------------------------------------------------- element Hessians (Sec. 3.1)
from oracle import elastic  # noqa: E402


def _deformed_tets(seed=0, T=5):
    rng = np.random.default_rng(seed)
    X = rng.random((4 * T, 3))
    tets = np.arange(4 * T).reshape(T, 4)
    # keep positive orientation
    for t in range(T):
        a, b, c, d = X[tets[t]]
        if np.linalg.det(np.stack([b - a, c - a, d - a], 1)) < 0:
            tets[t, [1, 2]] = tets[t, [2, 1]]
    x = X @ (np.eye(3) + 0.3 * rng.normal(size=(3, 3))).T + 0.05 * rng.normal(size=X.shape)
    return X, x, tets


def test_snh_gradient_and_hessian_by_central_differences():
    X, x, tets = _deformed_tets()
    E, nu = 1e6, 0.4
    e0, g = elastic.energy_and_gradient(X, x, tets, E, nu)
    h = 1e-6
    gd = np.zeros_like(x)
    for v in range(x.shape[0]):
        for i in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, i] += h
            xm[v, i] -= h
            gd[v, i] = (elastic.energy_and_gradient(X, xp, tets, E, nu)[0] -
                        elastic.energy_and_gradient(X, xm, tets, E, nu)[0]) / (2 * h)
    assert np.abs(gd - g).max() <= 1e-6 * np.abs(g).max()
    # the unprojected element Hessian is the derivative of the gradient
    He = elastic.element_hessians(X, x, tets, E, nu, project=False)
    for t in range(tets.shape[0]):
        Hd = np.zeros((12, 12))
        for a in range(4):
            for i in range(3):
                xp, xm = x.copy(), x.copy()
                xp[tets[t, a], i] += h
                xm[tets[t, a], i] -= h
                dg = (elastic.energy_and_gradient(X, xp, tets[t:t + 1], E, nu)[1] -
                      elastic.energy_and_gradient(X, xm, tets[t:t + 1], E, nu)[1]) / (2 * h)
                Hd[:, 3 * a + i] = dg[tets[t]].reshape(-1)
        assert np.abs(Hd - He[t]).max() <= 1e-5 * np.abs(He[t]).max()


def test_snh_rest_state_rotation_invariance_and_projection():
    mu, lam = elastic.lame(1e6, 0.4)
    _, g, _ = elastic.snh(np.eye(3), mu, lam)
    assert np.abs(g).max() <= 1e-9 * mu  # the rest state is stationary
    rng = np.random.default_rng(1)
    F = np.eye(3) + 0.4 * rng.normal(size=(3, 3))
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Q *= np.sign(np.linalg.det(Q))
    assert abs(elastic.snh(Q @ F, mu, lam)[0] - elastic.snh(F, mu, lam)[0]) <= 1e-9 * mu
    # projection: PSD output, identity on PSD input
    _, _, H = elastic.snh(np.diag([1.8, 0.3, 0.4]), mu, lam)
    assert np.linalg.eigvalsh(H).min() < 0  # a compressed state with a negative mode
    P = elastic.psd_project(H)
    assert np.linalg.eigvalsh(P).min() >= -1e-9 * np.abs(H).max()
    S = H @ H.T
    np.testing.assert_allclose(elastic.psd_project(S), S, rtol=0, atol=1e-9 * np.abs(S).max())


def test_system_triplets_assemble_the_scattered_element_hessians():
    from synth.mesh import tet_cube

    rng = np.random.default_rng(2)
    X, tets = tet_cube(3, rng)
    x = X + 0.05 * rng.normal(size=X.shape)
    E, nu, rho, dt = 1e5, 0.4, 1000.0, 0.01
    rows, cols, blocks = elastic.system_triplets(X, x, tets, E, nu, rho, dt)
    assert np.all(rows <= cols)
    rid, cid, au = assembly.assemble(rows, cols, blocks)
    V = X.shape[0]
    A = assembly.to_dense(V, rid, cid, au)
    # brute force: every element's 12 x 12 Hessian added at its nodes, plus the masses
    He = elastic.element_hessians(X, x, tets, E, nu)
    D = np.zeros_like(A)
    for t, tet in enumerate(tets):
        idx = (3 * np.asarray(tet)[:, None] + np.arange(3)).ravel()
        D[np.ix_(idx, idx)] += He[t]
    D += np.kron(np.diag(elastic.lumped_mass(X, tets, rho) / dt ** 2), np.eye(3))
    np.testing.assert_allclose(A, D, rtol=0, atol=1e-10 * np.abs(D).max())
    assert np.linalg.eigvalsh(A).min() > 0


# ---------------------------------------------------------------- Newton loop on the incremental potential
def _newton_case(n=3, seed=5, n_springs=6):
    from synth.mesh import tet_cube

    rng = np.random.default_rng(seed)
    X, tets = tet_cube(n, rng)
    V = X.shape[0]
    xt = X + 0.02 * rng.normal(size=X.shape)  # predicted positions
    pairs = rng.choice(V, size=(n_springs, 2), replace=False) if n_springs else np.zeros((0, 2), np.int64)
    nrm = rng.normal(size=(n_springs, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    K = 1e3 * nrm[:, :, None] * nrm[:, None, :]
    rest = 0.9 * (X[pairs[:, 0]] - X[pairs[:, 1]]) if n_springs else np.zeros((0, 3))
    return X, tets, xt, (pairs, K, rest)


def test_incremental_potential_gradient_by_central_differences():
    from oracle import newton

    X, tets, xt, springs = _newton_case()
    rng = np.random.default_rng(1)
    x = X + 0.05 * rng.normal(size=X.shape)
    args = (tets, 1e4, 0.3, 1000.0, 0.01, xt, springs)
    _, g = newton.incremental_potential(X, x, *args)
    h = 1e-6
    for _ in range(12):
        v, c = rng.integers(X.shape[0]), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[v, c] += h
        xm[v, c] -= h
        fd = (newton.incremental_potential(X, xp, *args)[0] - newton.incremental_potential(X, xm, *args)[0]) / (2 * h)
        assert abs(fd - g[v, c]) <= 1e-6 * max(1.0, abs(g).max())


def test_spring_hessian_is_the_exact_derivative_of_the_spring_gradient():
    from oracle import assembly, newton

    X, _, _, springs = _newton_case(n_springs=8)
    V = X.shape[0]
    rng = np.random.default_rng(2)
    x = X + 0.1 * rng.normal(size=X.shape)
    _, g0, (r, c, b) = newton.spring_terms(x, springs)
    A = assembly.to_dense(V, *assembly.assemble(r, c, b))
    dx = rng.normal(size=X.shape)
    _, g1, _ = newton.spring_terms(x + dx, springs)
    # the springs are quadratic: the gradient changes by exactly H dx
    assert np.allclose((g1 - g0).ravel(), A @ dx.ravel(), rtol=0, atol=1e-9 * abs(A).max())


def test_newton_stops_at_once_at_the_rest_state():
    from oracle import newton

    X, tets, _, (pairs, K, _) = _newton_case()
    rest = X[pairs[:, 0]] - X[pairs[:, 1]]  # springs at rest too
    x, hist = newton.newton(X, X, tets, 1e5, 0.4, 1000.0, 0.01, X, (pairs, K, rest))
    assert len(hist) == 1 and hist[0]["converged"] and hist[0]["dinf"] < 1e-12
    assert np.array_equal(x, X)


def test_newton_reaches_the_minimiser_found_by_a_derivative_free_method():
    import scipy.optimize as so

    from oracle import newton

    X, tets, xt, springs = _newton_case(n=2, seed=8, n_springs=3)
    args = (tets, 1e4, 0.3, 1000.0, 0.01, xt, springs)
    rng = np.random.default_rng(3)
    x0 = X + 0.03 * rng.normal(size=X.shape)
    x, hist = newton.newton(X, x0, *args, tol=1e-9)
    assert hist[-1]["converged"]
    energies = [h["energy"] for h in hist]
    assert all(b < a for a, b in zip(energies, energies[1:]))
    # Powell (no derivatives) on the energy alone, from the same start
    f = lambda z: newton.incremental_potential(X, z.reshape(-1, 3), *args)[0]
    res = so.minimize(f, x0.ravel(), method="Powell", options=dict(xtol=1e-12, ftol=1e-15, maxiter=200000))
    assert np.abs(res.x.reshape(-1, 3) - x).max() <= 1e-5
    assert f(x.ravel()) <= res.fun + 1e-9 * abs(res.fun)
