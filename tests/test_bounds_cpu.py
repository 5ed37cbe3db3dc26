"""The per-entry FP64 apply bound of tests/fp64bounds.py, on the CPU: it holds
between two FP64 evaluations of the same preconditioner that sum in different
orders, and it fails for the mistakes it is there to catch (one node moved to
another coarse item, one domain inverse perturbed)."""

import numpy as np

import fp64bounds
from oracle import assembly, mas, partition
from synth.workloads import make_tet_system


def _setup():
    s = make_tet_system(8, E=1e8, n_contacts=30, contact_mode="random", seed=4)
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    mp, _ = partition.map_remap(partition.recursive_bisection(s.X, 8), 8)
    om = mas.build_mas(mp, 8, 3, s.adj_ptr, s.adj, s.contacts, rid, cid, au)
    r = np.random.default_rng(5).normal(size=(3, 3 * s.n_vertices))
    return s, om, r


def test_bound_holds_between_two_evaluation_orders():
    s, om, r = _setup()
    assert om.levels.n_levels == 3
    z = om(r)
    Minv = mas.dense_preconditioner(om.levels, om.invs)
    z2 = (Minv @ r.T).T  # the same operator, summed as one dense product
    bound = fp64bounds.apply_bound(om, r)
    assert np.all(np.abs(z - z2) <= bound)
    # and the bound is far below the entries it guards
    assert np.median(bound / np.abs(z)) < 1e-6


def test_bound_catches_a_moved_node():
    s, om, r = _setup()
    lv = om.levels
    # move one node to another level-1 item of the same level-1 domain
    c1 = lv.coarse[1].copy()
    u = int(np.nonzero(np.bincount(c1) > 1)[0][0])  # an item with several nodes
    node = int(np.nonzero(c1 == u)[0][0])
    dom = u // lv.N
    other = next(a for a in range(dom * lv.N, dom * lv.N + lv.N) if a != u and a < lv.n_items[1])
    C = list(om.C)
    c1[node] = other
    C[1] = mas.coarsener(mas.Levels(**{**lv.__dict__, "coarse": [lv.coarse[0], c1] + list(lv.coarse[2:])}), 1)
    zbad = mas.apply(lv, om.invs, r, C)
    assert np.any(np.abs(zbad - om(r)) > fp64bounds.apply_bound(om, r))


def test_bound_catches_a_perturbed_domain_inverse():
    s, om, r = _setup()
    invs = [v.copy() for v in om.invs]
    invs[0][3] *= 1 + 1e-5  # one level-0 domain off by 1e-5 relative
    zbad = mas.apply(om.levels, invs, r, om.C)
    assert np.any(np.abs(zbad - om(r)) > fp64bounds.apply_bound(om, r))
