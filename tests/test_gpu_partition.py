"""Level-0 partition on the device (Sec. 3.2, Eq. num_subdomains; supplement
Algorithm 1): every rule bit for bit against the oracle's, on meshes, point
clouds with tied coordinates, bodies interleaved in space and the edge sizes
(fewer nodes than a domain, exactly one domain, one node per domain)."""

import numpy as np
import pytest
import torch

from oracle import partition
from synth.workloads import make_tet_system, uneven_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2411_06224_gb300.build import build

    build()
    from paper_2411_06224_gb300 import binding

    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.gs_create(0)
    yield c
    B.gs_destroy(c)


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def oracle_map(X, N, rule, adj_ptr=None, adj=None):
    if rule == 0:
        part = partition.recursive_bisection(X, N)
    elif rule == 1:
        part = partition.component_bisection(X, N, adj_ptr, adj)
    else:
        part = partition.morton_partition(X, N)
    mp, _ = partition.map_remap(part, N)
    return mp, int(part.max()) + 1


def check(B, ctx, X, N, rule, adj_ptr=None, adj=None):
    mp, nd = B.gs_partition_device(ctx, dev(X, torch.float64), N, rule,
                                   None if adj_ptr is None else dev(adj_ptr, torch.int32),
                                   None if adj is None else dev(adj, torch.int32))
    mo, ndo = oracle_map(X, N, rule, adj_ptr, adj)
    assert nd == ndo
    assert np.array_equal(mp.cpu().numpy(), mo)
    return mp.cpu().numpy(), nd


_MESH = {}


def mesh(n):
    if n not in _MESH:
        _MESH[n] = make_tet_system(n, E=1e6, n_contacts=0, seed=30 + n)
    return _MESH[n]


@pytest.mark.parametrize("rule", [0, 1, 2])
@pytest.mark.parametrize("n,N", [(11, 32), (11, 16), (13, 7), (4, 32), (6, 1)])
def test_device_partition_matches_oracle_on_meshes(B, ctx, rule, n, N):
    s = mesh(n)
    check(B, ctx, s.X, N, rule, s.adj_ptr, s.adj)
    if rule == 0:  # and the host partition
        mh, ndh = B.gs_partition(s.X, N)
        md, ndd = B.gs_partition_device(ctx, dev(s.X, torch.float64), N, 0)
        assert ndd == ndh and np.array_equal(md.cpu().numpy(), mh)


@pytest.mark.parametrize("rule", [0, 2])
def test_device_partition_ties_signed_zeros_and_small_sizes(B, ctx, rule):
    rng = np.random.default_rng(7)
    X = np.round(rng.random((700, 3)) * 4) / 4  # many equal coordinates: ties by index
    X[::5, 1] = -0.0
    X[1::5, 1] = 0.0
    for N in (32, 5):
        check(B, ctx, X, N, rule)
    for V in (1, 31, 32, 33):  # fewer nodes than a domain, exactly one, one more
        check(B, ctx, X[:V], 32, rule)
    check(B, ctx, np.zeros((40, 3)), 8, rule)  # every coordinate equal, flat box


def test_component_rule_separates_interleaved_bodies(B, ctx):
    # 64 cubes in the same unit box: plain bisection mixes their nodes in one
    # part, the component rule never does, and matches the oracle bit for bit
    bt = uneven_batch(12, seed=9)
    X, ptr, adj = bt.X, bt.adj_ptr, bt.adj
    mp, nd = check(B, ctx, X, 32, 1, ptr, adj)
    body = np.searchsorted(bt.node_off, np.arange(X.shape[0]), side="right") - 1
    part = mp // 32
    assert all(len(set(body[part == q])) == 1 for q in range(nd))
    mp0, nd0 = check(B, ctx, X, 32, 0)
    part0 = mp0 // 32
    assert any(len(set(body[part0 == q])) > 1 for q in range(nd0))


def test_mas_from_the_mesh_equals_mas_from_the_map(B, ctx):
    s = make_tet_system(9, E=1e6, n_contacts=30, contact_mode="random", seed=3)
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, dev(s.rows, torch.int32), dev(s.cols, torch.int32), dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, 16)
    args = (dev(s.adj_ptr, torch.int32), dev(s.adj, torch.int32), dev(s.contacts, torch.int32))
    m1 = B.gs_build_mas(ctx, mat, dev(mp, torch.int32), nd, *args, domain_size=16, max_levels=3)
    m2 = B.gs_build_mas_mesh(ctx, mat, dev(s.X, torch.float64), *args, domain_size=16, max_levels=3)
    nl, items = B.gs_mas_info(m1)
    assert (nl, items) == B.gs_mas_info(m2)
    for l in range(nl):  # the same levels, bit for bit
        assert torch.equal(B.gs_mas_export_coarse(ctx, m1, l, V), B.gs_mas_export_coarse(ctx, m2, l, V))
    r = dev(np.random.default_rng(0).normal(size=(2, 3 * V)), torch.float64)
    z1, z2 = torch.empty_like(r), torch.empty_like(r)
    B.gs_mas_apply(ctx, m1, r, z1, nrhs=2)
    B.gs_mas_apply(ctx, m2, r, z2, nrhs=2)
    # the coarse level matrices sum cross-domain blocks with atomics: equal up to rounding
    assert ((z1 - z2).abs().amax() / z1.abs().amax()).item() <= 1e-12
    B.gs_mas_destroy(m1)
    B.gs_mas_destroy(m2)
    B.gs_mat_destroy(mat)
