"""gs_mas_apply_noalloc: the MAS apply with its coarse-level scratch in a fixed
array compiled into the library, for callers that may not allocate device
memory once they run (a fixed device-memory budget handed over at start-up,
or code that must never stall or fail on a cudaMalloc).

Its output must match gs_mas_apply's, on two calls in a row (the array keeps
the previous call's contents, so the second call checks that the restricted
vectors are cleared).  Sizes beyond the fixed array are refused.
"""

import ctypes

import numpy as np
import pytest
import torch

from synth.workloads import make_tet_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2411_06224_gb300.build import build

    build()
    from paper_2411_06224_gb300 import binding

    return binding


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def _setup(B, ctx, n, N, L):
    s = make_tet_system(n, E=1e7, n_contacts=60, contact_mode="random", seed=21)
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, _dev(s.rows, torch.int32), _dev(s.cols, torch.int32), _dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, N)
    mas = B.gs_build_mas(ctx, mat, _dev(mp, torch.int32), nd, _dev(s.adj_ptr, torch.int32), _dev(s.adj, torch.int32),
                         _dev(s.contacts, torch.int32), domain_size=N, max_levels=L)
    return V, mat, mas


def _noalloc(B, ctx, mas, r, z, nrhs):
    st = B.lib().gs_mas_apply_noalloc(ctx, mas, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), nrhs)
    return st


def test_noalloc_apply_matches_apply_twice(B):
    ctx = B.gs_create(0)
    try:
        V, mat, mas = _setup(B, ctx, 12, 16, 3)
        assert B.gs_mas_info(mas)[0] == 3
        for nrhs, seed in ((4, 1), (2, 2)):
            r = _dev(np.random.default_rng(seed).normal(size=(nrhs, 3 * V)), torch.float64)
            ref = torch.empty_like(r)
            B.gs_mas_apply(ctx, mas, r, ref, nrhs=nrhs)
            for _ in range(2):
                z = torch.full_like(r, np.nan)
                assert _noalloc(B, ctx, mas, r, z, nrhs) == B.GS_OK
                torch.cuda.synchronize()
                err = ((z - ref).norm(dim=1) / ref.norm(dim=1)).max().item()
                assert err <= 1e-12, err
        B.gs_mas_destroy(mas)
        B.gs_mat_destroy(mat)
    finally:
        B.gs_destroy(ctx)


def test_noalloc_apply_refuses_oversized_scratch(B):
    ctx = B.gs_create(0)
    try:
        # 2-node domains: level 1 alone has ~6.9k items, so 16 RHS need more than the fixed array
        V, mat, mas = _setup(B, ctx, 24, 2, 6)
        nrhs = 16
        r = torch.zeros((nrhs, 3 * V), dtype=torch.float64, device="cuda")
        z = torch.zeros_like(r)
        st = _noalloc(B, ctx, mas, r, z, nrhs)
        assert st == B.GS_ERR_INVALID
        assert "above the fixed" in B.lib().gs_last_error().decode()
        B.gs_mas_destroy(mas)
        B.gs_mat_destroy(mat)
    finally:
        B.gs_destroy(ctx)
