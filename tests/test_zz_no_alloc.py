"""gs_mas_apply_noalloc: the MAS apply with its coarse-level scratch in a fixed
array compiled into the library, for callers that may not allocate device
memory once they run (a fixed device-memory budget handed over at start-up,
or code that must never stall or fail on a cudaMalloc).

Its output must match gs_mas_apply's, on two calls in a row (the array keeps
the previous call's contents, so the second call checks that the restricted
vectors are cleared), for every product path the apply can take: the FP64
products on the tensor cores (the default) or on the FP64 cores (tuned off,
or more than 8 right-hand sides), and the FP32 and BF16 preconditioners.  The
library's own allocation counter must not move across the calls.  Sizes
beyond the fixed array are refused, and a bounded-wait timeout of the
tensor-core product is reported by the call that raised it.
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


def _setup(B, ctx, n, N, L, precision=0):
    s = make_tet_system(n, E=1e7, n_contacts=60, contact_mode="random", seed=21)
    V = s.n_vertices
    mat = B.gs_assemble(ctx, V, _dev(s.rows, torch.int32), _dev(s.cols, torch.int32), _dev(s.blocks, torch.float64))
    mp, nd = B.gs_partition(s.X, N)
    mas = B.gs_build_mas(ctx, mat, _dev(mp, torch.int32), nd, _dev(s.adj_ptr, torch.int32), _dev(s.adj, torch.int32),
                         _dev(s.contacts, torch.int32), domain_size=N, max_levels=L, precision=precision)
    return V, mat, mas


def _noalloc(B, ctx, mas, r, z, nrhs):
    st = B.lib().gs_mas_apply_noalloc(ctx, mas, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), nrhs)
    return st


# (precision, GS_TUNE_F64_TC, right-hand sides, relative tolerance): FP64
# products agree to the FP64 apply's own tolerance; the FP32 and BF16 forms
# to a few FP32 roundings (their coarse levels read restricted vectors whose
# atomic sums may round differently from call to call).
_PATHS = [
    (0, 3, 4, 1e-12),   # FP64 accuracy on the tensor cores from symmetric digit bytes, every level
    (0, 1, 4, 1e-12),   # FP64 accuracy on the tensor cores from BF16 digit matrices, every level
    (0, 4, 8, 1e-12),   # the same with 256-thread CTAs at level 0
    (0, 0, 4, 1e-12),   # FP64 cores
    (0, 1, 12, 1e-12),  # more than 8 RHS: FP64 cores
    (1, 1, 4, 1e-5),    # FP32 inverses
    (2, 1, 4, 1e-5),    # BF16 factors on the tensor cores
    (2, 1, 12, 1e-5),   # BF16 factors on the FP32 cores
]


@pytest.mark.parametrize("prec,f64tc,nrhs,tol", _PATHS)
def test_noalloc_apply_matches_apply_twice(B, prec, f64tc, nrhs, tol):
    ctx = B.gs_create(0)
    try:
        B.gs_tune_set(ctx, B.GS_TUNE_F64_TC, f64tc)
        V, mat, mas = _setup(B, ctx, 12, 16, 3, precision=prec)
        assert B.gs_mas_info(mas)[0] == 3
        for k, seed in ((nrhs, 1), (max(nrhs // 2, 1), 2)):
            r = _dev(np.random.default_rng(seed).normal(size=(k, 3 * V)), torch.float64)
            ref = torch.empty_like(r)
            B.gs_mas_apply(ctx, mas, r, ref, nrhs=k)
            torch.cuda.synchronize()
            before = B.gs_ctx_alloc_stats(ctx)
            for _ in range(2):
                z = torch.full_like(r, np.nan)
                assert _noalloc(B, ctx, mas, r, z, k) == B.GS_OK, B.lib().gs_last_error()
                torch.cuda.synchronize()
                err = ((z - ref).abs().amax(dim=1) / ref.abs().amax(dim=1)).max().item()
                assert err <= tol, err
            assert B.gs_ctx_alloc_stats(ctx) == before
        B.gs_mas_destroy(mas)
        B.gs_mat_destroy(mat)
    finally:
        B.gs_destroy(ctx)


def test_noalloc_apply_reports_its_own_timeout(B):
    # A kernel whose bounded wait gave up leaves a bit in the context's device
    # error word.  The test sets that bit from the host (no kernel is made to
    # wait) and checks that the call reports it and clears it, so the next
    # call succeeds and matches the allocating apply.
    ctx = B.gs_create(0)
    try:
        V, mat, mas = _setup(B, ctx, 12, 16, 3)
        nrhs = 4
        r = _dev(np.random.default_rng(3).normal(size=(nrhs, 3 * V)), torch.float64)
        ref = torch.empty_like(r)
        B.gs_mas_apply(ctx, mas, r, ref, nrhs=nrhs)
        z = torch.empty_like(r)
        B.gs_debug_raise_flags(ctx, 8)
        assert _noalloc(B, ctx, mas, r, z, nrhs) == B.GS_ERR_TIMEOUT
        z.fill_(np.nan)
        assert _noalloc(B, ctx, mas, r, z, nrhs) == B.GS_OK
        torch.cuda.synchronize()
        assert ((z - ref).abs().amax() / ref.abs().amax()).item() <= 1e-12
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
