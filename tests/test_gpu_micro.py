"""Microbenchmark entry points give correct results: the FastHashReduction and
the library reduce-by-key both equal the per-key sums of the oracle's
definition; the library BSR SpMV on the full matrix equals the oracle SpMV."""

import numpy as np
import pytest
import torch

from oracle import assembly, pcg
from synth.workloads import make_tet_system

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


@pytest.mark.parametrize("dup", [1, 3, 40, 1000])
@pytest.mark.parametrize("method", [0, 1])
def test_segment_reduce_methods(B, ctx, dup, method):
    rng = np.random.default_rng(dup)
    nb = 50_000
    runs = rng.integers(1, 2 * dup, nb)  # run lengths around dup, ragged
    keys = np.repeat(np.cumsum(rng.integers(1, 5, runs.size)), runs)[:nb].astype(np.int64)
    blocks = rng.normal(size=(nb, 3, 3))
    out, ms = B.gs_micro_segment_reduce(ctx, torch.as_tensor(keys, device="cuda"),
                                        torch.as_tensor(blocks, device="cuda"), method)
    starts = np.flatnonzero(np.r_[True, keys[1:] != keys[:-1]])
    ref = np.add.reduceat(blocks, starts, axis=0)
    bound = 1e-13 * np.add.reduceat(np.abs(blocks), starts, axis=0)
    got = out.cpu().numpy()
    assert got.shape == ref.shape and np.all(np.abs(got - ref) <= bound + 1e-300)
    assert ms > 0


def test_full_bsr_library_spmv(B, ctx):
    s = make_tet_system(7, E=1e6, n_contacts=30, seed=4)
    V = s.n_vertices
    rid, cid, au = assembly.assemble(s.rows, s.cols, s.blocks)
    off = rid != cid
    r = np.concatenate([rid, cid[off]])
    c = np.concatenate([cid, rid[off]])
    a = np.concatenate([au, np.swapaxes(au[off], 1, 2)])
    o = np.lexsort((c, r))
    r, c, a = r[o], c[o], a[o]
    ptr = np.concatenate([[0], np.cumsum(np.bincount(r, minlength=V))]).astype(np.int32)
    x = np.random.default_rng(1).normal(size=(V, 3))
    y = torch.empty(3 * V, dtype=torch.float64, device="cuda")
    ms = B.gs_micro_bsr_spmv_cusparse(ctx, V, torch.as_tensor(ptr, device="cuda"),
                                      torch.as_tensor(c.astype(np.int32), device="cuda"),
                                      torch.as_tensor(np.ascontiguousarray(a), device="cuda"),
                                      torch.as_tensor(x.reshape(-1), device="cuda"), y, reps=3)
    y0 = pcg.spmv(rid, cid, au, x[None])[0].reshape(-1)
    bound = 1e-13 * pcg.spmv(rid, cid, np.abs(au), np.abs(x)[None])[0].reshape(-1)
    assert np.all(np.abs(y.cpu().numpy() - y0) <= bound) and ms > 0
