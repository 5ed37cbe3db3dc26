"""The hash assembly's hand-written primitives through the C ABI: the stable
LSD radix sort of (key, index) pairs against numpy's stable argsort, and the
exclusive scan against a cumulative sum, bit for bit, over sizes that span
one tile, several tiles and ragged tails, key widths of one to eight digits
and heavy duplication."""

import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("n", [1, 31, 2047, 2048, 2049, 100_003, 3_000_001])
@pytest.mark.parametrize("end_bit,distinct", [(8, 200), (20, 5000), (38, 1 << 30), (64, None)])
def test_sort_pairs_is_the_stable_sort(B, ctx, n, end_bit, distinct):
    rng = np.random.default_rng(n + end_bit)
    if distinct is None:  # full 64-bit keys, high bit set on half
        keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64) | (rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63))
    else:  # at most `distinct` values below 2^end_bit: many duplicates
        pool = rng.integers(0, 2 ** end_bit, min(distinct, 2 ** end_bit), dtype=np.uint64)
        keys = pool[rng.integers(0, pool.size, n)]
    # bits above end_bit are ignored by the sort: set some to check it
    if end_bit < 64:
        keys = keys | (rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(end_bit))
    vals = np.arange(n, dtype=np.int32)
    kd = torch.as_tensor(keys.view(np.int64), device="cuda")
    vd = torch.as_tensor(vals, device="cuda")
    ko, vo = B.gs_prim_sort_pairs(ctx, kd, vd, end_bit)
    order = np.argsort(keys & np.uint64((1 << end_bit) - 1) if end_bit < 64 else keys, kind="stable")
    assert np.array_equal(vo.cpu().numpy(), vals[order])
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(kd.cpu().numpy().view(np.uint64), keys)  # inputs untouched


def test_sort_rejects_bad_arguments(B, ctx):
    kd = torch.zeros(10, dtype=torch.int64, device="cuda")
    vd = torch.zeros(10, dtype=torch.int32, device="cuda")
    for eb in (0, 65):
        with pytest.raises(B.GsError):
            B.gs_prim_sort_pairs(ctx, kd, vd, eb)
    st = B.lib().gs_prim_sort_pairs(ctx, kd.data_ptr(), vd.data_ptr(), kd.data_ptr(), vd.data_ptr(), 10, 8)
    assert st == B.GS_ERR_INVALID  # in place


@pytest.mark.parametrize("n", [1, 4095, 4096, 4097, 1_000_003, 20_000_000])
def test_exclusive_scan(B, ctx, n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 3, n).astype(np.int32)
    xd = torch.as_tensor(x, device="cuda")
    out = B.gs_prim_exclusive_scan(ctx, xd)
    ref = np.concatenate([[0], np.cumsum(x, dtype=np.int64)[:-1]])
    assert np.array_equal(out.cpu().numpy(), ref)
    B.gs_prim_exclusive_scan(ctx, xd, out=xd)  # in place
    assert np.array_equal(xd.cpu().numpy(), ref)
