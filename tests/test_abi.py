"""The C-ABI library loads and exports every symbol the header declares; the
host-side partition matches the oracle bit for bit (no GPU needed)."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import partition
from synth.workloads import make_tet_system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gipc_mas_pcg.h")


@pytest.fixture(scope="module")
def B():
    from paper_2411_06224_gb300.build import build

    build()
    from paper_2411_06224_gb300 import binding

    return binding


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared()
    for n in ("gs_assemble", "gs_build_mas", "gs_pcg_solve", "gs_spmv", "gs_mas_apply", "gs_partition"):
        assert n in names


def test_binding_constants_match_the_header():
    """Every integer GS_* macro of the header has the same value in the binding."""
    from paper_2411_06224_gb300 import binding

    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    macros = dict(re.findall(r"#define\s+(GS_[A-Z0-9_]+)\s+(\(?-?\d+\)?)", text))
    assert len(macros) > 20
    for name, value in macros.items():
        assert hasattr(binding, name), name
        assert getattr(binding, name) == int(value.strip("()")), name


def test_autotuner_knows_every_tuning_parameter():
    """Every GS_TUNE_* parameter of the header has a name and a candidate list
    in the autotuner (bench.py copies the tuned values to every stream's
    context through that list)."""
    from paper_2411_06224_gb300 import autotune, binding

    params = {getattr(binding, n) for n in dir(binding) if n.startswith("GS_TUNE_") and n != "GS_TUNE_COUNT"}
    assert params == set(range(binding.GS_TUNE_COUNT))
    assert set(autotune.CANDIDATES) == params
    assert set(autotune.NAMES) == params
    assert len(set(autotune.NAMES.values())) == len(params)
    for p, values in autotune.CANDIDATES.items():
        assert len(values) >= 2 and len(set(values)) == len(values), p


def test_library_exports_every_declared_symbol(B):
    names = declared()
    L = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gs_\w+)", out))
    assert set(names) <= exported
    assert set(B.EXPORTS) == set(names)


def test_status_strings(B):
    assert B.lib().gs_status_string(0) == b"GS_OK"
    assert B.lib().gs_status_string(-3) == b"GS_ERR_NOT_SPD"


@pytest.mark.parametrize("n,N", [(4, 4), (8, 16), (16, 32), (10, 7), (12, 1)])
def test_partition_matches_oracle(B, n, N):
    s = make_tet_system(n, n_contacts=0, seed=3)
    mp, nd = B.gs_partition(s.X, N)
    part = partition.recursive_bisection(s.X, N)
    mo, _ = partition.map_remap(part, N)
    assert nd == -(-s.n_vertices // N)
    assert np.array_equal(mp, mo)


def test_partition_matches_oracle_ties_and_random(B):
    rng = np.random.default_rng(5)
    X = np.round(rng.normal(size=(777, 3)), 1)  # many equal coordinates
    for N in (3, 16, 32):
        mp, _ = B.gs_partition(X, N)
        mo, _ = partition.map_remap(partition.recursive_bisection(X, N), N)
        assert np.array_equal(mp, mo)


def test_partition_rejects_bad_input(B):
    with pytest.raises(B.GsError) as e:
        B.gs_partition(np.array([[0.0, np.nan, 0.0]]), 4)
    assert e.value.status == B.GS_ERR_INVALID
    with pytest.raises(B.GsError):
        B.gs_partition(np.zeros((4, 3)), 0)


def test_tune_entry_points_reject_a_null_context(B):
    v = ctypes.c_int32(0)
    assert B.lib().gs_tune_set(None, B.GS_TUNE_SPMV_LANES, 2) == B.GS_ERR_INVALID
    assert B.lib().gs_tune_get(None, B.GS_TUNE_SPMV_LANES, ctypes.byref(v)) == B.GS_ERR_INVALID
