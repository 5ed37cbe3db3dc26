"""Thin Python binding of the C ABI in include/gipc_mas_pcg.h.

Functions carry the C names and only marshal arguments: torch CUDA tensors
become device pointers, numpy arrays host pointers, and a non-zero status
raises GsError.  Every step of the solve runs in the CUDA library; if the
library has not been built this module raises instead of falling back.
"""

import ctypes
import os

import numpy as np
import torch

from .build import LIB_PATH

GS_OK = 0
GS_ERR_INVALID = -1
GS_ERR_CUDA = -2
GS_ERR_NOT_SPD = -3
GS_ERR_MAXITER = -4
GS_ERR_NONFINITE = -5
GS_ERR_UNSUPPORTED = -6
GS_ERR_TIMEOUT = -7

GS_SPMV_SRBK = 0
GS_SPMV_ROW = 1
GS_SPMV_ROW_FF = 2
GS_PART_RCB = 0
GS_PART_RCB_COMPONENTS = 1
GS_PART_MORTON = 2
GS_PREC_FP64 = 0
GS_PREC_FP32 = 1
GS_PREC_BF16 = 2

# kernel classes of the profiler (supplement Eq. 1-2 cost split)
GS_K_ASSEMBLE = 0
GS_K_LIBPRIM = 1
GS_K_SPMV = 2
GS_K_MAS_LEVELS = 3
GS_K_MAS_MATRICES = 4
GS_K_MAS_INVERT = 5
GS_K_MAS_APPLY_L0 = 6
GS_K_MAS_APPLY_COARSE = 7
GS_K_PCG_VECTOR = 8
GS_K_OTHER = 9
GS_K_ELEMENT = 10
GS_K_COUNT = 11
GS_TUNE_SPMV_LANES = 0
GS_TUNE_SPMV32_LANES = 1
GS_TUNE_APPLY_RHS = 2
GS_TUNE_BATCH_CHUNK = 3
GS_TUNE_BF16_TC = 4
GS_TUNE_F64_TC = 5
GS_TUNE_SPMV_WINDOW = 6
GS_TUNE_SPMV_WS = 7
GS_TUNE_SPMV_FF_RHS = 8
GS_TUNE_COUNT = 9

K_NAMES = ["assemble", "libprim", "spmv", "mas_levels", "mas_matrices", "mas_invert", "mas_apply_l0",
           "mas_apply_coarse", "pcg_vector", "other", "element"]

# Every symbol the header declares (checked by the test-suite).
EXPORTS = [
    "gs_status_string",
    "gs_last_error",
    "gs_create",
    "gs_set_stream",
    "gs_destroy",
    "gs_assemble",
    "gs_assemble_abd",
    "gs_mat_info",
    "gs_mat_export",
    "gs_mat_destroy",
    "gs_spmv",
    "gs_partition",
    "gs_partition_batch",
    "gs_build_mas",
    "gs_partition_device",
    "gs_build_mas_mesh",
    "gs_mas_info",
    "gs_mas_export_coarse",
    "gs_mas_export_inverse",
    "gs_mas_apply",
    "gs_mas_apply_noalloc",
    "gs_mas_destroy",
    "gs_pcg_solve",
    "gs_pcg_solve_mixed",
    "gs_pcg_solve_batch",
    "gs_adjoint",
    "gs_profile_begin",
    "gs_profile_end",
    "gs_tune_set",
    "gs_tune_get",
    "gs_micro_segment_reduce",
    "gs_micro_bsr_spmv_cusparse",
    "gs_ctx_alloc_stats",
    "gs_debug_raise_flags",
    "gs_fem_create",
    "gs_fem_set_springs",
    "gs_fem_info",
    "gs_fem_export_rest",
    "gs_fem_energy",
    "gs_fem_triplets",
    "gs_fem_assemble",
    "gs_fem_refill",
    "gs_fem_destroy",
    "gs_mas_refresh",
    "gs_fem_newton",
    "gs_prim_sort_pairs",
    "gs_prim_exclusive_scan",
    "gs_cloth_create",
    "gs_cloth_triplets",
    "gs_cloth_info",
    "gs_cloth_destroy",
]


class GsError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {_name(status)}: {_last_error()}")


class gs_mas_opts(ctypes.Structure):
    _fields_ = [("domain_size", ctypes.c_int32), ("max_levels", ctypes.c_int32), ("precision", ctypes.c_int32)]


class gs_newton_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_newton", ctypes.c_int32), ("pcg_tol", ctypes.c_double),
                ("pcg_max_iter", ctypes.c_int32), ("spmv_variant", ctypes.c_int32), ("domain_size", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("precision", ctypes.c_int32), ("part_rule", ctypes.c_int32),
                ("armijo", ctypes.c_double), ("max_halvings", ctypes.c_int32)]


class gs_newton_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("pcg_iterations", ctypes.c_int32), ("halvings", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("energy0", ctypes.c_double), ("energy", ctypes.c_double),
                ("step_inf", ctypes.c_double), ("ms", ctypes.c_double * 6)]


NEWTON_PHASES = ["energy_gradient", "hessian_assembly", "mas", "pcg", "line_search", "total"]


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing: build it with "
                "paper_2411_06224_gb300.build.build() (there is no CPU fallback)"
            )
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "gs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "gs_last_error": (ctypes.c_char_p, []),
            "gs_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
            "gs_set_stream": (ctypes.c_int, [_P, _P]),
            "gs_destroy": (ctypes.c_int, [_P]),
            "gs_assemble": (ctypes.c_int, [_P, _I32, _P, _P, _P, _I64, ctypes.POINTER(_P)]),
            "gs_assemble_abd": (
                ctypes.c_int,
                [_P, _I32, _I32, _I32, _P, _P, _P, _P, _P, _I64, ctypes.POINTER(_P)],
            ),
            "gs_mat_info": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
            "gs_mat_export": (ctypes.c_int, [_P, _P, _P, _P, _P]),
            "gs_mat_destroy": (ctypes.c_int, [_P]),
            "gs_spmv": (ctypes.c_int, [_P, _P, _P, _P, _I32, _I32]),
            "gs_partition": (ctypes.c_int, [_I32, _P, _I32, _P, ctypes.POINTER(_I32)]),
            "gs_partition_batch": (ctypes.c_int, [_I32, _P, _P, _I32, _P, ctypes.POINTER(_I32)]),
            "gs_partition_device": (ctypes.c_int, [_P, _I32, _P, _P, _P, _I32, _I32, _P, ctypes.POINTER(_I32)]),
            "gs_build_mas_mesh": (
                ctypes.c_int,
                [_P, _P, _P, _I32, _P, _P, _P, _I64, ctypes.POINTER(gs_mas_opts), ctypes.POINTER(_P)],
            ),
            "gs_build_mas": (
                ctypes.c_int,
                [_P, _P, _P, _I32, _P, _P, _P, _I64, ctypes.POINTER(gs_mas_opts), ctypes.POINTER(_P)],
            ),
            "gs_mas_info": (ctypes.c_int, [_P, ctypes.POINTER(_I32), _P]),
            "gs_mas_export_coarse": (ctypes.c_int, [_P, _P, _I32, _P]),
            "gs_mas_export_inverse": (ctypes.c_int, [_P, _P, _I32, _P]),
            "gs_mas_apply": (ctypes.c_int, [_P, _P, _P, _P, _I32]),
            "gs_mas_apply_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _I32]),
            "gs_mas_destroy": (ctypes.c_int, [_P]),
            "gs_pcg_solve": (ctypes.c_int, [_P, _P, _P, _P, _I32, _D, _I32, _I32, _P, _P, _P]),
            "gs_pcg_solve_mixed": (ctypes.c_int, [_P, _P, _P, _P, _I32, _D, _I32, _D, _P, _P, _P, _P]),
            "gs_pcg_solve_batch": (ctypes.c_int, [_P, _P, _P, _I32, _P, _P, _D, _I32, _I32, _P, _P, _P]),
            "gs_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P, _I32, _D, _I32, _I32, _P, _P, _P, _P]),
            "gs_profile_begin": (ctypes.c_int, [_P, ctypes.c_uint32]),
            "gs_tune_set": (ctypes.c_int, [_P, _I32, _I32]),
            "gs_micro_segment_reduce": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _I32, _P,
                                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_float)]),
            "gs_micro_bsr_spmv_cusparse": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P, _P, _P, _I32,
                                                           ctypes.POINTER(ctypes.c_float)]),
            "gs_tune_get": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_I32)]),
            "gs_profile_end": (ctypes.c_int, [_P, _P, _P]),
            "gs_ctx_alloc_stats": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
            "gs_debug_raise_flags": (ctypes.c_int, [_P, _I32]),
            "gs_fem_create": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _D, _D, _D, _D, ctypes.POINTER(_P)]),
            "gs_fem_set_springs": (ctypes.c_int, [_P, _P, _P, _P, _P, _I64]),
            "gs_fem_info": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_D),
                                           ctypes.POINTER(_D)]),
            "gs_fem_export_rest": (ctypes.c_int, [_P, _P, _P, _P, _P]),
            "gs_fem_energy": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(_D), _P]),
            "gs_fem_triplets": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
            "gs_fem_assemble": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(_P)]),
            "gs_fem_refill": (ctypes.c_int, [_P, _P, _P, _P]),
            "gs_fem_destroy": (ctypes.c_int, [_P]),
            "gs_mas_refresh": (ctypes.c_int, [_P, _P, _P]),
            "gs_fem_newton": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(gs_newton_opts),
                                             ctypes.POINTER(gs_newton_stats), _P]),
            "gs_prim_sort_pairs": (ctypes.c_int, [_P, _P, _P, _P, _P, _I64, _I32]),
            "gs_prim_exclusive_scan": (ctypes.c_int, [_P, _P, _P, _I64]),
            "gs_cloth_create": (ctypes.c_int, [_P, _I32, _P, _I64, _P, _I64, _P, _D, _D, _D, _D, _D,
                                               ctypes.POINTER(_P)]),
            "gs_cloth_triplets": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
            "gs_cloth_info": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
            "gs_cloth_destroy": (ctypes.c_int, [_P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _name(status):
    return lib().gs_status_string(status).decode()


def _last_error():
    return lib().gs_last_error().decode()


def _check(status, what):
    if status != GS_OK:
        raise GsError(status, what)


def _dev(t, dtype, name):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name}: expected a contiguous CUDA tensor of {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ----------------------------------------------------------------- context
def gs_create(device=0, stream=None):
    h = _P()
    with torch.cuda.device(device):
        _check(lib().gs_create(ctypes.byref(h), device, _stream(stream)), "gs_create")
    return h


def gs_set_stream(ctx, stream=None):
    _check(lib().gs_set_stream(ctx, _stream(stream)), "gs_set_stream")


def gs_destroy(ctx):
    _check(lib().gs_destroy(ctx), "gs_destroy")


# ----------------------------------------------------------------- assembly
def gs_assemble(ctx, n_block_rows, rows, cols, blocks):
    """rows, cols: int32 (K,) CUDA; blocks: float64 (K, 3, 3) CUDA.  Returns a gs_mat handle."""
    h = _P()
    K = rows.numel()
    _check(
        lib().gs_assemble(
            ctx, n_block_rows, _dev(rows, torch.int32, "rows"), _dev(cols, torch.int32, "cols"),
            _dev(blocks, torch.float64, "blocks"), K, ctypes.byref(h),
        ),
        "gs_assemble",
    )
    return h


def gs_assemble_abd(ctx, n_nodes, n_fem, n_bodies, body_of_node, xbar, rows, cols, blocks):
    h = _P()
    _check(
        lib().gs_assemble_abd(
            ctx, n_nodes, n_fem, n_bodies, _dev(body_of_node, torch.int32, "body_of_node"),
            _dev(xbar, torch.float64, "xbar"), _dev(rows, torch.int32, "rows"), _dev(cols, torch.int32, "cols"),
            _dev(blocks, torch.float64, "blocks"), rows.numel(), ctypes.byref(h),
        ),
        "gs_assemble_abd",
    )
    return h


def gs_mat_info(mat):
    n = _I32()
    nz = _I64()
    _check(lib().gs_mat_info(mat, ctypes.byref(n), ctypes.byref(nz)), "gs_mat_info")
    return n.value, nz.value


def gs_mat_export(ctx, mat, device="cuda"):
    """(rid, cid, au) as new CUDA tensors (int32, int32, float64 (U, 3, 3))."""
    n, nz = gs_mat_info(mat)
    rid = torch.empty(nz, dtype=torch.int32, device=device)
    cid = torch.empty(nz, dtype=torch.int32, device=device)
    au = torch.empty((nz, 3, 3), dtype=torch.float64, device=device)
    if nz:
        _check(
            lib().gs_mat_export(ctx, mat, _dev(rid, torch.int32, "rid"), _dev(cid, torch.int32, "cid"),
                                _dev(au, torch.float64, "au")),
            "gs_mat_export",
        )
    return rid, cid, au


def gs_mat_destroy(mat):
    _check(lib().gs_mat_destroy(mat), "gs_mat_destroy")


# ----------------------------------------------------------------- SpMV
def gs_spmv(ctx, mat, x, y, nrhs=1, variant=GS_SPMV_ROW):
    _check(
        lib().gs_spmv(ctx, mat, _dev(x, torch.float64, "x"), _dev(y, torch.float64, "y"), nrhs, variant),
        "gs_spmv",
    )


# ----------------------------------------------------------------- partition / MAS
def gs_partition(X, domain_size):
    """Host partition of positions X (V, 3) float64 -> (map int32 (V,), n_domains)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    V = X.shape[0]
    mp = np.empty(V, dtype=np.int32)
    nd = _I32()
    _check(
        lib().gs_partition(V, X.ctypes.data_as(_P), domain_size, mp.ctypes.data_as(_P), ctypes.byref(nd)),
        "gs_partition",
    )
    return mp, nd.value


def gs_partition_batch(X, node_off, domain_size):
    """Host partition of several meshes (nodes [node_off[s], node_off[s+1])) -> (map, n_domains)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    off = np.ascontiguousarray(node_off, dtype=np.int32)
    mp = np.empty(X.shape[0], dtype=np.int32)
    nd = _I32()
    _check(
        lib().gs_partition_batch(off.size - 1, off.ctypes.data_as(_P), X.ctypes.data_as(_P), domain_size,
                                 mp.ctypes.data_as(_P), ctypes.byref(nd)),
        "gs_partition_batch",
    )
    return mp, nd.value


def gs_partition_device(ctx, X, domain_size, rule=GS_PART_RCB, adj_ptr=None, adj=None):
    """Device partition of positions X ((V, 3) float64 CUDA tensor) -> (map int32 CUDA tensor (V,), n_domains)."""
    V = X.shape[0]
    mp = torch.empty(V, dtype=torch.int32, device=X.device)
    nd = _I32()
    _check(
        lib().gs_partition_device(ctx, V, _dev(X, torch.float64, "X"),
                                  _dev(adj_ptr, torch.int32, "adj_ptr") if adj_ptr is not None else None,
                                  _dev(adj, torch.int32, "adj") if adj is not None else None, domain_size, rule,
                                  _dev(mp, torch.int32, "map"), ctypes.byref(nd)),
        "gs_partition_device",
    )
    return mp, nd.value


def gs_build_mas_mesh(ctx, mat, X, adj_ptr, adj, contacts, domain_size=32, max_levels=2, precision=GS_PREC_FP64,
                      part_rule=GS_PART_RCB):
    """The MAS with its level-0 partition computed on the device from X ((V, 3) float64 CUDA tensor)."""
    h = _P()
    opts = gs_mas_opts(domain_size, max_levels, precision)
    P = 0 if contacts is None else contacts.shape[0]
    _check(
        lib().gs_build_mas_mesh(
            ctx, mat, _dev(X, torch.float64, "X"), part_rule, _dev(adj_ptr, torch.int32, "adj_ptr"),
            _dev(adj, torch.int32, "adj"), _dev(contacts, torch.int32, "contacts") if P else None, P,
            ctypes.byref(opts), ctypes.byref(h),
        ),
        "gs_build_mas_mesh",
    )
    return h


def gs_build_mas(ctx, mat, map_, n_domains0, adj_ptr, adj, contacts, domain_size=32, max_levels=2,
                 precision=GS_PREC_FP64):
    """map_, adj_ptr, adj, contacts: int32 CUDA tensors (contacts (P, 2) or None)."""
    h = _P()
    opts = gs_mas_opts(domain_size, max_levels, precision)
    P = 0 if contacts is None else contacts.shape[0]
    _check(
        lib().gs_build_mas(
            ctx, mat, _dev(map_, torch.int32, "map"), n_domains0, _dev(adj_ptr, torch.int32, "adj_ptr"),
            _dev(adj, torch.int32, "adj"), _dev(contacts, torch.int32, "contacts") if P else None, P,
            ctypes.byref(opts), ctypes.byref(h),
        ),
        "gs_build_mas",
    )
    return h


def gs_mas_info(mas):
    L = _I32()
    items = (ctypes.c_int32 * 8)()
    _check(lib().gs_mas_info(mas, ctypes.byref(L), ctypes.cast(items, _P)), "gs_mas_info")
    return L.value, [items[i] for i in range(L.value)]


def gs_mas_export_coarse(ctx, mas, level, n, device="cuda"):
    out = torch.empty(n, dtype=torch.int32, device=device)
    _check(lib().gs_mas_export_coarse(ctx, mas, level, _dev(out, torch.int32, "coarse")), "gs_mas_export_coarse")
    return out


def gs_mas_export_inverse(ctx, mas, level, n_domains, domain_size, device="cuda"):
    ld = 3 * domain_size
    out = torch.empty((n_domains, ld, ld), dtype=torch.float64, device=device)
    _check(lib().gs_mas_export_inverse(ctx, mas, level, _dev(out, torch.float64, "inv")), "gs_mas_export_inverse")
    return out


def gs_mas_apply(ctx, mas, r, z, nrhs=1):
    _check(lib().gs_mas_apply(ctx, mas, _dev(r, torch.float64, "r"), _dev(z, torch.float64, "z"), nrhs),
           "gs_mas_apply")


def gs_mas_destroy(mas):
    _check(lib().gs_mas_destroy(mas), "gs_mas_destroy")


# ----------------------------------------------------------------- PCG
def gs_pcg_solve(ctx, mat, mas, b, x, nrhs=1, tol=1e-6, max_iter=10_000, variant=GS_SPMV_ROW,
                 raise_on_maxiter=True):
    """Solve A x = b for nrhs stacked right-hand sides; returns (iters, rel_res, status)."""
    iters = np.zeros(nrhs, dtype=np.int32)
    rel = np.zeros(nrhs, dtype=np.float64)
    s = lib().gs_pcg_solve(
        ctx, mat, mas, _dev(b, torch.float64, "b"), nrhs, tol, max_iter, variant, _dev(x, torch.float64, "x"),
        iters.ctypes.data_as(_P), rel.ctypes.data_as(_P),
    )
    if s != GS_OK and not (s == GS_ERR_MAXITER and not raise_on_maxiter):
        raise GsError(s, "gs_pcg_solve")
    return iters, rel, s


def gs_pcg_solve_mixed(ctx, mat, mas, b, x, nrhs=1, tol=1e-6, max_iter=20_000, inner_tol=1e-3,
                       raise_on_maxiter=True):
    """FP64 refinement around FP32 MAS-PCG; returns (inner iters, true rel_res, outer steps, status)."""
    iters = np.zeros(nrhs, dtype=np.int32)
    rel = np.zeros(nrhs, dtype=np.float64)
    outer = _I32()
    s = lib().gs_pcg_solve_mixed(
        ctx, mat, mas, _dev(b, torch.float64, "b"), nrhs, tol, max_iter, inner_tol, _dev(x, torch.float64, "x"),
        iters.ctypes.data_as(_P), rel.ctypes.data_as(_P), ctypes.byref(outer),
    )
    if s != GS_OK and not (s == GS_ERR_MAXITER and not raise_on_maxiter):
        raise GsError(s, "gs_pcg_solve_mixed")
    return iters, rel, outer.value, s


def gs_pcg_solve_batch(ctx, mat, mas, node_off, b, x, tol=1e-6, max_iter=20_000, use_graph=True,
                       raise_on_maxiter=True):
    """Independent PCG per system of a block-diagonal batch; returns (iters, rel_res, status)."""
    off = np.ascontiguousarray(node_off, dtype=np.int32)
    S = off.size - 1
    iters = np.zeros(S, dtype=np.int32)
    rel = np.zeros(S, dtype=np.float64)
    s = lib().gs_pcg_solve_batch(ctx, mat, mas, S, off.ctypes.data_as(_P), _dev(b, torch.float64, "b"), tol,
                                 max_iter, 1 if use_graph else 0, _dev(x, torch.float64, "x"),
                                 iters.ctypes.data_as(_P), rel.ctypes.data_as(_P))
    if s != GS_OK and not (s == GS_ERR_MAXITER and not raise_on_maxiter):
        raise GsError(s, "gs_pcg_solve_batch")
    return iters, rel, s


def gs_adjoint(ctx, mat, mas, x, g, nrhs=1, tol=1e-10, max_iter=20_000, mixed=False, dLdH=None, dLdinput=None):
    """lambda = A^{-1} g (= dL/db) plus the optional block gradients; returns (lambda, iters)."""
    lam = torch.empty_like(g)
    iters = np.zeros(nrhs, dtype=np.int32)
    _check(
        lib().gs_adjoint(
            ctx, mat, mas, _dev(x, torch.float64, "x"), _dev(g, torch.float64, "g"), nrhs, tol, max_iter,
            1 if mixed else 0, _dev(lam, torch.float64, "lam"), _dev(dLdH, torch.float64, "dLdH"),
            _dev(dLdinput, torch.float64, "dLdinput"), iters.ctypes.data_as(_P),
        ),
        "gs_adjoint",
    )
    return lam, iters


# ----------------------------------------------------------------- measurement
def gs_profile_begin(ctx, timed_classes=()):
    mask = 0
    for k in timed_classes:
        mask |= 1 << k
    _check(lib().gs_profile_begin(ctx, mask), "gs_profile_begin")


def gs_profile_end(ctx):
    """Returns (launches int64[GS_K_COUNT], ms float64[GS_K_COUNT])."""
    launches = np.zeros(GS_K_COUNT, dtype=np.int64)
    ms = np.zeros(GS_K_COUNT, dtype=np.float64)
    _check(lib().gs_profile_end(ctx, launches.ctypes.data_as(_P), ms.ctypes.data_as(_P)), "gs_profile_end")
    return launches, ms


# ----------------------------------------------------------------- tuning
def gs_tune_set(ctx, param, value):
    _check(lib().gs_tune_set(ctx, param, value), "gs_tune_set")


def gs_tune_get(ctx, param):
    v = _I32()
    _check(lib().gs_tune_get(ctx, param, ctypes.byref(v)), "gs_tune_get")
    return v.value


def gs_ctx_alloc_stats(ctx):
    """(number, total bytes) of the device allocations the library made on ctx."""
    n, b = _I64(), _I64()
    _check(lib().gs_ctx_alloc_stats(ctx, ctypes.byref(n), ctypes.byref(b)), "gs_ctx_alloc_stats")
    return n.value, b.value


def gs_debug_raise_flags(ctx, flags):
    _check(lib().gs_debug_raise_flags(ctx, flags), "gs_debug_raise_flags")


# ----------------------------------------------------------------- microbenchmarks
def gs_micro_segment_reduce(ctx, keys, blocks, method):
    """keys: sorted uint64 as int64 CUDA tensor (nb,); blocks float64 (nb, 3, 3).
    Returns (reduced blocks (U, 3, 3), ms)."""
    nb = keys.numel()
    out = torch.empty((nb, 3, 3), dtype=torch.float64, device=keys.device)
    nu = ctypes.c_int64()
    ms = ctypes.c_float()
    _check(lib().gs_micro_segment_reduce(ctx, nb, _dev(keys, torch.int64, "keys"), _dev(blocks, torch.float64, "blocks"),
                                         method, _dev(out, torch.float64, "out"), ctypes.byref(nu), ctypes.byref(ms)),
           "gs_micro_segment_reduce")
    return out[: nu.value], ms.value


def gs_micro_bsr_spmv_cusparse(ctx, n, row_ptr, col_ind, vals, x, y, reps=10):
    ms = ctypes.c_float()
    _check(lib().gs_micro_bsr_spmv_cusparse(ctx, n, col_ind.numel(), _dev(row_ptr, torch.int32, "row_ptr"),
                                            _dev(col_ind, torch.int32, "col_ind"), _dev(vals, torch.float64, "vals"),
                                            _dev(x, torch.float64, "x"), _dev(y, torch.float64, "y"), reps,
                                            ctypes.byref(ms)),
           "gs_micro_bsr_spmv_cusparse")
    return ms.value


# ---------------------------------------------------------------- elastic bodies and Newton
def gs_fem_create(ctx, X, tets, E, nu, rho, dt):
    """X: (V, 3) float64, tets: (T, 4) int32 CUDA tensors (copied)."""
    h = _P()
    _check(lib().gs_fem_create(ctx, X.shape[0], tets.shape[0], _dev(X, torch.float64, "X"),
                               _dev(tets, torch.int32, "tets"), E, nu, rho, dt, ctypes.byref(h)), "gs_fem_create")
    return h


def gs_fem_set_springs(ctx, fem, pairs, K, rest):
    """pairs (P, 2) int32, K (P, 3, 3) float64, rest (P, 3) float64 CUDA tensors; P = 0 or None removes them."""
    n = 0 if pairs is None else pairs.shape[0]
    _check(lib().gs_fem_set_springs(ctx, fem, _dev(pairs, torch.int32, "pairs") if n else None,
                                    _dev(K, torch.float64, "K") if n else None,
                                    _dev(rest, torch.float64, "rest") if n else None, n), "gs_fem_set_springs")


def gs_fem_info(fem):
    """(stored blocks, element-only stored blocks, mu, lam)."""
    u, ue, mu, lam = _I64(), _I64(), _D(), _D()
    _check(lib().gs_fem_info(fem, ctypes.byref(u), ctypes.byref(ue), ctypes.byref(mu), ctypes.byref(lam)),
           "gs_fem_info")
    return u.value, ue.value, mu.value, lam.value


def gs_fem_export_rest(ctx, fem, T, V):
    """(w (T, 4, 3), vol (T,), mass (V,)) float64 CUDA tensors."""
    w = torch.empty((T, 4, 3), dtype=torch.float64, device="cuda")
    vol = torch.empty(T, dtype=torch.float64, device="cuda")
    mass = torch.empty(V, dtype=torch.float64, device="cuda")
    _check(lib().gs_fem_export_rest(ctx, fem, _dev(w, torch.float64, "w"), _dev(vol, torch.float64, "vol"),
                                    _dev(mass, torch.float64, "mass")), "gs_fem_export_rest")
    return w, vol, mass


def gs_fem_energy(ctx, fem, x, xt, grad=None):
    """E(x) as a float; the gradient written into grad ((V, 3) float64) when given."""
    e = _D()
    _check(lib().gs_fem_energy(ctx, fem, _dev(x, torch.float64, "x"), _dev(xt, torch.float64, "xt"), ctypes.byref(e),
                               _dev(grad, torch.float64, "grad")), "gs_fem_energy")
    return e.value


def gs_fem_triplets(ctx, fem, x, n_entries):
    """(rows, cols, blocks (n, 3, 3)) CUDA tensors of the Hessian at x."""
    rows = torch.empty(n_entries, dtype=torch.int32, device="cuda")
    cols = torch.empty(n_entries, dtype=torch.int32, device="cuda")
    blocks = torch.empty((n_entries, 3, 3), dtype=torch.float64, device="cuda")
    _check(lib().gs_fem_triplets(ctx, fem, _dev(x, torch.float64, "x"), _dev(rows, torch.int32, "rows"),
                                 _dev(cols, torch.int32, "cols"), _dev(blocks, torch.float64, "blocks")),
           "gs_fem_triplets")
    return rows, cols, blocks


def gs_prim_sort_pairs(ctx, keys, vals, end_bit):
    """Stable radix sort of (keys uint64 as torch.int64, vals int32) CUDA tensors by key bits
    [0, end_bit); returns new (keys, vals) tensors."""
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    if keys.numel() and not (keys.dtype == torch.int64 and vals.dtype == torch.int32 and keys.is_cuda and vals.is_cuda
                             and keys.is_contiguous() and vals.is_contiguous() and keys.numel() == vals.numel()):
        raise TypeError("gs_prim_sort_pairs: contiguous CUDA int64 keys and int32 values of one length")
    _check(lib().gs_prim_sort_pairs(ctx, ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                    ctypes.c_void_p(ko.data_ptr()), ctypes.c_void_p(vo.data_ptr()), keys.numel(),
                                    end_bit), "gs_prim_sort_pairs")
    return ko, vo


def gs_prim_exclusive_scan(ctx, x, out=None):
    """Exclusive prefix sum of an int32 CUDA tensor (out may be x)."""
    out = torch.empty_like(x) if out is None else out
    _check(lib().gs_prim_exclusive_scan(ctx, _dev(x, torch.int32, "in"), _dev(out, torch.int32, "out"), x.numel()),
           "gs_prim_exclusive_scan")
    return out


def gs_cloth_create(ctx, X, tris, hinges, E, lam, thickness, rho, dt):
    """X (V, 3) float64, tris (T, 3) int32, hinges (H, 4) int32 CUDA tensors (copied)."""
    h = _P()
    _check(lib().gs_cloth_create(ctx, X.shape[0], _dev(X, torch.float64, "X"), tris.shape[0],
                                 _dev(tris, torch.int32, "tris"), hinges.shape[0], _dev(hinges, torch.int32, "hinges"),
                                 E, lam, thickness, rho, dt, ctypes.byref(h)), "gs_cloth_create")
    return h


def gs_cloth_info(c):
    """Number of triplets gs_cloth_triplets writes."""
    n = _I64()
    _check(lib().gs_cloth_info(c, ctypes.byref(n)), "gs_cloth_info")
    return n.value


def gs_cloth_triplets(ctx, c, x):
    """(rows, cols, blocks (n, 3, 3)) CUDA tensors of the cloth Hessian at x ((V, 3) float64)."""
    n = gs_cloth_info(c)
    rows = torch.empty(n, dtype=torch.int32, device="cuda")
    cols = torch.empty(n, dtype=torch.int32, device="cuda")
    blocks = torch.empty((n, 3, 3), dtype=torch.float64, device="cuda")
    _check(lib().gs_cloth_triplets(ctx, c, _dev(x, torch.float64, "x"), _dev(rows, torch.int32, "rows"),
                                   _dev(cols, torch.int32, "cols"), _dev(blocks, torch.float64, "blocks")),
           "gs_cloth_triplets")
    return rows, cols, blocks


def gs_cloth_destroy(c):
    _check(lib().gs_cloth_destroy(c), "gs_cloth_destroy")


def gs_fem_assemble(ctx, fem, x):
    h = _P()
    _check(lib().gs_fem_assemble(ctx, fem, _dev(x, torch.float64, "x"), ctypes.byref(h)), "gs_fem_assemble")
    return h


def gs_fem_refill(ctx, fem, x, mat):
    _check(lib().gs_fem_refill(ctx, fem, _dev(x, torch.float64, "x"), mat), "gs_fem_refill")


def gs_fem_destroy(fem):
    _check(lib().gs_fem_destroy(fem), "gs_fem_destroy")


def gs_mas_refresh(ctx, mas, mat):
    _check(lib().gs_mas_refresh(ctx, mas, mat), "gs_mas_refresh")


def gs_fem_newton(ctx, fem, xt, x, adj_ptr, adj, tol=1e-3, max_newton=50, pcg_tol=1e-6, pcg_max_iter=10_000,
                  spmv_variant=GS_SPMV_ROW, domain_size=32, max_levels=3, precision=GS_PREC_FP64,
                  part_rule=GS_PART_RCB, armijo=1e-4, max_halvings=30, raise_on_maxiter=True):
    """Newton's method from x (overwritten).  Returns (stats dict, energies (iterations + 1,), status)."""
    o = gs_newton_opts(tol, max_newton, pcg_tol, pcg_max_iter, spmv_variant, domain_size, max_levels, precision,
                       part_rule, armijo, max_halvings)
    st = gs_newton_stats()
    en = np.zeros(max_newton + 1, dtype=np.float64)
    s = lib().gs_fem_newton(ctx, fem, _dev(xt, torch.float64, "xt"), _dev(x, torch.float64, "x"),
                            _dev(adj_ptr, torch.int32, "adj_ptr"), _dev(adj, torch.int32, "adj"), ctypes.byref(o),
                            ctypes.byref(st), en.ctypes.data_as(_P))
    if s != GS_OK and not (s == GS_ERR_MAXITER and not raise_on_maxiter):
        raise GsError(s, "gs_fem_newton")
    stats = dict(iterations=st.iterations, pcg_iterations=st.pcg_iterations, halvings=st.halvings,
                 converged=bool(st.converged), energy0=st.energy0, energy=st.energy, step_inf=st.step_inf,
                 ms={k: st.ms[i] for i, k in enumerate(NEWTON_PHASES)})
    return stats, en[: st.iterations + 1].copy(), s
