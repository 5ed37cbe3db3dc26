"""Launch-shape autotuner.

Every tunable launch shape of the library (``GS_TUNE_*``) is tried on the
caller's own matrix and preconditioner.  The kernel class that the shape
changes is timed with the library's CUDA-event profiling
(``gs_profile_begin``/``gs_profile_end``, events on the library's stream)
over a few repetitions after a warm-up, and the fastest value is left set in
the context.  Shapes change results only through the order of floating-point
sums; a shape the problem cannot launch (too many threads per block) is
skipped.

The shapes and the kernels they steer:
  * GS_TUNE_SPMV_LANES   lanes per block row of the row SpMV, FP64 or float-float (Sec. 5.3);
  * GS_TUNE_APPLY_RHS    right-hand sides per thread in the level-0 MAS product (Eq. 6);
  * GS_TUNE_SPMV32_LANES lanes per block row of the FP32 SpMV inside the mixed solve;
  * GS_TUNE_BATCH_CHUNK  vector entries per work item of the batched PCG reductions;
  * GS_TUNE_BF16_TC      BF16 level-0 apply on the tensor cores or on the FP32 cores;
  * GS_TUNE_F64_TC       FP64 apply on the BF16 tensor cores (exact digit
                         splitting) or on the FP64 cores.  The digit storage is
                         made when the preconditioner is built, so the sweep
                         stays within the storage built: the symmetric digit
                         bytes (3) or the FP64 cores, or the BF16 digit
                         matrices (one CTA per domain 1, persistent 2) or the
                         FP64 cores;
  * GS_TUNE_SPMV_WS      one thread group per row, or a persistent grid whose
                         warps steal the next rows;
  * GS_TUNE_SPMV_FF_RHS  right-hand sides per thread of the float-float SpMV
                         (8: a row's lanes share its blocks; 4 or 2: the lanes
                         split the right-hand sides, fewer registers and more
                         resident warps);
  * GS_TUNE_SPMV_WINDOW  rows per window of the SpMV's length order.  Not swept:
                         timed alone the SpMV prefers one global order (the
                         longest rows first also balance its tail), but windows
                         cut its DRAM traffic 2.3x at 64^3, which is what counts
                         when other streams share the GPU (8 % more solves/s on
                         three streams), so the window stays as set.
"""

import torch

from . import binding as B

CANDIDATES = {
    B.GS_TUNE_SPMV_LANES: (1, 2, 4, 8),
    B.GS_TUNE_APPLY_RHS: (2, 4, 8),
    B.GS_TUNE_SPMV32_LANES: (2, 4),
    B.GS_TUNE_BATCH_CHUNK: (1024, 2048, 4096, 8192, 16384),
    B.GS_TUNE_BF16_TC: (1, 0),
    B.GS_TUNE_F64_TC: (1, 2, 0),
    B.GS_TUNE_SPMV_WINDOW: (0, 256, 1024, 4096, 16384),
    B.GS_TUNE_SPMV_WS: (0, 1),
    B.GS_TUNE_SPMV_FF_RHS: (8, 4, 2, 1),
}

NAMES = {
    B.GS_TUNE_SPMV_LANES: "spmv_lanes",
    B.GS_TUNE_APPLY_RHS: "apply_rhs_per_thread",
    B.GS_TUNE_SPMV32_LANES: "spmv32_lanes",
    B.GS_TUNE_BATCH_CHUNK: "batch_chunk",
    B.GS_TUNE_BF16_TC: "bf16_tensor_cores",
    B.GS_TUNE_F64_TC: "fp64_on_tensor_cores",
    B.GS_TUNE_SPMV_WINDOW: "spmv_row_window",
    B.GS_TUNE_SPMV_WS: "spmv_work_stealing",
    B.GS_TUNE_SPMV_FF_RHS: "spmv_ff_rhs_per_pass",
}


def time_class(ctx, klass, fn, reps=10, warmup=2):
    """Mean device time (ms) of one launch of kernel class `klass` while `fn` runs."""
    for _ in range(warmup):
        fn()
    B.gs_profile_begin(ctx, [klass])
    try:
        for _ in range(reps):
            fn()
    finally:
        launches, ms = B.gs_profile_end(ctx)
    return float(ms[klass]) / max(int(launches[klass]), 1)


def sweep(ctx, param, klass, fn, reps=10, candidates=None):
    """Time every candidate of `param`; leave the fastest set.  Returns (best, {value: ms})."""
    times = {}
    for v in candidates or CANDIDATES[param]:
        B.gs_tune_set(ctx, param, v)
        try:
            times[v] = time_class(ctx, klass, fn, reps)
        except B.GsError as e:
            if e.status != B.GS_ERR_UNSUPPORTED:
                raise
    if not times:
        raise RuntimeError(f"autotune: no launchable value for {NAMES[param]}")
    best = min(times, key=times.get)
    B.gs_tune_set(ctx, param, best)
    return best, times


def tune(ctx, mat, mas, nrhs=1, reps=10, mixed=False, node_off=None, iters=20, seed=0, bf16=False, fp64=False,
         spmv_variant=B.GS_SPMV_ROW):
    """Tune the shapes a solve on (mat, mas) with `nrhs` right-hand sides uses.

    mixed:    also tune the FP32 SpMV of gs_pcg_solve_mixed;
    bf16:     `mas` holds BF16 factors: also choose tensor cores or FP32 cores
              for its level-0 product;
    fp64:     `mas` is FP64: also choose the digit-split tensor-core product or
              the FP64-core product for level 0;
    node_off: block-row offsets of a batch (gs_pcg_solve_batch); tunes the
              reduction chunk on `iters` fixed iterations;
    spmv_variant: the SpMV whose shapes are tuned (GS_SPMV_ROW or the
              float-float GS_SPMV_ROW_FF; they share the lane and schedule
              parameters).
    Returns {name: (best value, {value: ms per launch})}.
    """
    n = B.gs_mat_info(mat)[0]
    gen = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn((nrhs, 3 * n), dtype=torch.float64, device="cuda", generator=gen)
    y = torch.empty_like(x)
    out = {}
    spmv = lambda: B.gs_spmv(ctx, mat, x, y, nrhs=nrhs, variant=spmv_variant)
    sweep(ctx, B.GS_TUNE_SPMV_WS, B.GS_K_SPMV, spmv, reps)
    out[NAMES[B.GS_TUNE_SPMV_LANES]] = sweep(ctx, B.GS_TUNE_SPMV_LANES, B.GS_K_SPMV, spmv, reps)
    out[NAMES[B.GS_TUNE_SPMV_WS]] = sweep(ctx, B.GS_TUNE_SPMV_WS, B.GS_K_SPMV, spmv, reps)
    if spmv_variant == B.GS_SPMV_ROW_FF and nrhs > 1:
        out[NAMES[B.GS_TUNE_SPMV_FF_RHS]] = sweep(ctx, B.GS_TUNE_SPMV_FF_RHS, B.GS_K_SPMV, spmv, reps)
    apply = lambda: B.gs_mas_apply(ctx, mas, x, y, nrhs=nrhs)
    if fp64:
        built = B.gs_tune_get(ctx, B.GS_TUNE_F64_TC)  # the value `mas` was built with
        cands = (3, 0) if built == 3 else (1, 4, 2, 0) if built in (1, 2, 4) else (0,)
        out[NAMES[B.GS_TUNE_F64_TC]] = sweep(ctx, B.GS_TUNE_F64_TC, B.GS_K_MAS_APPLY_L0, apply, reps, cands)
    if not fp64 or B.gs_tune_get(ctx, B.GS_TUNE_F64_TC) == 0:  # the FP64-core kernel's shape
        out[NAMES[B.GS_TUNE_APPLY_RHS]] = sweep(ctx, B.GS_TUNE_APPLY_RHS, B.GS_K_MAS_APPLY_L0, apply, reps)
    if bf16:
        out[NAMES[B.GS_TUNE_BF16_TC]] = sweep(
            ctx, B.GS_TUNE_BF16_TC, B.GS_K_MAS_APPLY_L0, lambda: B.gs_mas_apply(ctx, mas, x, y, nrhs=nrhs), reps)
    if mixed:
        out[NAMES[B.GS_TUNE_SPMV32_LANES]] = sweep(
            ctx, B.GS_TUNE_SPMV32_LANES, B.GS_K_SPMV,
            lambda: B.gs_pcg_solve_mixed(ctx, mat, mas, x, y.zero_(), nrhs=nrhs, tol=0.0, max_iter=iters,
                                         raise_on_maxiter=False), max(2, reps // 5))
    if node_off is not None:
        b1, x1 = x[0].contiguous(), torch.empty(3 * n, dtype=torch.float64, device="cuda")
        out[NAMES[B.GS_TUNE_BATCH_CHUNK]] = sweep(
            ctx, B.GS_TUNE_BATCH_CHUNK, B.GS_K_PCG_VECTOR,
            lambda: B.gs_pcg_solve_batch(ctx, mat, mas, node_off, b1, x1.zero_(), tol=0.0, max_iter=iters,
                                         use_graph=False, raise_on_maxiter=False), max(2, reps // 5))
    return out


def current(ctx):
    """The context's launch shapes as {name: value}."""
    return {NAMES[p]: B.gs_tune_get(ctx, p) for p in CANDIDATES}
