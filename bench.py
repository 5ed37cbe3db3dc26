#!/usr/bin/env python3
"""Newton solves/s of the MAS-PCG linear solve on the 64^3 stiffness sweep.

Workload (synthetic, seeded): a 64^3-vertex tet cube (262,144 vertices,
786,432 DOF, 1,250,235 tets split 5 per cell), stable Neo-Hookean Hessian
with E in {1e5, 1e7, 1e9} Pa, nu = 0.4, lumped mass / dt^2 (rho = 1000,
dt = 0.01), 200k PSD contact blocks between vertices closer than 2h; 8 N(0,1)
right-hand sides; 3-level MAS with 32-node domains; PCG to 1e-6 relative
residual.  It stands in for the paper's FEM scenes, which are not available.

One step = one Newton solve of each of the three systems: hash-key assembly
of its 13.4M triplets, device MAS build, and 8-RHS PCG (supplement Eq. 1:
T = T_ga + T_pa + N_pcg T_pcg).  The level-0 partition is computed once per
mesh before timing, as the paper runs METIS once before the simulation.
`value` counts Newton solves (one system, all its right-hand sides) per
second with inputs resident in HBM; `e2e` repeats the step through the
same public API with the triplets and right-hand sides copied from pinned
host memory every step and the solutions copied back.
"""

import argparse
from concurrent.futures import ThreadPoolExecutor
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_FMA_PER_CLK_PER_SM = 2  # GB300: derived from the nominal 1.25 TFLOP/s FP64 at 2.07 GHz, 152 SMs
# DRAM bytes of one FP64-core level-0 apply launch per domain at 8 RHS, from
# an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) on the 40^3
# case: 172.9 MB over 2000 domains; traffic grows with the domain count.
APPLY_DRAM_BYTES_PER_DOMAIN_8RHS = 172.9e6 / 2000
# DRAM bytes per level-0 domain of the digit-split tensor-core apply at 8 RHS,
# from an ncu capture on the 64^3 case: 1,115.9 MB read + 48.4 MB written over
# 8,192 domains
F64TC_DRAM_BYTES_PER_DOMAIN_8RHS = (1115.9e6 + 48.4e6) / 8192
# DRAM bytes (read + written) of one work-stealing row-SpMV launch on the 64^3
# sweep system at 8 RHS and the 1024-row order window, by lanes per row, from
# ncu captures of that case
SPMV_WS_DRAM_BYTES_64 = {1: 426.5e6 + 75.6e6, 2: 225.2e6 + 39.8e6}
TOL = 1e-6
# The headline metric as named for this workload: `value` is the FP64 path's
# Newton solves/s; the mixed-precision forms are under forms.mixed_precision
# and the SpMV's HBM GB/s under roofline.hbm_gbs / kernels.spmv_hbm_gbs.
METRIC = "Newton solves/s to 1e-6 rel. residual (FP64 vs mixed MAS-PCG); SpMV HBM GB/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=64, help="vertices per cube edge (64 = the named workload)")
    p.add_argument("--nrhs", type=int, default=8)
    p.add_argument("--sweep", default="1e5,1e7,1e9",
                   help="Young's moduli of the step's systems (the named workload: 1e5,1e7,1e9; a single value "
                        "keeps profiling runs small)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--spmv", default="row", choices=["row", "srbk", "ff"],
                   help="row: FP64 row gather; srbk: the paper's SRBK; ff: row gather in float-float on the FP32 units")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--mixed-steps", type=int, default=3, help="timed steps of the mixed-precision form")
    p.add_argument("--no-lanes", dest="lanes", action="store_false",
                   help="solve the systems of a step one after another on one stream")
    p.add_argument("--streams", type=int, default=0,
                   help="with lanes: library contexts / streams working the queue (0 = one per system of a step)")
    p.add_argument("--step-sync", dest="queue", action="store_false",
                   help="with lanes: wait for all systems of a step before the next step starts, instead of one "
                        "queue over the timed steps' solves")
    p.add_argument("--no-autotune", dest="autotune", action="store_false",
                   help="keep the default launch shapes instead of tuning them first")
    p.add_argument("--batch-steps", type=int, default=2, help="timed steps of the batched form (64 uneven systems)")
    p.add_argument("--cloth", type=int, default=512,
                   help="vertices per edge of the stiff-cloth precision case (0 = skip)")
    p.add_argument("--set-tune", action="append", default=[], metavar="NAME=VALUE",
                   help="force a launch shape after tuning (names as in config.launch_shapes), e.g. "
                        "spmv_lanes=2; repeatable")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--micro", action="store_true",
                   help="instead of the solve benchmark: the paper's reduction and SpMV microbenchmarks")
    p.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)  # worker mode
    return p.parse_args()


# --------------------------------------------------------------------------- oracle sample
def oracle_sample(spec):
    """Time the oracle on bounded samples of the workload (run in a fresh
    single-threaded process).  Input generation is not timed.  Prints one
    JSON list with, per sample, the seconds of assembly (t_ga), MAS build
    (t_pa) and one PCG iteration on one RHS (t_iter)."""
    from oracle import assembly, mas, partition, pcg
    from synth.workloads import rhs, stiffness_sweep

    systems = stiffness_sweep(Es=tuple(spec["Es"]), n=spec["grid"])
    V = systems[0].n_vertices
    mp, _ = partition.map_remap(partition.recursive_bisection(systems[0].X, 32), 32)  # pre-simulation
    b = rhs(3 * V, 1)
    out = []
    for q in range(spec["samples"]):
        sys_ = systems[q % len(systems)]
        t0 = time.perf_counter()
        rid, cid, au = assembly.assemble(sys_.rows, sys_.cols, sys_.blocks)
        t1 = time.perf_counter()
        M = mas.build_mas(mp, 32, 3, sys_.adj_ptr, sys_.adj, sys_.contacts, rid, cid, au)
        A = pcg.SymmetricMatrix(V, rid, cid, au)
        t2 = time.perf_counter()
        pcg.pcg(A, M, b, fixed_iters=spec["iters"])
        t3 = time.perf_counter()
        out.append({"E": sys_.params["E"], "t_ga": t1 - t0, "t_pa": t2 - t1, "t_iter": (t3 - t2) / spec["iters"],
                    "k": spec["iters"], "V": V})
    print(json.dumps(out))


def run_oracle_sample(grid, Es, samples, iters=3):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    spec = json.dumps({"grid": grid, "Es": list(Es), "samples": samples, "iters": iters})
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", spec], env=env,
                       capture_output=True, text=True, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_rate(sample, iters_per_solve):
    """Newton solves/s of the oracle: T_ga + T_pa + (PCG iterations summed over the RHS) * T_iter."""
    t = sample["t_ga"] + sample["t_pa"] + iters_per_solve * sample["t_iter"]
    return 1.0 / t, t


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- workload on the GPU
def autotune_current(B, ctx):
    from paper_2411_06224_gb300 import autotune

    return autotune.current(ctx)


def make_workload(grid, nrhs, rank, Es=(1e5, 1e7, 1e9)):
    import numpy as np

    from synth.workloads import rhs, stiffness_sweep

    systems = stiffness_sweep(Es=tuple(Es), n=grid, seed=1002 + rank)
    b = rhs(3 * systems[0].n_vertices, nrhs, seed0=2000 + 100 * rank)
    return systems, np.ascontiguousarray(b)


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample(json.loads(args.oracle_sample))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.micro:
        return micro(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2411_06224_gb300.build import build

    build()
    from paper_2411_06224_gb300 import binding as B

    dev = torch.device("cuda", local)
    systems, b_host = make_workload(args.grid, args.nrhs, rank, Es=[float(e) for e in args.sweep.split(",")])
    V = systems[0].n_vertices
    N, L = 32, 3
    prec = B.GS_PREC_FP32 if args.precision == "fp32" else B.GS_PREC_FP64
    variant = {"row": B.GS_SPMV_ROW, "srbk": B.GS_SPMV_SRBK, "ff": B.GS_SPMV_ROW_FF}[args.spmv]
    mp, ndom = B.gs_partition(systems[0].X, N)  # once per mesh, before timing
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    shared = dict(map=t(mp, torch.int32), adj_ptr=t(systems[0].adj_ptr, torch.int32), adj=t(systems[0].adj, torch.int32),
                  contacts=t(systems[0].contacts, torch.int32))
    dsys = [dict(rows=t(s.rows, torch.int32), cols=t(s.cols, torch.int32), blocks=t(s.blocks.reshape(-1, 3, 3), torch.float64),
                 E=s.params["E"]) for s in systems]
    b = t(b_host, torch.float64)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()
    ctx = B.gs_create(local, stream)

    def solve_one(rows, cols, blocks, bb, xx, c=None):
        c = c or ctx
        mat = B.gs_assemble(c, V, rows, cols, blocks)
        mas = B.gs_build_mas(c, mat, shared["map"], ndom, shared["adj_ptr"], shared["adj"], shared["contacts"],
                             domain_size=N, max_levels=L, precision=prec)
        it, rel, _ = B.gs_pcg_solve(c, mat, mas, bb, xx, nrhs=args.nrhs, tol=TOL, max_iter=20000, variant=variant)
        info = (B.gs_mat_info(mat)[1], B.gs_mas_info(mas))
        B.gs_mas_destroy(mas)
        B.gs_mat_destroy(mat)
        return it, rel, info

    # The systems of a step are independent Newton solves.  With --lanes (the
    # default) each runs on its own library context and CUDA stream, driven by
    # its own host thread, so the FP64-pipe-bound SpMV of one system overlaps
    # the HBM- and tensor-bound MAS apply of another.
    n_lanes = (args.streams if args.streams > 0 and args.queue else len(dsys)) if args.lanes else 1
    lane_streams = [torch.cuda.Stream(device=dev) for _ in range(n_lanes)] if args.lanes else [stream]
    lane_ctx = [B.gs_create(local, s_) for s_ in lane_streams] if args.lanes else [ctx]
    # solution buffers per lane and system: two steps' solves of one system
    # may run at once on two lanes
    lane_xs = [[torch.zeros_like(b) for _ in dsys] for _ in range(n_lanes)] if args.lanes else [[x] * len(dsys)]
    last_lane = {}  # system -> lane of its latest finished solve
    pool = ThreadPoolExecutor(max_workers=n_lanes)

    def fork():
        ev = torch.cuda.Event()
        ev.record(stream)
        for s_ in lane_streams:
            s_.wait_event(ev)

    def join():
        for s_ in lane_streams:
            ev = torch.cuda.Event()
            ev.record(s_)
            stream.wait_event(ev)

    def lane_run(i, fn):
        torch.cuda.set_device(local)
        with torch.cuda.stream(lane_streams[i]):
            return fn(i)

    def step():
        if n_lanes == 1:
            return [solve_one(s["rows"], s["cols"], s["blocks"], b, x) for s in dsys]
        fork()
        futs = [pool.submit(lane_run, i, lambda i, s=s: solve_one(s["rows"], s["cols"], s["blocks"], b, lane_xs[i][i],
                                                                   lane_ctx[i]))
                for i, s in enumerate(dsys)]
        out = [f.result() for f in futs]
        join()
        for i in range(len(dsys)):
            last_lane[i] = i
        return out

    def queue(n_steps, order, job):
        """The solves of n_steps steps as one queue over the lanes: each lane's
        thread takes the next solve as soon as its previous one is done, so no
        lane idles while a step's slowest system finishes.  order: the systems
        of a step, longest first.  job(lane, system) -> result."""
        jobs = [si for _ in range(n_steps) for si in order]
        nxt = iter(range(len(jobs)))
        lock = threading.Lock()
        out = {}

        def worker(i):
            while True:
                with lock:
                    j = next(nxt, None)
                if j is None:
                    return
                r = job(i, jobs[j])
                with lock:
                    out[jobs[j]] = r
                    last_lane[jobs[j]] = i

        fork()
        futs = [pool.submit(lane_run, i, worker) for i in range(n_lanes)]
        [f.result() for f in futs]
        join()
        return [out[si] for si in range(len(dsys))]

    def solve_job(i, si):
        s = dsys[si]
        return solve_one(s["rows"], s["cols"], s["blocks"], b, lane_xs[i][si], lane_ctx[i])

    def profile_begin(classes):
        for c in lane_ctx:
            B.gs_profile_begin(c, classes)

    def profile_end():
        tot_l, tot_ms = None, None
        for c in lane_ctx:
            l_, m_ = B.gs_profile_end(c)
            tot_l = l_ if tot_l is None else tot_l + l_
            tot_ms = m_ if tot_ms is None else tot_ms + m_
        return tot_l, tot_ms

    def barrier():
        if world > 1:
            dist.barrier()

    # launch shapes: the autotuner times each candidate on the stiffest system
    # (outside the timed region) and leaves the fastest set in the context
    tuned = None
    if args.autotune:
        from paper_2411_06224_gb300 import autotune

        s = dsys[-1]
        mat = B.gs_assemble(ctx, V, s["rows"], s["cols"], s["blocks"])
        mas = B.gs_build_mas(ctx, mat, shared["map"], ndom, shared["adj_ptr"], shared["adj"], shared["contacts"],
                             domain_size=N, max_levels=L, precision=prec)
        res = autotune.tune(ctx, mat, mas, nrhs=args.nrhs, reps=5, mixed=args.mixed_steps > 0,
                            fp64=prec == B.GS_PREC_FP64,
                            spmv_variant=variant if variant != B.GS_SPMV_SRBK else B.GS_SPMV_ROW)
        B.gs_mas_destroy(mas)
        if args.mixed_steps > 0 and args.nrhs <= 8:  # BF16 level-0 product: tensor cores or FP32 cores
            mas = B.gs_build_mas(ctx, mat, shared["map"], ndom, shared["adj_ptr"], shared["adj"], shared["contacts"],
                                 domain_size=N, max_levels=L, precision=B.GS_PREC_BF16)
            xr = torch.randn((args.nrhs, 3 * V), dtype=torch.float64, device=dev)
            yr = torch.empty_like(xr)
            res[autotune.NAMES[B.GS_TUNE_BF16_TC]] = autotune.sweep(
                ctx, B.GS_TUNE_BF16_TC, B.GS_K_MAS_APPLY_L0, lambda: B.gs_mas_apply(ctx, mas, xr, yr, nrhs=args.nrhs),
                reps=5)
            B.gs_mas_destroy(mas)
        tuned = {k: {"best": v[0], "ms_per_launch": {str(c): round(m, 4) for c, m in v[1].items()}}
                 for k, v in res.items()}
        B.gs_mat_destroy(mat)
        for c in lane_ctx:  # every lane uses the tuned shapes
            for prm in autotune.CANDIDATES:
                B.gs_tune_set(c, prm, B.gs_tune_get(ctx, prm))
    if args.set_tune:  # forced shapes, on every context
        from paper_2411_06224_gb300 import autotune

        by_name = {v: k for k, v in autotune.NAMES.items()}
        for item in args.set_tune:
            name, value = item.split("=")
            for c in {id(c): c for c in [ctx] + lane_ctx}.values():
                B.gs_tune_set(c, by_name[name], int(value))

    # warm-up
    for _ in range(args.warmup):  # with the queue its own lanes, so --streams may differ from the systems
        warm = queue(1, list(range(len(dsys))), solve_job) if (n_lanes > 1 and args.queue) else step()
    iters = [[int(v) for v in o[0]] for o in warm]
    # the queue takes a step's systems longest first (by the warm-up's iterations)
    order = sorted(range(len(dsys)), key=lambda si: -max(iters[si]))
    use_queue = n_lanes > 1 and args.queue
    nnzb = warm[0][2][0]
    mas_levels = warm[0][2][1]
    # per-class breakdown of one step, the systems one after another on the
    # main context (isolated kernel times; outside the timed region)
    B.gs_profile_begin(ctx, range(B.GS_K_COUNT))
    for s in dsys:
        solve_one(s["rows"], s["cols"], s["blocks"], b, x)
    launches_1, ms_1 = B.gs_profile_end(ctx)

    # timed region: the dominant kernels are bracketed by CUDA events on the library's stream
    timed_classes = [B.GS_K_MAS_APPLY_L0, B.GS_K_SPMV]
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    profile_begin(timed_classes)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    e0.record(stream)
    if use_queue:
        res = queue(args.steps, order, solve_job)
    else:
        for _ in range(args.steps):
            res = step()
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    launches, kms = profile_end()
    barrier()
    clk = clocks.stop()
    from paper_2411_06224_gb300 import replicas

    # independent replicas: every rank solved its own systems; the slowest rank sets the time
    value, elapsed = replicas.throughput(len(dsys) * args.steps, e0.elapsed_time(e1) / 1e3, dev)

    # true residuals of the last step (checked on the device through the library's SpMV)
    true_rel = []
    if n_lanes > 1:
        x.copy_(lane_xs[last_lane[len(dsys) - 1]][len(dsys) - 1])
    Ax = torch.empty_like(x)
    for s in dsys[-1:]:
        mat = B.gs_assemble(ctx, V, s["rows"], s["cols"], s["blocks"])
        B.gs_spmv(ctx, mat, x, Ax, nrhs=args.nrhs, variant=B.GS_SPMV_ROW)
        true_rel = ((b - Ax).norm(dim=1) / b.norm(dim=1)).tolist()
        B.gs_mat_destroy(mat)

    # end-to-end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        hsys = [dict(rows=torch.as_tensor(s.rows).pin_memory(), cols=torch.as_tensor(s.cols).pin_memory(),
                     blocks=torch.as_tensor(np.ascontiguousarray(s.blocks.reshape(-1, 3, 3))).pin_memory())
                for s in systems]
        hb = torch.as_tensor(b_host).pin_memory()
        hx = torch.empty_like(hb).pin_memory()
        h2d = sum(h["rows"].nbytes + h["cols"].nbytes + h["blocks"].nbytes + hb.nbytes for h in hsys)
        d2h = hx.nbytes * len(hsys)
        barrier()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        hxs = [[torch.empty_like(hb).pin_memory() for _ in hsys] for _ in range(n_lanes)]

        def e2e_one(i, si, c):  # lane i, system si
            h = hsys[si]
            rows = h["rows"].to(dev, non_blocking=True)
            cols = h["cols"].to(dev, non_blocking=True)
            blocks = h["blocks"].to(dev, non_blocking=True)
            bb = hb.to(dev, non_blocking=True)
            xx = torch.empty_like(bb)
            solve_one(rows, cols, blocks, bb, xx, c)
            hxs[i][si].copy_(xx, non_blocking=True)
            torch.cuda.current_stream().synchronize()  # the host holds the answer

        f0.record(stream)
        if use_queue:
            queue(args.e2e_steps, order, lambda i, si: e2e_one(i, si, lane_ctx[i]))
        else:
            for _ in range(args.e2e_steps):
                if n_lanes == 1:
                    for si in range(len(hsys)):
                        e2e_one(0, si, ctx)
                else:
                    fork()
                    futs = [pool.submit(lane_run, i, lambda i: e2e_one(i, i, lane_ctx[i])) for i in range(len(hsys))]
                    [f.result() for f in futs]
                    join()
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_rate, el = replicas.throughput(len(hsys) * args.e2e_steps, f0.elapsed_time(f1) / 1e3, dev)
        e2e = {"value": e2e_rate, "unit": "Newton solves/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # the mixed-precision forms on the same workload and right-hand sides:
    #   f64_pcg_f32_mas   FP64 PCG, MAS inverses stored and applied in FP32
    #   f64_pcg_bf16_mas  FP64 PCG, BF16 level-0 inverse Cholesky factors on the tensor cores
    #   f32_inner_pcg     FP32 PCG (FP32 SpMV + FP32 MAS) with FP64 reliable updates
    mixed = None
    if args.mixed_steps > 0 and args.nrhs <= 8:
        x_fp64 = x.clone()  # FP64 solution of the last system (last timed step)
        variants = [("f64_pcg_f32_mas", B.GS_PREC_FP32, False), ("f64_pcg_bf16_mas", B.GS_PREC_BF16, False),
                    ("f32_inner_pcg", B.GS_PREC_FP32, True)]
        mixed = {}
        def run_variant(vprec, inner32):
            def mixed_one(s):
                mat = B.gs_assemble(ctx, V, s["rows"], s["cols"], s["blocks"])
                mas = B.gs_build_mas(ctx, mat, shared["map"], ndom, shared["adj_ptr"], shared["adj"],
                                     shared["contacts"], domain_size=N, max_levels=L, precision=vprec)
                try:
                    if inner32:
                        it, rel, outer, _ = B.gs_pcg_solve_mixed(ctx, mat, mas, b, x, nrhs=args.nrhs, tol=TOL,
                                                                 max_iter=20000)
                    else:
                        it, rel, _ = B.gs_pcg_solve(ctx, mat, mas, b, x, nrhs=args.nrhs, tol=TOL, max_iter=20000,
                                                    variant=variant)
                        outer = None
                finally:
                    B.gs_mas_destroy(mas)
                    B.gs_mat_destroy(mat)
                return [int(v) for v in it], [float(v) for v in rel], outer

            for s in dsys:  # warm-up, one solve per system
                mixed_one(s)
            barrier()
            torch.cuda.synchronize()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            mres = []
            for _ in range(args.mixed_steps):
                mres = [mixed_one(s) for s in dsys]
            g1.record(stream)
            torch.cuda.synchronize()
            mrate, mel = replicas.throughput(len(dsys) * args.mixed_steps, g0.elapsed_time(g1) / 1e3, dev)
            # true residuals of the last system, recomputed in FP64 through the library's SpMV
            s = dsys[-1]
            mat = B.gs_assemble(ctx, V, s["rows"], s["cols"], s["blocks"])
            B.gs_spmv(ctx, mat, x, Ax, nrhs=args.nrhs, variant=B.GS_SPMV_ROW)
            B.gs_mat_destroy(mat)
            return {
                "value": mrate, "unit": "Newton solves/s", "ms_per_step": mel / args.mixed_steps * 1e3,
                "steps": args.mixed_steps,
                "iterations": [r[0] for r in mres], "outer_steps": [r[2] for r in mres],
                "true_rel_residual_last_system": ((b - Ax).norm(dim=1) / b.norm(dim=1)).tolist(),
                # both solves stop on the 1e-6 residual test; their distance (last system)
                "rel_error_vs_fp64_max": float(((x - x_fp64).norm(dim=1) / x_fp64.norm(dim=1)).max()),
            }

        for name, vprec, inner32 in variants:
            try:
                mixed[name] = run_variant(vprec, inner32)
            except B.GsError as e:  # a form that fails is reported; the main measurement stands
                mixed[name] = {"error": str(e)[:300]}

    # the precision forms on a stiff cloth sheet (the paper's strain-limited cloth:
    # cubic strain limiting with E = 1e8, 512 x 512 vertices, 4 RHS): FP64 PCG
    # with the FP64 / FP32 / BF16 preconditioner, time per solve and the
    # distance of each answer from the FP64 one
    cloth = None
    if args.cloth > 0:
        from synth.cloth import make_cloth_system

        cs = make_cloth_system(args.cloth, seed=1003 + rank)
        Vc, nrc = cs.n_vertices, 4
        cmap, cnd = B.gs_partition(cs.X, N)
        cd = dict(rows=t(cs.rows, torch.int32), cols=t(cs.cols, torch.int32),
                  blocks=t(cs.blocks.reshape(-1, 3, 3), torch.float64), map=t(cmap, torch.int32),
                  adj_ptr=t(cs.adj_ptr, torch.int32), adj=t(cs.adj, torch.int32))
        cb = t(np.stack([np.random.default_rng(2000 + k).normal(size=3 * Vc) for k in range(nrc)]), torch.float64)
        cloth = {"workload": f"cloth {args.cloth}x{args.cloth} ({Vc} vertices, {cs.rows.size} triplets), strain "
                             f"limiting E=1e8, {nrc} RHS, 3-level MAS N=32, FP64 PCG tol 1e-6"}
        xc64 = None
        for name, cprec in (("fp64", B.GS_PREC_FP64), ("fp32", B.GS_PREC_FP32), ("bf16", B.GS_PREC_BF16)):
            def csolve():
                mat = B.gs_assemble(ctx, Vc, cd["rows"], cd["cols"], cd["blocks"])
                mas = B.gs_build_mas(ctx, mat, cd["map"], cnd, cd["adj_ptr"], cd["adj"], None, domain_size=N,
                                     max_levels=L, precision=cprec)
                xc = torch.zeros_like(cb)
                try:
                    it, _, _ = B.gs_pcg_solve(ctx, mat, mas, cb, xc, nrhs=nrc, tol=TOL, max_iter=20000)
                    Ac = torch.empty_like(xc)
                    B.gs_spmv(ctx, mat, xc, Ac, nrhs=nrc)
                    true = ((cb - Ac).norm(dim=1) / cb.norm(dim=1)).max().item()
                finally:
                    B.gs_mas_destroy(mas)
                    B.gs_mat_destroy(mat)
                return it, true, xc

            try:
                csolve()  # warm-up
                torch.cuda.synchronize()
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                it, true, xc = csolve()
                c1.record(stream)
                torch.cuda.synchronize()
                row = {"ms_per_solve": c0.elapsed_time(c1), "iterations": [int(v) for v in it],
                       "true_rel_residual_max": true}
                if name == "fp64":
                    xc64 = xc
                else:
                    row["rel_error_vs_fp64_max"] = float(((xc - xc64).norm(dim=1) / xc64.norm(dim=1)).max())
                cloth[name] = row
            except B.GsError as e:
                cloth[name] = {"error": str(e)[:300]}

    # the batched form: 64 independent uneven tet cubes (1k-50k vertices, E 1e5-1e9,
    # contacts on 5% of the vertices), one RHS each, solved as one block-diagonal
    # batch with one PCG recurrence per system and the loop in one CUDA graph;
    # compared with solving the same systems one after another on the plain path
    batched = None
    if args.batch_steps > 0:
        from synth.workloads import uneven_batch

        bt = uneven_batch(64, seed=1004 + rank)
        Vb = bt.n_vertices
        bmap, bnd = B.gs_partition_batch(bt.X, bt.node_off, N)  # once per mesh set, before timing
        bd = dict(rows=t(bt.rows, torch.int32), cols=t(bt.cols, torch.int32),
                  blocks=t(bt.blocks.reshape(-1, 3, 3), torch.float64), map=t(bmap, torch.int32),
                  adj_ptr=t(bt.adj_ptr, torch.int32), adj=t(bt.adj, torch.int32), contacts=t(bt.contacts, torch.int32))
        bb = t(rhs_batch := np.random.default_rng(3000 + rank).normal(size=3 * Vb), torch.float64)
        bx = torch.zeros_like(bb)

        def batch_solve(prec_b):
            mat = B.gs_assemble(ctx, Vb, bd["rows"], bd["cols"], bd["blocks"])
            mas = B.gs_build_mas(ctx, mat, bd["map"], bnd, bd["adj_ptr"], bd["adj"], bd["contacts"],
                                 domain_size=N, max_levels=L, precision=prec_b)
            it, rel, _ = B.gs_pcg_solve_batch(ctx, mat, mas, bt.node_off, bb, bx, tol=TOL, max_iter=20000,
                                              use_graph=True)
            B.gs_mas_destroy(mas)
            B.gs_mat_destroy(mat)
            return it, rel

        def timed(fn, steps):
            fn()  # warm-up
            torch.cuda.synchronize()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            out = None
            for _ in range(steps):
                out = fn()
            q1.record(stream)
            torch.cuda.synchronize()
            return q0.elapsed_time(q1) / 1e3 / steps, out

        tb64, (it64, rel64) = timed(lambda: batch_solve(B.GS_PREC_FP64), args.batch_steps)
        tb32, (it32, rel32) = timed(lambda: batch_solve(B.GS_PREC_FP32), args.batch_steps)
        # the same 64 systems one at a time on the plain path
        seq = []
        for si, sysb in enumerate(bt.systems):
            Vs = sysb.n_vertices
            mps, nds = B.gs_partition(sysb.X, N)
            seq.append((Vs, t(sysb.rows, torch.int32), t(sysb.cols, torch.int32),
                        t(sysb.blocks.reshape(-1, 3, 3), torch.float64), t(mps, torch.int32), nds,
                        t(sysb.adj_ptr, torch.int32), t(sysb.adj, torch.int32), t(sysb.contacts, torch.int32),
                        t(rhs_batch[3 * bt.node_off[si]:3 * bt.node_off[si + 1]], torch.float64)))

        def sequential():
            for (Vs, r_, c_, bl_, mp_, nd_, ap_, aj_, ct_, b_) in seq:
                mat = B.gs_assemble(ctx, Vs, r_, c_, bl_)
                mas = B.gs_build_mas(ctx, mat, mp_, nd_, ap_, aj_, ct_, domain_size=N, max_levels=L)
                xs = torch.empty_like(b_)
                B.gs_pcg_solve(ctx, mat, mas, b_, xs, nrhs=1, tol=TOL, max_iter=20000)
                B.gs_mas_destroy(mas)
                B.gs_mat_destroy(mat)

        tseq, _ = timed(sequential, 1)
        batched = {
            "workload": "64 tet cubes, vertices log-uniform 1k-50k (%d total), E log-uniform 1e5-1e9, contacts on 5%% of "
                        "vertices, 1 RHS each, 3-level MAS N=32, tol 1e-6" % Vb,
            "fp64": {"value": 64 / tb64, "unit": "Newton solves/s", "ms_per_batch": tb64 * 1e3,
                     "max_iterations": int(max(it64)), "true_rel_residual_max": float(max(rel64))},
            "fp32_preconditioner": {"value": 64 / tb32, "unit": "Newton solves/s", "ms_per_batch": tb32 * 1e3,
                                    "max_iterations": int(max(it32))},
            "sequential_plain_fp64": {"value": 64 / tseq, "unit": "Newton solves/s", "ms_for_64": tseq * 1e3},
            "graph": "whole PCG loop = one CUDA graph launch (conditional WHILE node)",
        }

    # roofline of the dominant kernel class
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_mhz_max = (clk or {}).get("sm_max_mhz") or 2070.0
    fp64_peak_tflops = sms * FP64_FMA_PER_CLK_PER_SM * 2 * sm_mhz_max * 1e6 / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    ld = 3 * N
    n_dom0 = ndom
    real0 = np.bincount(mp // N, minlength=n_dom0)
    apply_flops = 2.0 * float(np.sum((3 * real0) ** 2)) * args.nrhs
    inv_bytes = (8 if prec == B.GS_PREC_FP64 else 4) * n_dom0 * ld * ld
    apply_bytes = inv_bytes + 2 * 8 * 3 * V * args.nrhs
    n_off = nnzb - V
    spmv_flops = args.nrhs * (18.0 * V + 36.0 * n_off)
    spmv_bytes = 76.0 * nnzb + 4.0 * (V + 1) + 2 * 8 * 3 * V * args.nrhs
    k_apply = launches[B.GS_K_MAS_APPLY_L0]
    k_spmv = launches[B.GS_K_SPMV]
    t_apply = kms[B.GS_K_MAS_APPLY_L0] / 1e3 / max(k_apply, 1)
    t_spmv = kms[B.GS_K_SPMV] / 1e3 / max(k_spmv, 1)
    # the same kernels timed alone (the sequential per-class step): with the
    # systems on concurrent streams, the live durations include the overlap
    t_apply_iso = ms_1[B.GS_K_MAS_APPLY_L0] / 1e3 / max(launches_1[B.GS_K_MAS_APPLY_L0], 1)
    t_spmv_iso = ms_1[B.GS_K_SPMV] / 1e3 / max(launches_1[B.GS_K_SPMV], 1)

    def fp64_line(flops, nbytes, tsec, traffic):
        return {"bound": "alu", "achieved": flops / tsec / 1e12, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": flops / tsec / 1e12 / fp64_peak_tflops, "traffic": traffic,
                "hbm_gbs": nbytes / tsec / 1e9, "hbm_frac": nbytes / tsec / 1e9 / hbm,
                "flops_per_launch": flops, "bytes_per_launch": nbytes, "avg_launch_ms": tsec * 1e3}

    f64tc = (prec == B.GS_PREC_FP64 and args.nrhs <= 8 and ld % 16 == 0
             and B.gs_tune_get(ctx, B.GS_TUNE_F64_TC) == 1)
    if f64tc:
        # FP64-accurate apply on the BF16 tensor cores: the 7 BF16 digit matrices
        # of every level-0 inverse (14 B per entry) stream from HBM once per apply,
        # plus r read and z written (FP64), plus the coarse z read once per node
        dig_bytes = 7 * 2 * n_dom0 * ld * ld
        tc_bytes = dig_bytes + 2 * 8 * 3 * V * args.nrhs
        traffic = (F64TC_DRAM_BYTES_PER_DOMAIN_8RHS * n_dom0
                   if args.nrhs == 8 and N == 32 and F64TC_DRAM_BYTES_PER_DOMAIN_8RHS else None)
        apply_line = {"bound": "hbm", "achieved": tc_bytes / t_apply / 1e9, "peak": hbm, "unit": "GB/s",
                      "frac": tc_bytes / t_apply / 1e9 / hbm, "traffic": traffic,
                      "fp64_equivalent_tflops": apply_flops / t_apply / 1e12,
                      "fp64_equivalent_frac_of_fp64_peak": apply_flops / t_apply / 1e12 / fp64_peak_tflops,
                      "flops_per_launch": apply_flops, "bytes_per_launch": tc_bytes, "avg_launch_ms": t_apply * 1e3,
                      "kernel": "k_level0_f64tc (level-0 MAS apply in FP64 accuracy by exact BF16 digit "
                                "splitting on tcgen05, + prolongation)"}
    else:
        traffic = (APPLY_DRAM_BYTES_PER_DOMAIN_8RHS * n_dom0
                   if args.nrhs == 8 and prec == B.GS_PREC_FP64 and N == 32
                   and B.gs_tune_get(ctx, B.GS_TUNE_APPLY_RHS) == 4 else None)  # the captured shape
        apply_line = fp64_line(apply_flops, apply_bytes, t_apply, traffic)
        apply_line["kernel"] = (f"k_domain_product<double,{B.gs_tune_get(ctx, B.GS_TUNE_APPLY_RHS)},1> "
                                "(level-0 MAS apply + prolongation)")
    spmv_ws = args.spmv in ("row", "ff") and B.gs_tune_get(ctx, B.GS_TUNE_SPMV_WS) == 1
    if args.spmv == "ff":
        # float-float on the FP32 units: 12 FP32 instructions per term (exact
        # product, two-sum, small parts), 9 terms per block use and RHS, one use
        # per diagonal block and two per off-diagonal block
        ff_inst = args.nrhs * 9 * 12.0 * (V + 2.0 * n_off)
        fp32_peak = sms * 128 * sm_mhz_max * 1e6 / 1e12  # T FP32 instructions/s
        spmv_line = {"bound": "alu", "achieved": ff_inst / t_spmv / 1e12, "peak": fp32_peak,
                     "unit": "T FP32 instructions/s", "frac": ff_inst / t_spmv / 1e12 / fp32_peak, "traffic": None,
                     "hbm_gbs": spmv_bytes / t_spmv / 1e9, "hbm_frac": spmv_bytes / t_spmv / 1e9 / hbm,
                     "fp64_equivalent_tflops": spmv_flops / t_spmv / 1e12,
                     "fp64_equivalent_frac_of_fp64_peak": spmv_flops / t_spmv / 1e12 / fp64_peak_tflops,
                     "instructions_per_launch": ff_inst, "flops_per_launch": spmv_flops,
                     "bytes_per_launch": spmv_bytes, "avg_launch_ms": t_spmv * 1e3}
        spmv_line["kernel"] = "k_spmv_ff_ws" if spmv_ws else "k_spmv_ff_row"
        spmv_line["isolated"] = {"avg_launch_ms": t_spmv_iso * 1e3,
                                 "achieved": ff_inst / t_spmv_iso / 1e12,
                                 "frac": ff_inst / t_spmv_iso / 1e12 / fp32_peak,
                                 "hbm_frac": spmv_bytes / t_spmv_iso / 1e9 / hbm}
    else:
        spmv_traffic = (SPMV_WS_DRAM_BYTES_64.get(B.gs_tune_get(ctx, B.GS_TUNE_SPMV_LANES))
                        if spmv_ws and args.grid == 64 and args.nrhs == 8
                        and B.gs_tune_get(ctx, B.GS_TUNE_SPMV_WINDOW) == 1024 else None)  # the captured shapes
        spmv_line = fp64_line(spmv_flops, spmv_bytes, t_spmv, spmv_traffic)
        spmv_line["kernel"] = "k_spmv_row_ws" if spmv_ws else f"k_spmv_{args.spmv}"
        # alone: the same arithmetic over the sequential step's durations
        spmv_line["isolated"] = {"avg_launch_ms": t_spmv_iso * 1e3,
                                 "achieved": spmv_flops / t_spmv_iso / 1e12,
                                 "frac": spmv_flops / t_spmv_iso / 1e12 / fp64_peak_tflops}
    apply_iso_ach = (tc_bytes / t_apply_iso / 1e9) if f64tc else (apply_flops / t_apply_iso / 1e12)
    apply_line["isolated"] = {"avg_launch_ms": t_apply_iso * 1e3, "achieved": apply_iso_ach,
                              "frac": apply_iso_ach / apply_line["peak"]}
    for ln in (apply_line, spmv_line):
        ln["concurrent_streams"] = n_lanes
    dominant = apply_line if kms[B.GS_K_MAS_APPLY_L0] >= kms[B.GS_K_SPMV] else spmv_line
    mine = int(sum(launches[k] for k in range(B.GS_K_COUNT) if k != B.GS_K_LIBPRIM))

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "Newton solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec == B.GS_PREC_FP64 else "f64+f32-precond",
        "data": "synthetic",
        "config": {
            "workload": f"tet cube {args.grid}^3 stiffness sweep E=1e5,1e7,1e9; {len(systems[0].contacts)} contacts; "
                        f"{args.nrhs} RHS; 3-level MAS N=32; PCG tol 1e-6",
            "vertices": V, "dof": 3 * V, "triplets_per_system": int(systems[0].rows.size), "stored_blocks": int(nnzb),
            "mas_levels": mas_levels[1], "nrhs": args.nrhs, "spmv": args.spmv, "precision": args.precision,
            "pcg_iterations": iters, "true_rel_residual_last_system": true_rel,
            "l2": "inputs larger than L2 (1.07 GB of triplets and 0.6 GB of level-0 inverses per system vs 129 MB L2); no flush",
            "parallelism": f"independent systems per GPU x{world}",
            "schedule": (f"one queue over the timed steps' {len(dsys)} x steps solves on {n_lanes} streams, "
                         "each step's systems longest first" if use_queue else
                         (f"{n_lanes} streams, one system each, synchronised per step" if n_lanes > 1
                          else "one stream, systems one after another")),
            "launch_shapes": autotune_current(B, ctx),
            "autotune": tuned,
        },
        "roofline": dominant,
        "kernels": {"mas_apply_l0": apply_line, "spmv": spmv_line,
                    "spmv_hbm_gbs": spmv_line["hbm_gbs"]},
        "phase_ms_one_step": {B.K_NAMES[k]: float(ms_1[k]) for k in range(B.GS_K_COUNT)},
        "launches_one_step": {B.K_NAMES[k]: int(launches_1[k]) for k in range(B.GS_K_COUNT)},
        "e2e": e2e,
        "forms": {"mixed_precision": mixed, "batched": batched, "precision_cloth": cloth},
        "clocks": clk,
        "gpu_launches": mine,
        "libprim_calls": int(launches[B.GS_K_LIBPRIM]),
        "wall_s": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            smp = run_oracle_sample(args.grid, [1e5], 1)[0]
            mean_iters = float(np.mean([sum(i) for i in iters]))
            rate, tsolve = oracle_rate(smp, mean_iters)
            line["cpu_baseline"] = {
                "value": rate, "unit": "Newton solves/s", "cores": 1, "kind": "oracle",
                "sample": (f"FP64 numpy/scipy oracle, single thread, on the E=1e5 system: full assembly "
                           f"({smp['t_ga']:.1f} s), full 3-level MAS build ({smp['t_pa']:.1f} s), {smp['k']} PCG "
                           f"iterations on 1 RHS ({smp['t_iter']:.3f} s each); solve time extrapolated with the "
                           f"GPU run's mean PCG iterations summed over the {args.nrhs} RHS ({mean_iters:.0f})"),
            }
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline"] = {"value": None, "error": str(e)[:300]}
    B.gs_destroy(ctx)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def micro(args):
    """The paper's microbenchmarks, one JSON line.

    reduce: 2^24 3x3 blocks with sorted keys, every key repeated 2^d times;
      the paper's FastHashReduction against the CUB library's ReduceByKey on
      the same sorted input (both gather nothing; inputs resident in HBM).
    spmv: random symmetric patterns, 2^18 block rows with about b blocks per
      full row (diagonal plus (b-1)/2 random upper blocks per row); the
      paper's symmetric storage with atomic scatter (SRBK), the row-gather
      over the same storage, and the cuSPARSE library's BSR SpMV on the full
      matrix; one right-hand side."""
    import numpy as np
    import torch

    from paper_2411_06224_gb300.build import build

    build()
    from paper_2411_06224_gb300 import binding as B

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = B.gs_create(0, torch.cuda.current_stream())
    gen = torch.Generator(device=dev).manual_seed(1007)
    out = {"metric": "microbenchmarks", "config": {"workload": "paper reduction / SpMV microbenchmarks"}}
    nb = 1 << 24
    blocks = torch.randn((nb, 3, 3), dtype=torch.float64, device=dev, generator=gen)
    red = []
    for d in (0, 1, 2, 4, 7, 10, 13, 16):
        keys = torch.arange(nb, device=dev, dtype=torch.int64) >> d
        row = {"dup": 1 << d}
        for method, name in ((0, "fast_hash_reduction"), (1, "cub_reduce_by_key")):
            times = []
            for _ in range(4):
                o, ms = B.gs_micro_segment_reduce(ctx, keys, blocks, method)
                times.append(ms)
            t_ms = float(np.median(times[1:]))
            u = o.shape[0]
            row[name] = {"ms": t_ms, "gbs": (nb * 80 + u * 72) / t_ms / 1e6}
        row["speedup"] = row["cub_reduce_by_key"]["ms"] / row["fast_hash_reduction"]["ms"]
        red.append(row)
        del keys
    del blocks
    out["reduce_16M_blocks"] = red
    n = 1 << 18
    sp = []
    for bpr in (1, 2, 4, 8, 16, 32, 64):
        m = (bpr - 1) / 2.0
        k_off = int(round(m * n))
        r_off = torch.randint(0, n - 1, (k_off,), device=dev, generator=gen)
        span = (n - 1 - r_off).to(torch.float64)
        c_off = r_off + 1 + (torch.rand(k_off, device=dev, generator=gen, dtype=torch.float64) * span).long()
        rows = torch.cat([torch.arange(n, device=dev), r_off]).int()
        cols = torch.cat([torch.arange(n, device=dev), c_off]).int()
        vals = torch.randn((rows.numel(), 3, 3), dtype=torch.float64, device=dev, generator=gen)
        mat = B.gs_assemble(ctx, n, rows, cols, vals)
        _, nnzb = B.gs_mat_info(mat)
        x = torch.randn((1, 3 * n), dtype=torch.float64, device=dev, generator=gen)
        y = torch.empty_like(x)
        row = {"blocks_per_full_row": bpr, "upper_blocks": int(nnzb)}
        for variant, name in ((B.GS_SPMV_SRBK, "srbk_symmetric"), (B.GS_SPMV_ROW, "row_gather_symmetric")):
            B.gs_spmv(ctx, mat, x, y, nrhs=1, variant=variant)
            B.gs_profile_begin(ctx, [B.GS_K_SPMV])
            for _ in range(10):
                B.gs_spmv(ctx, mat, x, y, nrhs=1, variant=variant)
            launches, kms = B.gs_profile_end(ctx)
            row[name] = {"ms": float(kms[B.GS_K_SPMV] / max(launches[B.GS_K_SPMV], 1))}
        rid, cid, au = B.gs_mat_export(ctx, mat)
        off = rid != cid
        fr = torch.cat([rid, cid[off]]).long()
        fc = torch.cat([cid, rid[off]]).long()
        fa = torch.cat([au, au[off].transpose(1, 2)])
        order = torch.argsort(fr * n + fc)
        fr, fc, fa = fr[order], fc[order], fa[order].contiguous()
        ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
        ptr[1:] = torch.cumsum(torch.bincount(fr, minlength=n), 0)
        yf = torch.empty(3 * n, dtype=torch.float64, device=dev)
        B.gs_micro_bsr_spmv_cusparse(ctx, n, ptr.int(), fc.int(), fa, x[0].contiguous(), yf, reps=2)
        ms = B.gs_micro_bsr_spmv_cusparse(ctx, n, ptr.int(), fc.int(), fa, x[0].contiguous(), yf, reps=10)
        row["cusparse_bsr_full"] = {"ms": ms, "full_blocks": int(fc.numel())}
        row["max_rel_diff_vs_row_gather"] = float((yf - y[0]).abs().max() / y[0].abs().max())
        for name in ("srbk_symmetric", "row_gather_symmetric", "cusparse_bsr_full"):
            # algorithmic bytes of the symmetric storage: 76 B per stored block + 48 B per row
            row[name]["gbs_symmetric_bytes"] = (nnzb * 76 + n * 48) / row[name]["ms"] / 1e6
            row[name]["gflops"] = (2 * 9 * (2 * nnzb - n)) / row[name]["ms"] / 1e6
        sp.append(row)
        B.gs_mat_destroy(mat)
    out["spmv_random_2p18_rows"] = sp
    B.gs_destroy(ctx)
    print(json.dumps(out), flush=True)


def reference_arm(args, rank, world):
    """The oracle timed on the host cores (rank 0 only), same metric and workload."""
    if rank != 0:
        return
    import json as _json

    golden = os.path.join(ROOT, "tests", "golden", "sweep64_pcg_iterations.json")
    iters = None
    if os.path.exists(golden):
        g = _json.load(open(golden))
        iters = float(sum(sum(v) for v in g["iterations"].values()) / len(g["iterations"]))
    Es = (1e5, 1e7, 1e9)
    allv = run_oracle_sample(args.grid, Es, args.warmup + args.steps, iters=2)
    vals = allv[args.warmup:] or allv[-1:]
    n_it = iters if iters is not None else 8 * 150.0
    rates = [oracle_rate(v, n_it)[0] for v in vals]
    value = statistics.mean(rates)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "Newton solves/s",
        "n_gpus": world,
        "steps": len(vals),
        "warmup": args.warmup,
        "ms_per_step": 1e3 / value,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"tet cube {args.grid}^3 stiffness sweep E=1e5,1e7,1e9; 8 RHS; 3-level MAS N=32; PCG tol 1e-6"},
        "cpu_baseline": {"value": value, "unit": "Newton solves/s", "cores": 1, "kind": "oracle",
                         "sample": ("FP64 numpy/scipy oracle, single thread: per step full assembly + full MAS build "
                                    "+ 2 PCG iterations on 1 RHS of one system (E cycles 1e5, 1e7, 1e9); solve time "
                                    "extrapolated with the oracle's own iteration counts summed over 8 RHS "
                                    + ("(tests/golden/sweep64_pcg_iterations.json)" if iters else "(assumed 150 per RHS)"))},
        "e2e": {"value": value, "unit": "Newton solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
