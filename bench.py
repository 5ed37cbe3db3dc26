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
TOL = 1e-6
METRIC = "Newton solves/s to 1e-6 rel. residual (FP64 MAS-PCG)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=64, help="vertices per cube edge (64 = the named workload)")
    p.add_argument("--nrhs", type=int, default=8)
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--spmv", default="row", choices=["row", "srbk"])
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
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
def make_workload(grid, nrhs, rank):
    import numpy as np

    from synth.workloads import rhs, stiffness_sweep

    systems = stiffness_sweep(n=grid, seed=1002 + rank)
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
    systems, b_host = make_workload(args.grid, args.nrhs, rank)
    V = systems[0].n_vertices
    N, L = 32, 3
    prec = B.GS_PREC_FP32 if args.precision == "fp32" else B.GS_PREC_FP64
    variant = B.GS_SPMV_ROW if args.spmv == "row" else B.GS_SPMV_SRBK
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

    def solve_one(rows, cols, blocks, bb, xx):
        mat = B.gs_assemble(ctx, V, rows, cols, blocks)
        mas = B.gs_build_mas(ctx, mat, shared["map"], ndom, shared["adj_ptr"], shared["adj"], shared["contacts"],
                             domain_size=N, max_levels=L, precision=prec)
        it, rel, _ = B.gs_pcg_solve(ctx, mat, mas, bb, xx, nrhs=args.nrhs, tol=TOL, max_iter=20000, variant=variant)
        info = (B.gs_mat_info(mat)[1], B.gs_mas_info(mas))
        B.gs_mas_destroy(mas)
        B.gs_mat_destroy(mat)
        return it, rel, info

    def step():
        out = []
        for s in dsys:
            out.append(solve_one(s["rows"], s["cols"], s["blocks"], b, x))
        return out

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    for _ in range(args.warmup):
        warm = step()
    iters = [[int(v) for v in o[0]] for o in warm]
    nnzb = warm[0][2][0]
    mas_levels = warm[0][2][1]
    # per-class breakdown of one step (all classes timed with events; outside the timed region)
    B.gs_profile_begin(ctx, range(B.GS_K_COUNT))
    step()
    launches_1, ms_1 = B.gs_profile_end(ctx)

    # timed region: the dominant kernels are bracketed by CUDA events on the library's stream
    timed_classes = [B.GS_K_MAS_APPLY_L0, B.GS_K_SPMV]
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    B.gs_profile_begin(ctx, timed_classes)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        res = step()
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    launches, kms = B.gs_profile_end(ctx)
    barrier()
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    if world > 1:
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    solves = len(dsys) * args.steps * world
    value = solves / elapsed

    # true residuals of the last step (checked on the device through the library's SpMV)
    true_rel = []
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
        f0.record(stream)
        for _ in range(args.e2e_steps):
            for h in hsys:
                rows = h["rows"].to(dev, non_blocking=True)
                cols = h["cols"].to(dev, non_blocking=True)
                blocks = h["blocks"].to(dev, non_blocking=True)
                bb = hb.to(dev, non_blocking=True)
                xx = torch.empty_like(bb)
                solve_one(rows, cols, blocks, bb, xx)
                hx.copy_(xx, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        el = f0.elapsed_time(f1) / 1e3
        if world > 1:
            tt = torch.tensor([el], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = float(tt.item())
        e2e = {"value": len(hsys) * args.e2e_steps * world / el, "unit": "Newton solves/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

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

    def fp64_line(flops, nbytes, tsec, traffic):
        return {"bound": "alu", "achieved": flops / tsec / 1e12, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": flops / tsec / 1e12 / fp64_peak_tflops, "traffic": traffic,
                "hbm_gbs": nbytes / tsec / 1e9, "hbm_frac": nbytes / tsec / 1e9 / hbm,
                "flops_per_launch": flops, "bytes_per_launch": nbytes, "avg_launch_ms": tsec * 1e3}

    apply_line = fp64_line(apply_flops, apply_bytes, t_apply, None)
    apply_line["kernel"] = "k_domain_product<double,4,1> (level-0 MAS apply + prolongation)"
    spmv_line = fp64_line(spmv_flops, spmv_bytes, t_spmv, None)
    spmv_line["kernel"] = f"k_spmv_{args.spmv}"
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
        },
        "roofline": dominant,
        "kernels": {"mas_apply_l0": apply_line, "spmv": spmv_line,
                    "spmv_hbm_gbs": spmv_line["hbm_gbs"]},
        "phase_ms_one_step": {B.K_NAMES[k]: float(ms_1[k]) for k in range(B.GS_K_COUNT)},
        "launches_one_step": {B.K_NAMES[k]: int(launches_1[k]) for k in range(B.GS_K_COUNT)},
        "e2e": e2e,
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
