"""Benchmark: time to 1e-8 relative residual of the multigrid-preconditioned
FGMRES solve of the condensed momentum system on one GB300.

One step = one complete solve (FGMRES(30) + one V(2,2) cycle per iteration,
rtol 1e-8 on the FP64 true residual) of the 2d 256x256 Q1 workload
(198,147 unknowns, 7 levels), V-cycle in FP32, outer FGMRES in FP64.  The
right-hand side is resident in HBM when the timed region starts; the L2 is
flushed (a 256 MB write) before every timed solve, outside the per-solve
events.  The same solve through the C ABI with host buffers gives "e2e"; the
plain FP64 path on the same mesh is timed beside it, both solutions are
compared with the FP64 oracle's, and compact records of the 3d 96^3 workload
and of a serving sample follow on the same line (last, so that they stay in
view at the end of the output).

--impl reference times the FP64 CPU oracle (same method, same workload) on
the host cores instead.  Under torchrun (N > 1) every rank solves its own
copy of the workload (replicas; the path has no exchange step).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-8 rel. residual (mixed vs FP64 MG) and HBM GB/s; p50/p99 latency"
WORKLOADS = {
    # the solid region is read on the coarsest mesh (every level resolves the same interface)
    "cfg2": ("2d 256x256 Q1 condensed-momentum Jacobian (198,147 unknowns), solid x>0.6 read on the coarsest "
             "4x4 mesh (interface x=0.5 on every level), 7 MG levels, V(2,2) Vanka 2x2-cell patches "
             "(27 unknowns), FGMRES(30) rtol 1e-8"),
    "cfg3": ("3d 32^3 Q1 condensed-momentum Jacobian (143,748 unknowns), solid z<0.25 read on the coarsest 4^3 "
             "mesh (interface z=0.25), 4 MG levels, V(2,2) Vanka 2x2x2-cell patches (108 unknowns), "
             "FGMRES(30) rtol 1e-8"),
    "cfg4": ("3d 96^3 Q1 condensed-momentum Jacobian (3,650,692 unknowns), solid z<0.25 read on the coarsest 3^3 "
             "mesh (interface z=1/3), 6 MG levels, V(2,2) Vanka 2x2x2-cell patches (108 unknowns), "
             "FGMRES(30) rtol 1e-8"),
    # the ALE-extension solve (problem (3)) on the same meshes: d displacement components per node
    "ale2": ("2d 256x256 Q1 ALE-extension operator (vector Laplacian on the fluid, 132,098 unknowns), "
             "solid fixed (interface x=0.5), 7 MG levels, V(2,2) Vanka 2x2-cell patches (18 unknowns), "
             "FGMRES(30) rtol 1e-8"),
    "ale3": ("3d 32^3 Q1 ALE-extension operator (vector Laplacian on the fluid, 107,811 unknowns), "
             "solid fixed (interface z=0.25), 4 MG levels, V(2,2) Vanka 2x2x2-cell patches (81 unknowns), "
             "FGMRES(30) rtol 1e-8"),
    "ale4": ("3d 96^3 Q1 ALE-extension operator (vector Laplacian on the fluid, 2,738,019 unknowns), "
             "solid fixed (interface z=1/3), 6 MG levels, V(2,2) Vanka 2x2x2-cell patches (81 unknowns), "
             "FGMRES(30) rtol 1e-8"),
    # a mid-size 3d mesh whose finest patch inverses (645 MB FP32) exceed the L2, for kernel captures
    "3d48": ("3d 48^3 Q1 condensed-momentum Jacobian (470,596 unknowns), solid z<0.25, 4 MG levels, V(2,2) "
             "Vanka 2x2x2-cell patches (108 unknowns), FGMRES(30) rtol 1e-8"),
}
# the mesh each ALE workload shares with a condensed-momentum workload
ALE_BASE = {"ale2": "cfg2", "ale3": "cfg3", "ale4": "cfg4"}


def load_workload(name):
    """The seeded synthetic system of a workload and its unknowns per node."""
    from gen import build_ale_system, build_system, config_problem
    if name in ALE_BASE:
        p = config_problem(ALE_BASE[name])
        return build_ale_system(p), p.dim
    if name == "3d48":
        from gen import Problem
        p = Problem(dim=3, n=(48, 48, 48), levels=4, solid=(2, -1, 0.25))
    else:
        p = config_problem(name)
    return build_system(p), p.dim + 1
# DRAM bytes (read + write) per launch of the roofline kernel, from one ncu
# capture of the current kernel source (profiles/k_vanka_apply_*.md); a
# workload or precision without a capture of the current source reports null.
PROFILED_TRAFFIC = {
    ("cfg2", 1): 48_786_944 + 44_544,       # k_vanka_apply_ring<float,float,2,3,128,2>, 2d 256x256, FP32
    ("cfg3", 1): 191_715_072 + 4_028_672,   # k_vanka_apply_ring<float,float,3,3,128,1>, 3d 32^3, FP32
}
WORKLOAD = "cfg2"
WORKLOAD_DESC = WORKLOADS[WORKLOAD]


def apply_kernel_name(problem, ncomp, precision):
    """The library's finest-level apply kernel: the streaming ring for FP32 and
    BF16 inverses, except 2d extension patches and 3d extension levels of more
    than 4096 patches, which take the warp-per-patch kernel (as FP64 does)."""
    patches = 1
    for c in problem.n[:problem.dim]:
        patches *= c // 2
    lean = ncomp == problem.dim
    ring = precision != 0 and (not lean or (problem.dim == 3 and patches <= 4096))
    return "k_vanka_apply_ring" if ring else "k_vanka_apply"


def workload_config(sysm):
    """The workload as both arms name it (no implementation details)."""
    return {"workload": WORKLOAD_DESC, "unknowns": int(sysm.unknowns), "levels": int(sysm.problem.levels),
            "rtol": 1e-8, "parallelism": "single GPU"}


def sig(v, digits=4):
    """Compact float for the output line (digits significant)."""
    if v is None or isinstance(v, (int, bool, str)):
        return v
    return float(f"{v:.{digits}g}")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nmg", choices=["nmg", "reference"])
    ap.add_argument("--precision", type=int, default=1, help="V-cycle precision: 0 FP64, 1 FP32, 2 BF16")
    ap.add_argument("--no-graph", action="store_true", help="plain launches, host-stepped FGMRES (use_graph 0)")
    ap.add_argument("--graph", type=int, default=2, choices=[0, 1, 2],
                    help="1: V-cycle graphs with host-stepped FGMRES; 2: also one on-device loop per restart cycle")
    ap.add_argument("--engine", default="auto", choices=["auto", "kernels", "persistent", "fused"],
                    help="V-cycle engine (auto: the autotuner picks it on the first solve)")
    ap.add_argument("--tile-patches", type=int, default=0,
                    help="engine kernels: levels with at most this many patches run tile-fused Vanka steps")
    ap.add_argument("--tail-patches", type=int, default=0,
                    help="with --engine kernels/fused: levels with at most this many patches run in the cluster tail")
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU oracle baseline")
    ap.add_argument("--serving", action="store_true",
                    help="serving workload: Poisson stream of solves over resident 2d/3d hierarchies")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--mesh", default=None,
                    help="serving: one mesh only, e.g. 2d:128 or 3d:32 (many right-hand sides on one hierarchy)")
    ap.add_argument("--rhs", type=int, default=8,
                    help="columns of the multi-right-hand-side measurement (nmg_solve_many); 0 skips it")
    ap.add_argument("--batch", type=int, default=0,
                    help="serving: requests on one hierarchy run as columns of a multi-vector solve (up to 8)")
    ap.add_argument("--workspaces", type=int, default=0,
                    help="serving: extra concurrent requests per hierarchy (nmg_server_set_workspaces)")
    ap.add_argument("--profile-range", action="store_true",
                    help="after the warm-up, run one solve between cudaProfilerStart/Stop (for "
                         "ncu --profile-from-start off) and exit")
    ap.add_argument("--profile-many", action="store_true",
                    help="run one 8-column multi-vector V-cycle and one single V-cycle (plain launches) between "
                         "cudaProfilerStart and cudaProfilerStop, then exit (for an ncu launch list)")
    ap.add_argument("--workload", default="cfg2", choices=sorted(WORKLOADS),
                    help="cfg2 is the measured workload; the others are for investigation")
    ap.add_argument("--large-patches", default="none", choices=["none", "solid", "fluid", "all"],
                    help="Vanka patches of 4^d cells on this region (patch-size study); none: 2^d-cell patches")
    ap.add_argument("--no-large", action="store_true", help="omit the compact 3d 96^3 record")
    ap.add_argument("--no-serving-sample", action="store_true", help="omit the compact serving record")
    ap.add_argument("--serving-sample", type=int, default=300, help="requests of the compact serving record")
    return ap.parse_args()


def max_over_ranks(values, dist, device):
    """Element-wise maximum of a list of floats over all ranks (the replicas'
    slowest time is the job's time); identity without a process group."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(world, ms_max):
    """Solves per second of the whole job: every rank solves its own replica."""
    return world * 1000.0 / ms_max


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [v.strip() for v in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ----------------------------------------------------------------------------

CHILD = r"""
import json, os, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from bench import load_workload
from oracle.solver import OracleSolver
s, _ = load_workload({wl!r})
o = OracleSolver(s.levels, s.dirichlet)
times, cpu = [], []
info = None
for _ in range({reps}):
    t, c = time.perf_counter(), time.process_time()
    x, info = o.solve(s.rhs, rtol=1e-8)
    times.append(time.perf_counter() - t)
    cpu.append(time.process_time() - c)
if {save!r}:
    np.save({save!r}, x)
print(json.dumps({{"times": times, "cpu_times": cpu, "iterations": info["iterations"],
                   "rel_residual": info["rel_residual"], "setup_s": o.setup_seconds}}))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle(reps: int, threads: int = 1, save: str = ""):
    """Runs the FP64 oracle solve reps times in a child process (no GPU) with
    the BLAS/OpenMP thread pools capped at threads; save: .npy path for the
    last solution."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, wl=WORKLOAD, reps=reps, save=save)],
                         capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    t0 = time.time()
    sysm, _ = load_workload(WORKLOAD)
    cores = host_cores()
    res = run_oracle(args.warmup + args.steps, threads=cores)
    times = res["times"][args.warmup:]
    ms = 1000.0 * statistics.mean(times)
    eff = sum(res["cpu_times"][args.warmup:]) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(sysm),
        "solver": "FP64 CPU oracle (numpy/scipy), same method",
        "iterations": res["iterations"], "rel_residual": res["rel_residual"],
        "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
                         "effective_cores": sig(eff, 3),
                         "sample": f"{args.steps} full oracle solves of the workload (setup excluded), "
                                   f"BLAS/OpenMP pools of {cores} threads"},
        "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.time() - t0,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def gpu_arm(args):
    import ctypes as C

    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    else:
        dist = None

    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import Session, solve_opts

    sysm, ncomp = load_workload(WORKLOAD)
    stream = torch.cuda.Stream()
    prec_mask = (1 << nmg.NMG_PREC_FP64) | (1 << args.precision)
    S = Session(sysm.problem.dim, sysm.problem.n, [(l.row_ptr, l.col_idx, l.vals) for l in sysm.levels], sysm.dirichlet,
                precisions=prec_mask, stream=stream.cuda_stream, ncomp=ncomp)
    if args.large_patches != "none":
        from gen.q1fsi import solid_cells
        solid = solid_cells(sysm.problem, sysm.problem.n)
        S.set_large_patches({"solid": solid, "fluid": ~solid, "all": np.ones_like(solid)}[args.large_patches])
    n = sysm.unknowns
    b = torch.from_numpy(sysm.rhs).cuda()
    x = torch.empty_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    use_graph = 0 if args.no_graph else args.graph
    engine = {"auto": nmg.NMG_ENGINE_AUTO, "kernels": nmg.NMG_ENGINE_KERNELS,
              "persistent": nmg.NMG_ENGINE_PERSISTENT, "fused": nmg.NMG_ENGINE_FUSED}[args.engine]

    def timed_solves(prec, k, graph, profile=0, engine=engine):
        times, infos = [], []
        if profile:
            nmg.check(nmg.nmg_profile_enable(S.handle, profile))
        with torch.cuda.stream(stream):
            for _ in range(k):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = S.solve(b, x, precision=prec, use_graph=graph, engine=engine, tail_patches=args.tail_patches,
                                tile_patches=args.tile_patches)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                infos.append(info)
                if profile:   # drain the library's event pool after every solve: every launch is counted
                    nmg.check(nmg.nmg_profile_read(S.handle, None, None, None))
        prof = None
        if profile:
            import ctypes as C
            ms, cnt, bpl = C.c_double(), C.c_int64(), C.c_double()
            nmg.check(nmg.nmg_profile_read(S.handle, ms, cnt, bpl))
            nmg.check(nmg.nmg_profile_enable(S.handle, 0))
            prof = (ms.value, cnt.value, bpl.value)
        return times, infos, prof

    if args.profile_many:
        K = 8
        R = torch.from_numpy(np.tile(sysm.rhs.astype(np.float32), (K, 1))).cuda()
        Z = torch.zeros_like(R)
        z1 = torch.zeros_like(R[0])
        om = solve_opts(precision=args.precision, use_graph=0)
        o1 = solve_opts(precision=args.precision, use_graph=0, engine=nmg.NMG_ENGINE_KERNELS)
        for _ in range(max(1, args.warmup)):
            nmg.check(nmg.nmg_vcycle_many(S.handle, om, K, R, Z))
            nmg.check(nmg.nmg_vcycle(S.handle, o1, R[0], z1))
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        nmg.check(nmg.nmg_vcycle_many(S.handle, om, K, R, Z))
        nmg.check(nmg.nmg_vcycle(S.handle, o1, R[0], z1))
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        if rank == 0:
            print(json.dumps({"profile_many": WORKLOAD, "columns": K}), flush=True)
        return

    # warm-up (also captures the V-cycle graphs)
    timed_solves(args.precision, args.warmup, use_graph)
    if args.profile_range:
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            info = S.solve(b, x, precision=args.precision, use_graph=use_graph, engine=engine,
                           tail_patches=args.tail_patches, tile_patches=args.tile_patches)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        if rank == 0:
            print(json.dumps({"profile_range": WORKLOAD, "iterations": info.iterations, "launches": info.launches,
                              "status": info.status}), flush=True)
        return
    timed_solves(nmg.NMG_PREC_FP64, max(1, args.warmup // 2), use_graph)

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    times, infos, _ = timed_solves(args.precision, args.steps, use_graph)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    clk = clocks.stop()

    xr = x.cpu().numpy()          # the mixed solution of the timed solves
    # the dominant kernel (finest-level Vanka apply) timed per launch with events on its launch
    # stream (plain launches of the per-step engine), and whole V-cycles in the timed configuration
    # in the solve: every launch of plain-launch solves (engine KERNELS), events around each launch
    _, _, prof = timed_solves(args.precision, args.steps, 0, profile=2, engine=nmg.NMG_ENGINE_KERNELS)
    _, _, sprof = timed_solves(args.precision, args.steps, 0, profile=3, engine=nmg.NMG_ENGINE_KERNELS)
    # alone: one launch at a time after an L2-evicting write
    cold = cold_launches(nmg, S, sysm, stream, flush, args.precision, 2, args.steps)
    scold = cold_launches(nmg, S, sysm, stream, flush, args.precision, 3, args.steps)
    plain_apply = plain_read_cold(cold[2], stream, flush, args.steps) if cold[1] else None
    plain_spmv = plain_read_cold(scold[2], stream, flush, args.steps) if scold[1] else None
    _, _, vprof = timed_solves(args.precision, args.steps, min(use_graph, 1), profile=1)
    rep = C.create_string_buffer(32768)
    nmg.check(nmg.nmg_autotune_report(S.handle, rep, 32768))
    tuned = json.loads(rep.value.decode())
    # plain FP64 path on the same mesh
    t64, i64, _ = timed_solves(nmg.NMG_PREC_FP64, args.steps, use_graph)
    x64 = x.cpu().numpy()

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    bh = torch.from_numpy(sysm.rhs.copy()).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t = time.perf_counter()
        S.solve(bh, xh, precision=args.precision, use_graph=use_graph)
        e2e.append(1000.0 * (time.perf_counter() - t))

    set_ms = _setup_ms(nmg, S, sysm)
    # (the layout study runs before the multi-vector solves: a layout is set before those)
    uniform = args.large_patches == "none"
    sizes = _patch_sizes(args, S, sysm, stream, flush, use_graph) if ncomp == sysm.problem.dim + 1 and uniform \
        else None
    multi = _multi_rhs(args, S, sysm, stream, flush, use_graph) if args.rhs > 0 and args.precision != 0 and uniform \
        else None

    ms = statistics.mean(times)
    ms_max, wall_max = max_over_ranks([ms, wall], dist, "cuda")

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    hbm, peak_kind = peaks()
    kms, klaunch, kbytes = prof
    vms, vcount, vbytes = vprof
    achieved = kbytes / (kms / klaunch * 1e-3) / 1e9 if klaunch else None
    choice = tuned["choice"][args.precision]
    line = {
        "metric": METRIC,
        "value": ms_max,
        "unit": "ms",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 * wall_max / args.steps,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {0: "f64", 1: "f32+f64", 2: "bf16/f32+f64"}[args.precision],
        "data": "synthetic",
        "config": dict(workload_config(sysm), parallelism="replicas" if world > 1 else "single GPU"),
        "impl_detail": {"vcycle_precision": {0: "fp64", 1: "fp32", 2: "bf16 factors"}[args.precision],
                        "outer": "fp64 FGMRES(30)",
                        "graphs": {0: "none (plain launches, host-stepped FGMRES)",
                                   1: "V-cycle graph, host-stepped FGMRES",
                                   2: "V-cycle inside one on-device graph loop per restart cycle"}[use_graph],
                        "device_loop": bool(infos[-1].device_loop),
                        "engine": {1: "kernels", 2: "persistent", 3: "fused"}.get(infos[-1].engine, "?"),
                        "autotuned": {k: choice[k] for k in ("tail_patches", "tile_patches", "fused")},
                        "l2": "flushed before every solve (256 MB write, outside the per-solve events)"},
        "roofline": {"kernel": apply_kernel_name(sysm.problem, ncomp, args.precision) +
                               " (finest-level Vanka apply)", "bound": "hbm",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None,
                     "traffic": PROFILED_TRAFFIC.get((WORKLOAD, args.precision)),
                     "peak_kind": peak_kind, "launch_ms": kms / klaunch if klaunch else None,
                     "bytes_per_launch": kbytes,
                     "timed": f"all {klaunch} launches of {args.steps} plain-launch solves, events around each on "
                              "its stream (the level's data partly L2-resident between smoothing steps)",
                     "cold": _cold_line(cold, hbm, plain_apply)},
        "e2e": {"value": statistics.mean(e2e), "unit": "ms", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(sum(i.launches for i in infos)),
        "clocks": clk,
        "p50_ms": sig(statistics.median(times)),
        "p99_ms": sig(sorted(times)[max(0, int(0.99 * len(times)) - 1)]),
        "solves_per_s": sig(job_throughput(world, ms_max)),
    }
    oracle = _oracle_legs(args, sysm, xr, x64) if not args.skip_cpu else {}
    if "cpu_baseline" in oracle:
        line["cpu_baseline"] = oracle.pop("cpu_baseline")
    # compact records, most important last
    line["vcycle"] = {"us": sig(1000.0 * vms / vcount) if vcount else None,
                      "GBps": sig(vbytes / (vms / vcount * 1e-3) / 1e9) if vcount else None,
                      "algorithmic_MB": sig(vbytes / 1e6)}
    line["setup"] = _setup_line(sysm, set_ms)
    line["multi_rhs"] = multi
    line["patch_sizes"] = sizes
    line["spmv"] = dict(_spmv_line(sprof, hbm) or {}, cold=_cold_line(scold, hbm, plain_spmv))
    if world == 1 and not args.no_serving_sample:
        line["serving"] = _serving_sample(args)
    if world == 1 and not args.no_large and WORKLOAD == "cfg2":
        S.close()                 # room for the 3d 96^3 hierarchy
        line["cfg4"] = _large_record(args, hbm, flush)
    line["rel_residual"] = sig(infos[-1].rel_residual, 3)
    line["check"] = {"rel_residual_host": sig(float(np.linalg.norm(sysm.rhs - _matvec(sysm, xr)) /
                                                    np.linalg.norm(sysm.rhs)), 3)}
    line.update(oracle)
    line["fp64_path"] = {"ms": sig(statistics.mean(t64)), "iterations": i64[-1].iterations,
                         "speedup_of_mixed": sig(statistics.mean(t64) / ms)}
    line["iterations"] = infos[-1].iterations
    print(json.dumps(line), flush=True)
    S.close()
    if dist:
        dist.destroy_process_group()


def _oracle_legs(args, sysm, x_mixed, x_fp64):
    """The FP64 CPU oracle on the host: one solve with single-threaded BLAS /
    OpenMP pools (its solution is the reference of rel_error_vs_oracle) and one
    with pools of every host core (the cpu_baseline)."""
    import tempfile

    import numpy as np
    out = {}
    cores = host_cores()
    try:
        with tempfile.TemporaryDirectory() as tmp:
            path = os.path.join(tmp, "x_oracle.npy")
            one = run_oracle(1, threads=1, save=path)
            xo = np.load(path)
        allc = run_oracle(1, threads=cores)
        eff = allc["cpu_times"][0] / allc["times"][0]
        out["cpu_baseline"] = {"value": 1000.0 * allc["times"][0], "unit": "ms", "cores": cores, "kind": "oracle",
                               "effective_cores": sig(eff, 3), "single_thread_ms": sig(1000.0 * one["times"][0]),
                               "sample": "one full FP64 oracle solve of the same workload (setup excluded); "
                                         f"BLAS/OpenMP pools of {cores} threads, and of 1 thread",
                               "iterations": one["iterations"]}
        nrm = np.linalg.norm(xo)
        out["rel_error_vs_oracle"] = {
            "mixed": sig(float(np.linalg.norm(x_mixed - xo) / nrm), 3),
            "fp64": sig(float(np.linalg.norm(x_fp64 - xo) / nrm), 3),
            "oracle_iterations": one["iterations"]}
    except Exception as e:   # the GPU numbers stand without it
        out["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
    return out


def _large_record(args, hbm, flush):
    """The 3d 96^3 workload (3,650,692 unknowns, 6 levels) measured in the same
    run: time to 1e-8 with FP32 and BF16 patch inverses and with the plain FP64
    path (graphs, on-device restart loops, L2 flushed before each solve), the
    finest Vanka apply and SpMV against the HBM copy rate, and the set-up."""
    import numpy as np
    import torch
    from gen import build_system, config_problem
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import Session

    t0 = time.time()
    sysm = build_system(config_problem("cfg4"))
    gen_s = time.time() - t0
    stream = torch.cuda.Stream()
    S = Session(sysm.problem.dim, sysm.problem.n, [(l.row_ptr, l.col_idx, l.vals) for l in sysm.levels],
                sysm.dirichlet, stream=stream.cuda_stream)
    b = torch.from_numpy(sysm.rhs).cuda()
    x = torch.empty_like(b)

    def solves(prec, k, graph=2, profile=0, engine=nmg.NMG_ENGINE_AUTO):
        ts, info = [], None
        if profile:
            nmg.check(nmg.nmg_profile_enable(S.handle, profile))
        with torch.cuda.stream(stream):
            for _ in range(k):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = S.solve(b, x, precision=prec, use_graph=graph, engine=engine)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
                if profile:
                    nmg.check(nmg.nmg_profile_read(S.handle, None, None, None))
        prof = None
        if profile:
            import ctypes as C
            ms, cnt, bpl = C.c_double(), C.c_int64(), C.c_double()
            nmg.check(nmg.nmg_profile_read(S.handle, ms, cnt, bpl))
            nmg.check(nmg.nmg_profile_enable(S.handle, 0))
            prof = bpl.value / (ms.value / cnt.value * 1e-3) / 1e9 if cnt.value else None
        return statistics.mean(ts), info, prof

    rec = {"unknowns": int(sysm.unknowns)}
    for name, prec in (("fp32", 1), ("bf16", 2), ("fp64_path", 0)):
        solves(prec, 2)                                  # warm-up (autotune, graph capture)
        ms, info, _ = solves(prec, 3 if prec else 2)
        rec[name] = {"ms": sig(ms), "iterations": info.iterations, "rel_residual": sig(info.rel_residual, 3)}
    rec["speedup_fp32"] = sig(rec["fp64_path"]["ms"] / rec["fp32"]["ms"], 3)
    rec["speedup_bf16"] = sig(rec["fp64_path"]["ms"] / rec["bf16"]["ms"], 3)
    rates = []
    for mode in (2, 3):
        ms, cnt, nbytes = cold_launches(nmg, S, sysm, stream, flush, 1, mode, 5)
        rates.append(nbytes / (ms / cnt * 1e-3) / 1e9 if cnt else None)
    apply_gbs, spmv_gbs = rates
    rec["apply_fp32_frac"] = sig(apply_gbs / hbm, 3) if apply_gbs else None
    rec["spmv_fp32_frac"] = sig(spmv_gbs / hbm, 3) if spmv_gbs else None
    rec["setup_ms"] = sig(_setup_ms(nmg, S, sysm))
    rec["host_gen_s"] = sig(gen_s, 3)
    S.close()
    del sysm
    return rec


def cold_launches(nmg, S, sysm, stream, flush, prec, mode, reps):
    """Device time of the finest level's Vanka apply (mode 2) or residual
    product (mode 3), one launch at a time through nmg_smooth (one step: the
    apply alone from a zero iterate, or product + apply from a given one),
    each launch after a 256 MB write that evicts the L2 (the write also keeps
    the stream busy while the launch is enqueued, so no host gap enters the
    events the library records around the launch).  Returns (total ms,
    launches, algorithmic bytes per launch)."""
    import ctypes as C

    import numpy as np
    import torch
    L = sysm.problem.levels - 1
    dt = torch.float64 if prec == 0 else torch.float32
    b = torch.from_numpy(sysm.rhs).to(dt).cuda()
    x = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, sysm.unknowns)).to(dt).cuda()
    x_zero = 1 if mode == 2 else 0
    with torch.cuda.stream(stream):
        for warm in (True, False):
            nmg.check(nmg.nmg_profile_enable(S.handle, mode))
            for _ in range(2 if warm else reps):
                flush.fill_(1.0)
                nmg.check(nmg.nmg_smooth(S.handle, L, prec, b, x, 1, x_zero, 0.8, nmg.NMG_WEIGHT_AVERAGE))
                nmg.check(nmg.nmg_profile_read(S.handle, None, None, None))
    ms, cnt, bpl = C.c_double(), C.c_int64(), C.c_double()
    nmg.check(nmg.nmg_profile_read(S.handle, ms, cnt, bpl))
    nmg.check(nmg.nmg_profile_enable(S.handle, 0))
    return ms.value, cnt.value, bpl.value


def _patch_sizes(args, S, sysm, stream, flush, use_graph):
    """The Vanka patch-size study of Section 5.5.1 on this workload: small
    patches (2^d cells) everywhere, large ones (4^d cells) on the solid, on the
    fluid, and everywhere (F/S: unknowns per patch in the fluid / the solid).
    Per layout: FGMRES iterations, time per solve with the per-step-kernel
    engine (the only one for two patch sizes; L2 flushed before each) and the
    re-factorisation of every level in that layout (nmg_set_large_patches on
    the resident hierarchy)."""
    import numpy as np
    import torch
    from gen.q1fsi import solid_cells
    p = sysm.problem
    small, large = 3 ** p.dim * p.ncomp, 5 ** p.dim * p.ncomp
    solid = solid_cells(p, p.n)
    layouts = [(f"F{small}/S{small}", None), (f"F{small}/S{large}", solid), (f"F{large}/S{small}", ~solid),
               (f"F{large}/S{large}", np.ones_like(solid))]
    b = torch.from_numpy(sysm.rhs).cuda()
    x = torch.empty_like(b)
    out = {}
    for name, region in layouts:
        torch.cuda.synchronize()
        t = time.perf_counter()
        S.set_large_patches(region)
        torch.cuda.synchronize()
        set_ms = 1000.0 * (time.perf_counter() - t)
        ts, info = [], None
        with torch.cuda.stream(stream):
            for k in range(2 + max(3, args.steps // 4)):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = S.solve(b, x, precision=args.precision, use_graph=use_graph, engine=1)   # per-step kernels
                e1.record(stream)
                e1.synchronize()
                if k >= 2:
                    ts.append(e0.elapsed_time(e1))
        out[name] = {"iterations": info.iterations, "ms": sig(statistics.mean(ts)), "refactor_ms": sig(set_ms, 3),
                     "ok": info.status == 0}
    S.set_large_patches(None)
    return out


def _multi_rhs(args, S, sysm, stream, flush, use_graph):
    """Many right-hand sides against the same hierarchy: K columns (the
    workload's own right-hand side, then seeded uniform vectors with the
    Dirichlet entries zero) solved by nmg_solve_many, against the same K
    columns solved one by one with nmg_solve in the timed configuration; and
    the multi-vector V-cycle against the single V-cycle per column."""
    import numpy as np
    import torch
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts

    K, prec = args.rhs, args.precision
    rng = np.random.default_rng(2024)
    mask = np.asarray(sysm.dirichlet, dtype=bool).reshape(-1)
    cols = [sysm.rhs]
    for _ in range(1, K):
        v = rng.uniform(-1.0, 1.0, sysm.rhs.size)
        v[mask] = 0.0
        cols.append(v)
    B = torch.from_numpy(np.stack(cols)).cuda()
    X = torch.zeros_like(B)
    x1 = torch.empty_like(B[0])

    def timed(fn, reps):
        out = []
        with torch.cuda.stream(stream):
            for _ in range(reps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = fn()
                e1.record(stream)
                e1.synchronize()
                out.append((e0.elapsed_time(e1), r))
        return out

    many = lambda: S.solve_many(B, X, K, precision=prec, use_graph=1)
    timed(many, 2)
    runs = timed(many, max(3, args.steps // 2))
    ms_many = statistics.mean(t for t, _ in runs)
    infos = runs[-1][1]

    def singles():
        its = []
        for k in range(K):
            its.append(S.solve(B[k], x1, precision=prec, use_graph=use_graph).iterations)
        return its
    timed(singles, 1)
    sruns = timed(singles, 3)
    ms_single = statistics.mean(t for t, _ in sruns)

    R = B.to(torch.float32)
    Z = torch.zeros_like(R)
    o = solve_opts(precision=prec, use_graph=1)
    vm = lambda: nmg.check(nmg.nmg_vcycle_many(S.handle, o, K, R, Z))
    timed(vm, 2)
    v_many = statistics.mean(t for t, _ in timed(vm, 10))
    z1 = torch.zeros_like(R[0])
    vs = lambda: nmg.check(nmg.nmg_vcycle(S.handle, solve_opts(precision=prec, use_graph=1), R[0], z1))
    timed(vs, 2)
    v_single = statistics.mean(t for t, _ in timed(vs, 10))
    its = [i.iterations for i in infos]
    return {"columns": K, "ms_per_column": sig(ms_many / K), "single_ms_per_column": sig(ms_single / K),
            "speedup": sig(ms_single / ms_many, 3), "iterations_equal": its == list(sruns[-1][1]),
            "vcycle_us_per_column": sig(1000.0 * v_many / K), "single_vcycle_us": sig(1000.0 * v_single)}


def plain_read_cold(nbytes, stream, flush, reps):
    """Microseconds of a plain library read of nbytes (torch.sum over an FP32
    buffer of that size), timed exactly as cold_launches times a kernel: after
    the same L2-evicting write, events on the same stream.  It is the rate a
    memory-bound launch of that size reaches under this timing, for comparison
    with the copy peak measured on gigabytes."""
    import torch
    buf = torch.ones(max(1, int(nbytes) // 4), dtype=torch.float32, device="cuda")
    out = torch.empty((), dtype=torch.float32, device="cuda")
    times = []
    with torch.cuda.stream(stream):
        for r in range(reps + 2):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.sum(buf, dim=0, out=out)
            e1.record(stream)
            e1.synchronize()
            if r >= 2:
                times.append(1000.0 * e0.elapsed_time(e1))
    return sum(times) / len(times)


def _cold_line(prof, hbm, plain_us=None):
    """Rate of launches timed alone after an L2-evicting write (cold_launches),
    beside a plain read of the same bytes timed the same way."""
    ms, cnt, nbytes = prof
    if not cnt:
        return None
    gbs = nbytes / (ms / cnt * 1e-3) / 1e9
    line = {"us": sig(1000.0 * ms / cnt), "GBps": sig(gbs), "frac": sig(gbs / hbm, 3)}
    if plain_us:
        line["plain_read"] = {"what": "torch.sum over the same bytes, same timing", "us": sig(plain_us),
                              "frac": sig(nbytes / (plain_us * 1e-6) / 1e9 / hbm, 3),
                              "kernel_over_plain": sig(1000.0 * ms / cnt / plain_us, 3)}
    return line


def _spmv_line(prof, hbm):
    """The finest-level residual product (block SpMV), timed per launch with
    events on its stream inside plain-launch solves: algorithmic bytes (Q1
    blocks once, x, b and r once) over the mean launch time."""
    ms, cnt, nbytes = prof
    if not cnt:
        return None
    gbs = nbytes / (ms / cnt * 1e-3) / 1e9
    return {"GBps": sig(gbs), "frac": sig(gbs / hbm, 3),
            "us": sig(1000.0 * ms / cnt), "MB": sig(nbytes / 1e6), "launches": cnt}


# FP64 peak of one GB300 derived from its units and clock: 152 SMs x 2 FP64 FMA
# lanes per SM clock x 2 flops x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07


def _setup_ms(nmg, S, sysm):
    """Median of 3 re-factorisations of the finest level through
    nmg_set_jacobian from device buffers (a new Jacobian: stencil copy, FP32
    copy, patch extraction and FP64 inversion of every patch)."""
    import numpy as np
    import torch
    fin = sysm.fine
    rp_d = torch.from_numpy(np.ascontiguousarray(fin.row_ptr, dtype=np.int64)).cuda()
    ci_d = torch.from_numpy(np.ascontiguousarray(fin.col_idx, dtype=np.int32)).cuda()
    v_d = torch.from_numpy(np.ascontiguousarray(fin.vals, dtype=np.float64)).cuda()
    out = []
    for _ in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        nmg.check(nmg.nmg_set_jacobian(S.handle, sysm.problem.levels - 1, fin.nodes, ci_d.numel(), rp_d, ci_d, v_d, 1))
        torch.cuda.synchronize()
        out.append(1000.0 * (time.perf_counter() - t))
    return statistics.median(out)


def _setup_line(sysm, ms):
    """Re-factorisation of the finest level: Gauss-Jordan inversion of every
    n_p x n_p patch, n_p^3 FP64 FMAs each, against the FP64 ALU peak."""
    d = sysm.problem.dim
    patches = 1
    for nk in sysm.problem.n:
        patches *= nk // 2
    n_p = 3 ** d * int(sysm.fine.vals.shape[1])
    gflops = 2.0 * patches * n_p ** 3 / (ms * 1e-3) / 1e9
    return {"ms": sig(ms), "patches": patches, "n_p": n_p, "GFLOPs_fp64": sig(gflops),
            "frac_fp64_alu": sig(gflops / FP64_PEAK_GFLOPS, 3)}


def _matvec(sysm, x):
    import scipy.sparse as sp
    f = sysm.fine
    nc = f.vals.shape[1]
    A = sp.bsr_matrix((f.vals, f.col_idx, f.row_ptr), shape=(f.nodes * nc,) * 2)
    return A @ x


def _serve(args, sizes, seeds, n_requests, n_burst):
    """Continuous-batching serving of condensed-momentum solves.

    Each mesh size of sizes ((dim, n) pairs) has a pool of resident
    hierarchies, one per coefficient seed in seeds; request i draws its mesh
    and hierarchy from numpy default_rng(2) (2d and 3d 50/50) and its
    right-hand side from the CUDA generator seeded 11 + 2 i.  Arrivals are a
    Poisson stream (seed 2) at 80% of the saturated throughput measured first
    on a burst of n_burst requests of the same mix.  One server (16 slots,
    150 GB) serves the warm-up, the burst and the timed stream.
    """
    import ctypes as C

    import numpy as np
    import torch

    from gen import Problem, build_system
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import Session, solve_opts

    torch.cuda.set_device(0)
    pool = []
    t0 = time.time()
    for dim, n in sizes:
        for cseed in seeds:
            levels = int(np.log2(n)) - 1
            p = Problem(dim=dim, n=(n,) * dim, levels=levels,
                        solid=(0, +1, 0.6) if dim == 2 else (2, -1, 0.25), conv_seed=cseed)
            sy = build_system(p)
            S = Session(dim, p.n, [(l.row_ptr, l.col_idx, l.vals) for l in sy.levels], sy.dirichlet,
                        precisions=1 << nmg.NMG_PREC_FP32)
            mask = torch.from_numpy(sy.dirichlet.astype(bool)).cuda()
            pool.append((dim, n, S, mask))
            del sy
    setup_s = time.time() - t0
    rng = np.random.default_rng(2)
    opts = solve_opts(precision=nmg.NMG_PREC_FP32, engine=nmg.NMG_ENGINE_KERNELS,
                      use_graph=0 if args.no_graph else args.graph)
    budget = 150 * 10**9
    both = len({d for d, _ in sizes}) > 1

    def make_requests(count, seed0):
        out = []
        for i in range(count):
            d2 = rng.random() < 0.5
            cands = [k for k, (dim, n, S, m) in enumerate(pool) if (dim == 2) == d2 or not both]
            k = int(rng.choice(cands))
            dim, n, S, mask = pool[k]
            g = torch.Generator(device="cuda").manual_seed(seed0 + 2 * i)
            b = torch.rand(mask.numel(), dtype=torch.float64, device="cuda", generator=g) * 2.0 - 1.0
            b[mask] = 0.0
            out.append((k, b, torch.zeros_like(b)))
        torch.cuda.synchronize()
        return out

    server = C.c_void_p()
    nmg.check(nmg.nmg_server_create(budget, 16, server))
    nmg.check(nmg.nmg_server_set_workspaces(server, args.workspaces))
    nmg.check(nmg.nmg_server_set_batching(server, args.batch))

    def run(reqs, rate):
        tickets = []
        start = time.perf_counter()
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs))) if rate else np.zeros(len(reqs))
        for (k, b, x), at in zip(reqs, arrivals):
            now = time.perf_counter() - start
            if at > now:
                time.sleep(at - now)
            t = C.c_uint64()
            nmg.check(nmg.nmg_submit(server, pool[k][2].handle, b, x, opts, t))
            tickets.append(t.value)
        lat, its, bad = [], [], 0
        for t in tickets:
            info = nmg.nmg_solve_info()
            st = nmg.nmg_poll(server, t, 600000, info)
            bad += st != 0
            lat.append(info.ms_total)
            its.append(info.iterations)
        wall = time.perf_counter() - start
        return wall, lat, its, bad

    burst = make_requests(n_burst, 1_000_011)
    run(burst[:20], 0)                       # warm-up (graphs captured, engines resolved)
    wall_b, _, _, _ = run(burst, 0)
    saturated = len(burst) / wall_b
    del burst
    reqs = make_requests(n_requests, 11)
    rate = 0.8 * saturated
    wall, lat, its, bad = run(reqs, rate)
    nmg.nmg_server_destroy(server)
    for _, _, S, _ in pool:
        S.close()
    lat_sorted = sorted(lat)
    return {"requests": len(reqs), "hierarchies": len(pool), "p50_ms": statistics.median(lat),
            "p99_ms": lat_sorted[max(0, int(0.99 * len(lat)) - 1)], "solves_per_s": len(reqs) / wall,
            "arrival_rate_per_s": rate, "saturated_solves_per_s": saturated, "failed": bad,
            "mean_iterations": statistics.mean(its), "setup_s": setup_s}


SERVING_SIZES = [(2, 64), (2, 128), (2, 256), (2, 512), (3, 16), (3, 32), (3, 64)]


def serving_arm(args):
    """The serving workload as its own bench line (--serving): 2000 requests
    over two resident hierarchies per mesh size (or one mesh, --mesh)."""
    sizes, seeds = SERVING_SIZES, (10, 12)
    if args.mesh:
        d, nn = args.mesh.split(":")
        sizes, seeds = [(int(d[0]), int(nn))], (10,)
    r = _serve(args, sizes, seeds, args.requests, 200)
    line = {
        "metric": METRIC, "value": r["p50_ms"], "unit": "ms (p50 submit-to-completion latency)",
        "n_gpus": 1, "steps": r["requests"], "warmup": 20, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": ("serving: Poisson stream of condensed-momentum solves, 2d 64^2-512^2 and 3d "
                                "16^3-64^3 (50/50), 14 resident hierarchies, FP32 V-cycle / FP64 FGMRES(30), "
                                "rtol 1e-8, memory budget 150 GB, 16 slots") if not args.mesh else
                               (f"serving: Poisson stream of condensed-momentum solves on one resident {args.mesh} "
                                "hierarchy (right-hand sides seeded per request), FP32 V-cycle / FP64 FGMRES(30), "
                                "rtol 1e-8, memory budget 150 GB, 16 slots"),
                   "extra_workspaces_per_hierarchy": args.workspaces,
                   "batched_columns": args.batch,
                   "arrival_rate_per_s": r["arrival_rate_per_s"],
                   "saturated_solves_per_s": r["saturated_solves_per_s"]},
        "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "solves_per_s": r["solves_per_s"], "failed": r["failed"],
        "mean_iterations": r["mean_iterations"], "setup_s": r["setup_s"],
    }
    print(json.dumps(line), flush=True)


def _serving_sample(args):
    """A bounded sample of the serving workload for the main line: every mesh
    size of the serving mix with one resident hierarchy each, a burst of 100
    requests for the saturated rate, then args.serving_sample requests at 80%
    of it."""
    r = _serve(args, SERVING_SIZES, (10,), args.serving_sample, 100)
    return {"requests": r["requests"], "hierarchies": r["hierarchies"], "p50_ms": sig(r["p50_ms"]), "p99_ms": sig(r["p99_ms"]),
            "solves_per_s": sig(r["solves_per_s"]), "saturated_per_s": sig(r["saturated_solves_per_s"]),
            "failed": r["failed"]}


def main():
    global WORKLOAD, WORKLOAD_DESC
    args = parse()
    WORKLOAD, WORKLOAD_DESC = args.workload, WORKLOADS[args.workload]
    if args.serving:
        serving_arm(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
