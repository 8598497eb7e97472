"""Benchmark of the nonlinear Newmark-beta time stepper on GB300.

Workload (default): the single large model -- 800 x 800 x 260 m, 5 m hexahedra
(160 x 160 x 52) split into 7,987,200 quadratic tetrahedra (10,819,305 nodes,
32.5 M DOF), soft layer over bedrock with a seeded random interface 20-60 m
deep, 4 points per element, 150 springs per point (191.7 GB of spring state,
resident in HBM), dt = 0.005 s, CG tolerance 1e-8, FP64.  One benchmark step =
one time step of the whole hot path (right-hand side, block-Jacobi set-up, PCG,
Newmark update, multi-spring update at every integration point).

Timed window: the input is a full-length record (2000 steps) tapered over 0.2 s;
before the warm-up the model is advanced through a lead-in until the S waves have
crossed the bedrock and the deepest soft layer (synth.lead_in_steps: 187 steps),
so the warm-up and timed steps fall in the strong motion of the soft soil.

Printed JSON line (rank 0): value = element-steps/s over all ranks (device time
with CUDA events inside the library, all streams joined), e2e = the same metric
through the public API with the input record copied from host and the surface
response read back every run, roofline of the dominant kernel, the CPU oracle
timed on a bounded sample as cpu_baseline, the streamed-state link rate when the
state is partly kept in pinned host memory (Alg. 3), and the SM clocks sampled
during the timed region.

--impl reference times the CPU oracle (the reference arm) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_02755_gb300 import dist, synth  # noqa: E402

METRIC = "elem-steps/s at oracle tol"
N_TUNE_STEPS = 14  # candidate spring launch shapes at 150 springs (7 tiles x two register budgets)
UNIT = "elem-steps/s"
# algorithmic bytes of the multi-spring update: the 40-byte state of each spring read and
# written, 2 x 4 points x S springs x 40 B = 320 S bytes per element-step
SPRING_STATE_BYTES_PER_SPRING = 80.0
# the FP64-accuracy operator: 1,800 flop per element (dense 30 x 30 element matvec)
EBE_FLOP_PER_ELEM = 1800.0
# ncu summary holding the spring kernel's DRAM bytes and warp instructions per spring
# (both scale with springs)
SPRING_PROFILE = "k_springs_large_model_cut_16x16x52.md"
# rated bandwidth of GB300's host link (NVLink-C2C, both directions together)
C2C_RATED_GBPS = 900.0
ARITHMETIC = ("FP64 state, Newmark update, outer CG and residuals; spring law (strains, power, Halley "
              "step, tangent) in double-float (~48-bit) arithmetic on the FP32 pipes with an FP64 fallback; "
              "inner preconditioner CG and its operator in FP32 (FP16 tangent storage with --solver fp64-ir16)")


def profiled_bytes(name, key):
    """A per-unit figure (DRAM bytes, warp instructions) that an ncu capture recorded for a
    kernel (a `key = value` line of its summary under profiles/), or None when there is no
    such summary."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        for line in open(path):
            if line.strip().startswith(key + " ="):
                return float(line.split("=", 1)[1])
    except OSError:
        pass
    return None


def measured_peaks():
    """The machine's measured copy bandwidth and GEMM rate, when the file is present."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def sample_clocks_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def sample_clocks_stop(proc, f, path, gpu_index=0):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.close()
    sm, smax, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        p = [x.strip() for x in line.split(",")]
        if len(p) < 9 or p[0] != str(gpu_index):
            continue
        try:
            sm.append(float(p[1]))
            smax = max(smax, float(p[2]))
        except ValueError:
            continue
        for n, v in zip(names, p[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def link_probe(sizes_mb=(256, 1024, 4096), streams=(1, 2)):
    """Pinned host <-> HBM copy rates (GB/s, CUDA events, best of three): H2D alone, D2H
    alone and both directions at once (bytes of both summed), for each copy size and for
    one or two streams per direction (each stream copying its share).  Pinned buffers come
    from cudaHostAlloc (torch pin_memory), the device buffers from the caching allocator."""
    import torch
    nmax = max(sizes_mb) << 20
    h1 = torch.empty(nmax, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(nmax, dtype=torch.uint8, pin_memory=True)
    d1 = torch.empty(nmax, dtype=torch.uint8, device="cuda")
    d2 = torch.empty(nmax, dtype=torch.uint8, device="cuda")
    ss = [torch.cuda.Stream() for _ in range(4)]

    def timed(n, k, what):
        best = 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            used, moved = [], 0
            for dirn in (("h2d", "d2h") if what == "bidir" else (what,)):
                for j in range(k):
                    s_ = ss[len(used)]
                    s_.wait_event(e0)
                    a, b = j * n // k, (j + 1) * n // k
                    with torch.cuda.stream(s_):
                        if dirn == "h2d":
                            d1[a:b].copy_(h1[a:b], non_blocking=True)
                        else:
                            h2[a:b].copy_(d2[a:b], non_blocking=True)
                    used.append(s_)
                moved += n
            for s_ in used:
                ev = torch.cuda.Event()
                ev.record(s_)
                torch.cuda.current_stream().wait_event(ev)
            e1.record()
            torch.cuda.synchronize()
            best = max(best, moved / (e0.elapsed_time(e1) / 1e3) / 1e9)
        return best

    out = {}
    for mb in sizes_mb:
        for k in streams:
            for what in ("h2d", "d2h", "bidir"):
                out["%s_%dMB_%ds" % (what, mb, k)] = timed(mb << 20, k, what)
    del h1, h2, d1, d2
    torch.cuda.empty_cache()
    best = {w: max(v for key, v in out.items() if key.startswith(w + "_")) for w in ("h2d", "d2h", "bidir")}
    return {"best_GBps": best, "runs_GBps": out, "rated_bidir_GBps": C2C_RATED_GBPS,
            "buffers": "cudaHostAlloc pinned (torch pin_memory) <-> device, sizes %s MB, %s stream(s) per direction"
                       % (list(sizes_mb), list(streams))}


def oracle_sample(steps=1, column=(0, 0, 8, 8), omp=False):
    """The CPU oracle on a bounded column of the large model (same spacing,
    interface field, springs, dt and input); returns elem-steps/s, the threads it used
    and a description.  omp: the OpenMP build of the same oracle on all host cores."""
    import oracle
    wl = synth.large_single_model(column=column)
    wl.wave = synth.main_motion_record()
    cores = oracle.threads(os.cpu_count() or 1) if omp else 1
    o = oracle.Oracle.from_workload(wl, omp=omp)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
    dt = time.perf_counter() - t0
    desc = ("oracle (plain C, FP64, %s) on a %dx%dx%d-hexahedron column of the large model "
            "(%d elements, %d springs/point), %d step(s) from rest, %.1f s" %
            ("OpenMP build, %d threads" % cores if omp else "1 thread", column[2], column[3], wl.mesh.dims[2],
             wl.mesh.n_elems, wl.n_springs, steps, dt))
    return wl.mesh.n_elems * steps / dt, cores, desc


def reference_arm(args):
    rank, ws, _ = dist.world()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    col = (0, 0, 6, 6)
    wl = synth.large_single_model(column=col)
    wl.wave = synth.main_motion_record()
    cores = oracle.threads(os.cpu_count() or 1)
    o = oracle.Oracle.from_workload(wl, omp=True)
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step()
    el = time.perf_counter() - t0
    v = wl.mesh.n_elems * args.steps / el
    sample = ("%d time steps of a 6x6x52-hexahedron column (%d elements, 150 springs/point) of the large model "
              "after %d warm-up steps, OpenMP build of the oracle on %d threads" % (args.steps, wl.mesh.n_elems,
                                                                                 args.warmup, cores))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "elements": 160 * 160 * 52 * 6, "springs_per_point": wl.n_springs,
                       "dt": wl.dt, "cg_tol": 1e-8, "numbering": "grid",
                       "sample": "a %dx%dx52-hexahedron column of it (%d elements) on the host cores"
                                 % (col[2], col[3], wl.mesh.n_elems)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def served(args, dd, rank, ws, local):
    """Served ensemble: a Poisson trace of requests of uneven size submitted at their
    arrival times to the serving runtime; value = all requests' element-steps over the
    makespan (first arrival to last completion), with p50/p99 time to solution."""
    from paper_2604_02755_gb300 import binding as B
    trace = synth.served_trace(R=args.requests, step_scale=args.step_scale, seed=5 + rank, e_lo=args.e_lo,
                               e_hi=args.e_hi)
    prec = {"fp64-ir": B.NS_PREC_FP64_IR, "fp64-ir16": B.NS_PREC_FP64_IR16, "fp64-pcg": B.NS_PREC_FP64}[args.solver]
    clk_path = os.path.join(tempfile.gettempdir(), "ns_clocks_%d.csv" % rank)
    srv = B.Server(device=local, pinned_budget=int(args.pinned_gb * 1e9), max_active=args.max_active,
                   quantum_steps=16, batch=args.batch)
    dist.barrier(dd)
    proc, fh = sample_clocks_start(clk_path)
    t0 = time.perf_counter()
    ids = []
    for r in trace:
        delay = r.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(srv.submit(r.workload, r.n_steps, precision=prec, graphs=1))
    st = [srv.wait(i, 3600.0) for i in ids]
    res_bytes = 0
    for i in ids:
        res_bytes += sum(a.nbytes for a in srv.result(i).values())
    wall = time.perf_counter() - t0
    clocks = sample_clocks_stop(proc, fh, clk_path, local)
    srv.close()
    failed = [s_ for s_ in st if s_["state"] != B.NS_CASE_DONE]
    work = float(sum(s_["elem_steps"] for s_ in st))
    job_s, work_all = dist.reduce_time_and_work(dd, wall, work, device="cuda")
    tts = np.array([s_["t_done"] - s_["t_submit"] for s_ in st])
    wait = np.array([s_["t_admit"] - s_["t_submit"] for s_ in st])
    if rank == 0:
        sizes = [r.workload.mesh.n_elems for r in trace]
        line = {"metric": "served elem-steps/s; time to solution p50/p99", "value": work_all / job_s,
                "unit": "elem-steps/s", "n_gpus": ws, "steps": len(trace), "warmup": 0,
                "ms_per_step": job_s / max(1, len(trace)) * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "served ensemble: %d requests, Poisson arrivals 4/s, %d-%d elements "
                                       "(log-uniform in %g-%g), 20-150 springs, steps U[1000,4000] x %g" %
                                       (len(trace), min(sizes), max(sizes), args.e_lo, args.e_hi, args.step_scale),
                           "max_active": args.max_active, "solver": args.solver, "graphs": 1,
                           "batch": "continuous batching of each solver class" if args.batch else
                                    "one context per request",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "time_to_solution_s": {"p50": float(np.percentile(tts, 50)), "p99": float(np.percentile(tts, 99)),
                                       "max": float(tts.max())},
                "queue_wait_s": {"p50": float(np.percentile(wait, 50)), "max": float(wait.max())},
                "streamed_requests": int(sum(s_["streamed"] for s_ in st)), "failed": len(failed),
                "batching": ({"batches_per_request": float(np.mean([s_["batches"] for s_ in st])),
                              "requests_batched": int(sum(s_["batches"] > 0 for s_ in st)),
                              "reform_s_per_request": float(np.mean([s_["t_reform"] for s_ in st]))}
                             if args.batch else None),
                "offered_load": {"requests_per_s": 4.0,
                                 "elem_steps_per_request_mean": float(np.mean([r.workload.mesh.n_elems * r.n_steps
                                                                               for r in trace])),
                                 "value": 4.0 * float(np.mean([r.workload.mesh.n_elems * r.n_steps for r in trace])),
                                 "unit": "elem-steps/s"},
                "e2e": {"value": work_all / job_s, "unit": "elem-steps/s",
                        "h2d_bytes_per_step": int(sum(r.workload.mesh.xyz.nbytes + r.workload.mesh.conn.nbytes +
                                                      r.workload.wave.nbytes for r in trace) / len(trace)),
                        "d2h_bytes_per_step": int(res_bytes / len(trace))},
                "gpu_launches": int(sum(s_["kernel_launches"] for s_ in st)), "clocks": clocks,
                "roofline": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    dist.finalize(dd)
    return 0 if not failed else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "precision", "ensemble", "served", "tiny"],
                    help="large: the single large model (default); precision: the 1M-element three-layer "
                         "precision-form model; ensemble: --members cases on a shared 201,600-element mesh "
                         "advanced together; tiny: the 3,600-element two-layer case")
    ap.add_argument("--members", type=int, default=64, help="members of the ensemble workload")
    ap.add_argument("--union", action="store_true",
                    help="ensemble: store the disjoint union of the members' mesh copies instead of one shared mesh")
    ap.add_argument("--stage", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="FP32 inner operator: stage element tiles in shared memory with bulk copies (1), "
                         "per-warp asynchronous tangent copies (2), per-thread loads (0), or automatic (-1: "
                         "2 with the FP32 tangent, 0 with the FP16 one)")
    ap.add_argument("--spring-tile", type=int, default=0,
                    help="spring kernel points per block before (or without) the autotuner; 0: heuristic")
    ap.add_argument("--spring-blocks", type=int, default=4, choices=[1, 4],
                    help="spring kernel register budget (resident blocks per SM) before (or without) the autotuner")
    ap.add_argument("--spring-tensor", type=int, default=0, choices=[0, 1],
                    help="assemble the spring tangent on the tensor cores (1) or in double-float sums (0, default)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the library's autotuner (the spring kernel's launch shape, tuned on the last %d "
                         "lead-in steps)" % N_TUNE_STEPS)
    ap.add_argument("--prefetch", type=int, default=1, choices=[0, 1],
                    help="element operators prefetch their element rows into L2 (bulk prefetch)")
    ap.add_argument("--local-gather", type=int, default=0, choices=[0, 1],
                    help="FP32 inner operator: gather each block's distinct nodes into shared memory once (1) or "
                         "per element (0)")
    ap.add_argument("--pair-op", type=int, default=0, choices=[0, 1],
                    help="FP64-accuracy operator applications in double-float arithmetic on the FP32 pipes")
    ap.add_argument("--x0", default="zero", choices=["prev", "zero"],
                    help="CG start: zero (default: no operator application for the initial residual) or the "
                         "previous step's increment")
    ap.add_argument("--numbering", default="grid", choices=["grid", "morton", "shuffled"],
                    help="element and node numbering of the mesh: the generator's lexicographic grid order, "
                         "Morton order of centroids, or a seeded shuffle (gather-locality worst case)")
    ap.add_argument("--inner-tol", type=float, default=1e-4,
                    help="relative residual at which the FP32 inner CG stops early")
    ap.add_argument("--inner-iters", type=int, default=45,
                    help="FP32 inner CG iterations per outer iteration of the flexible solver")
    ap.add_argument("--requests", type=int, default=12, help="requests of the served trace")
    ap.add_argument("--step-scale", type=float, default=0.01,
                    help="served trace: fraction of the 1000-4000 steps each request runs")
    ap.add_argument("--max-active", type=int, default=4, help="served: requests in flight together")
    ap.add_argument("--e-lo", type=float, default=5e4, help="served: smallest mesh (elements, log-uniform)")
    ap.add_argument("--e-hi", type=float, default=2e6, help="served: largest mesh (elements, log-uniform)")
    ap.add_argument("--batch", type=int, default=0, choices=[0, 1],
                    help="served: continuous batching of compatible requests in one batched context (1) or one "
                         "context per request (0)")
    ap.add_argument("--pinned-gb", type=float, default=32.0, help="served: pinned host budget for streamed state")
    ap.add_argument("--graphs", type=int, default=-1, choices=[-1, 0, 1],
                    help="replay solver iterations as captured CUDA graphs (1) or launch them one by one (0, "
                         "keeps per-kernel times); default: 1 for the launch-bound tiny case, else 0")
    ap.add_argument("--dims", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                    help="hexahedra of a smaller cut of the large model (same spacing, interface and springs), "
                         "used for profiling captures that must stay small")
    ap.add_argument("--no-stream", action="store_true", help="skip the streamed-state measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the short runs of the tiny and precision-form configurations")
    ap.add_argument("--lead-in", type=int, default=-1,
                    help="steps taken before the warm-up (default: the large model's lead-in into the strong "
                         "motion, 0 for cuts and other workloads)")
    ap.add_argument("--stream-gb", type=float, default=128.0, help="spring state kept in pinned host memory (GB)")
    ap.add_argument("--ring-depth", type=int, default=12, help="device chunk buffers of the streamed state")
    ap.add_argument("--zero-copy", action="store_true",
                    help="also measure the streamed state updated in place in pinned host memory (no ring)")
    ap.add_argument("--multigrid", type=int, default=1, choices=[0, 1],
                    help="two-level preconditioner (default on): the inner FP32 solve starts from the interpolated "
                         "solution of the linear-element coarse model (Sec. 2.2, after [SC14])")
    ap.add_argument("--coarse-iters", type=int, default=20, help="multigrid: coarse PCG iterations at most")
    ap.add_argument("--coarse-tol", type=float, default=1e-3, help="multigrid: coarse relative residual target")
    ap.add_argument("--solver", default="fp64-ir", choices=["fp64-ir", "fp64-ir16", "fp64-pcg"],
                    help="fp64-ir: FP64 flexible CG with an FP32 PCG preconditioner (the paper's precision policy); "
                         "fp64-ir16: the same with the inner operator reading D in FP16; "
                         "fp64-pcg: plain FP64 block-Jacobi PCG")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)

    rank, ws, local = dist.world()
    import torch
    torch.cuda.set_device(local)
    dd = dist.init()
    from paper_2604_02755_gb300 import binding as B
    from paper_2604_02755_gb300 import build as nsbuild
    if rank == 0:
        nsbuild.build()
    dist.barrier(dd)
    nsbuild.build()
    if args.workload == "served":
        return served(args, dd, rank, ws, local)

    ens = None
    lead = 0
    if args.workload == "ensemble":
        n_total = args.warmup + 2 * args.steps + 2
        ens = synth.ensemble_members(M=args.members, nt=max(n_total, 400),
                                     dims=tuple(args.dims) if args.dims else (40, 40, 21))
        wl = ens.member(0)
        wl.name = ens.name
    elif args.workload == "tiny":
        wl = synth.tiny_two_layer()
    elif args.workload == "precision":
        wl = synth.precision_form_model(dims=tuple(args.dims) if args.dims else (64, 64, 41))
    elif args.dims:
        wl = synth.large_single_model(dims=tuple(args.dims))
        wl.name = "cut of the single large model: %dx%dx%d hexahedra at 5 m, 150 springs" % tuple(args.dims)
    else:
        wl = synth.large_single_model()
    if args.workload == "large":
        # full-length record whose strong part starts after a short taper; the lead-in carries
        # the model into the strong motion of the soft layer before warm-up and timing
        wl.wave = synth.main_motion_record()
        lead = args.lead_in if args.lead_in >= 0 else (0 if args.dims else synth.lead_in_steps(wl.dt))
    elif ens is None:
        wl.wave = synth.band_limited_wave(2, max(args.warmup + 2 * args.steps + 3, 400), wl.dt)
    if args.numbering != "grid":
        if ens is not None:
            ens.mesh = synth.renumber(ens.mesh, args.numbering, seed=9)
            wl.mesh = ens.mesh
        else:
            wl.mesh = synth.renumber(wl.mesh, args.numbering, seed=9)
    M = len(ens.members) if ens else 1
    E = wl.mesh.n_elems * M
    wave = wl.wave
    prec = {"fp64-ir": B.NS_PREC_FP64_IR, "fp64-ir16": B.NS_PREC_FP64_IR16, "fp64-pcg": B.NS_PREC_FP64}[args.solver]
    graphs = args.graphs if args.graphs >= 0 else (1 if args.workload == "tiny" else 0)
    kw = dict(device=local, timing=1, surface_ring_steps=max(args.steps, 1), precision=prec, graphs=graphs,
              stage_elements=args.stage, inner_max_iter=args.inner_iters, inner_tol=args.inner_tol, x0_prev=int(args.x0 == "prev"),
              pair_operator=args.pair_op, l2_prefetch=args.prefetch, spring_tile_points=args.spring_tile,
              spring_tile_blocks=args.spring_blocks, spring_tensor_cores=args.spring_tensor,
              local_gather=args.local_gather)
    if args.multigrid and ens is None and prec != B.NS_PREC_FP64:
        kw.update(multigrid=1, coarse_max_iter=args.coarse_iters, coarse_tol=args.coarse_tol)
    else:
        args.multigrid = 0  # one member and a flexible solver form only
    sim = B.BatchSimulation(ens, shared=not args.union, **kw) if ens else B.Simulation(wl, **kw)
    # the spring kernel's launch shape is tuned on the last steps of the lead-in (one per
    # candidate shape; they are ordinary steps of the run), or on steps before the warm-up
    n_tune = N_TUNE_STEPS if args.autotune else 0
    t_lead = time.perf_counter()
    if lead > n_tune:
        sim.advance(lead - n_tune)
    tuning = B.ns_autotune_steps(sim.ctx, n_tune) if n_tune else None
    t_lead = time.perf_counter() - t_lead
    lead = max(lead, n_tune)
    sim.advance(args.warmup)
    if tuning:  # later contexts of this run (the streamed-state legs) start from the tuned shape
        args.spring_tile, args.spring_blocks = tuning["chosen_tile_points"], tuning["chosen_tile_blocks"]
    B.ns_reset_stats(sim.ctx)
    st0 = sim.stats()

    clk_path = os.path.join(tempfile.gettempdir(), "ns_clocks_%d.csv" % rank)
    proc, fh = sample_clocks_start(clk_path)
    dist.barrier(dd)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps' launches
    sim.advance(args.steps)
    torch.cuda.nvtx.range_pop()
    dist.barrier(dd)
    clocks = sample_clocks_stop(proc, fh, clk_path, local)
    st = sim.stats()
    dev_s = st["ms_advance"] / 1e3
    job_s, work = dist.reduce_time_and_work(dd, dev_s, float(E * args.steps), device="cuda")
    value = work / job_s
    launches = st["kernel_launches"] - st0["kernel_launches"]
    first_timed = st0["steps"] + 1
    window = {"lead_in_steps": lead, "warmup_steps": args.warmup, "timed_steps": [first_timed, st["steps"]],
              "timed_t_s": [first_timed * wl.dt, st["steps"] * wl.dt], "lead_in_wall_s": t_lead,
              "cg_outer_iters_per_step": st["cg_iters_total"] / args.steps,
              "inner_iters_per_step": st["inner_iters_total"] / args.steps,
              "coarse_iters_per_step": st["coarse_iters_total"] / args.steps,
              "springs_moved_per_step": st["spring_moved"] / args.steps,
              "spring_reversal_rate": st["spring_reversals"] / max(st["spring_moved"], 1),
              "spring_fp64_root_rate": st["spring_fp64_roots"] / max(st["spring_moved"], 1)}

    # roofline of the dominant kernel.  The multi-spring update (the largest share of the
    # step) is HBM-bound by its algorithmic bytes: the 40-byte state of every spring read and
    # written, 320 S bytes per element-step, against the measured copy bandwidth.  Its DRAM
    # traffic and warp instructions per spring come from the ncu summary of the kernel.
    hbm_peak = measured_peaks().get("hbm_gbs")
    roof = None
    if st["n_spring"] > 0:
        per = st["ms_spring"] / st["n_spring"] / 1e3
        n_spr = 4 * st["resident_elems"] * wl.n_springs / max(st["n_spring"] / args.steps, 1)
        gbs = SPRING_STATE_BYTES_PER_SPRING * n_spr / per / 1e9
        bps = profiled_bytes(SPRING_PROFILE, "dram_bytes_per_spring")
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak if hbm_peak else None,
                "traffic": bps * n_spr if bps else None,
                "kernel": "k_springs (multi-spring update at every integration point)",
                "work_per_launch": "320 S B per element-step: 2 x %d springs x 40 B (state read and written)" % n_spr,
                "avg_launch_ms": per * 1e3, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per spring (%s) x springs"
                                  % SPRING_PROFILE}
        # what binds it: instruction issue (one warp instruction per clock on each of the 4
        # schedulers of the 152 SMs), from the profiled warp instructions per spring
        ips = profiled_bytes(SPRING_PROFILE, "warp_instructions_per_spring")
        if ips:
            mhz = (clocks or {}).get("sm_mhz") or 2070.0
            issue_peak = 152 * 4 * mhz / 1e3
            gips = ips * n_spr / per / 1e9
            roof["issue"] = {"achieved": gips, "peak": issue_peak, "unit": "G warp-instructions/s",
                             "frac": gips / issue_peak,
                             "peak_source": "152 SMs x 4 schedulers x 1 warp-instruction/clk x median SM clock (derived)",
                             "per_unit": "%g warp-instructions/spring (ncu smsp__inst_executed, spring profile)" % ips}

    # the HBM-bound matvec: the inner FP32 operator, per launch that did work.  Algorithmic
    # bytes: per element connectivity 40, geometry 40, material 4, tangent 336 (FP32) or 168
    # (FP16); per node the gathered x read once (16) and y read and written once (32), i.e.
    # 48 N/E per element (the ncu DRAM count of the kernel agrees: 484 B per element on the
    # large model's numbering, N/E = 1.35)
    matvec = None
    if st["inner_iters_total"] > 0 and st["ms_ebe32"] > 0:
        n_per_e = (wl.mesh.n_nodes * M) / E
        bpe = (252.0 if prec == B.NS_PREC_FP64_IR16 else 420.0) + 48.0 * n_per_e
        # active launches: one per inner iteration, plus (multigrid) the residual of the
        # interpolated start once per outer iteration
        active = st["inner_iters_total"] + (st["cg_iters_total"] if args.multigrid else 0)
        per32 = st["ms_ebe32"] / active / 1e3
        gbs = bpe * E / per32 / 1e9
        matvec = {"kernel": "k_ebe<float> (inner FP32 EBE operator)", "bound": "hbm", "achieved": gbs,
                  "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak if hbm_peak else None,
                  "bytes_per_element": bpe, "nodes_per_element": n_per_e, "avg_active_launch_ms": per32 * 1e3,
                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    ebe64 = None
    if st["n_ebe64"] > 0 and st["ms_ebe64"] > 0:  # per-kernel events are not recorded inside graphs
        per64 = st["ms_ebe64"] / st["n_ebe64"] / 1e3
        ebe64 = {"kernel": "k_ebe<double> (FP64-accuracy operator)", "avg_launch_ms": per64 * 1e3,
                 "achieved_TFLOPs": EBE_FLOP_PER_ELEM * E / per64 / 1e12,
                 "flop_per_element": EBE_FLOP_PER_ELEM}

    # end to end through the public API: input record from host, advance, surface read-back to host
    t0 = time.perf_counter()
    if ens:
        for m in range(M):
            B.ns_set_member_ground_motion(sim.ctx, m, ens.waves[m], wl.dt)
        h2d = sum(w.nbytes for w in ens.waves) / args.steps
    else:
        B.ns_set_ground_motion(sim.ctx, wave, wl.dt)
        h2d = wave.nbytes / args.steps
    sim.advance(args.steps)
    s = sim.surface(st["steps"] + 1, args.steps)
    e2e_s = time.perf_counter() - t0
    e2e_s, e2e_work = dist.reduce_time_and_work(dd, e2e_s, float(E * args.steps), device="cuda")
    d2h = sum(a.nbytes for a in s.values()) / args.steps
    e2e = {"value": e2e_work / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    phases = {k: st[k] / args.steps for k in ("ms_rhs", "ms_jacobi", "ms_solve", "ms_newmark", "ms_springs")}
    kernels = {"ebe64": {"launches_per_step": st["n_ebe64"] / args.steps,
                         "avg_ms": st["ms_ebe64"] / max(st["n_ebe64"], 1)},
               "ebe32": {"launches_per_step": st["n_ebe32"] / args.steps,
                         "avg_ms": st["ms_ebe32"] / max(st["n_ebe32"], 1),
                         "active_launches_per_step": st["inner_iters_total"] / args.steps,
                         "avg_active_ms": st["ms_ebe32"] / max(st["inner_iters_total"], 1)},
               "springs": {"launches_per_step": st["n_spring"] / args.steps,
                           "avg_ms": st["ms_spring"] / max(st["n_spring"], 1)}}
    sim_steps = sim.stats()["steps"]
    sim.close()
    del sim

    stream = None
    if ws == 1 and not args.no_stream and args.workload == "large" and not args.dims:
        link = link_probe()
        per_elem = B.ns_state_bytes(1, wl.n_springs)
        stream_elems = int(args.stream_gb * 1e9 / per_elem)
        budget = (E - stream_elems) * per_elem
        ring = args.ring_depth

        def streamed_run(mode):
            sim = B.Simulation(wl, device=local, timing=1, device_state_budget=budget, chunk_elems=100000,
                               ring_depth=ring, precision=prec, graphs=graphs, stage_elements=args.stage,
                               inner_max_iter=args.inner_iters, inner_tol=args.inner_tol, stream_mode=mode, x0_prev=int(args.x0 == "prev"),
                               pair_operator=args.pair_op, l2_prefetch=args.prefetch,
                               spring_tile_points=args.spring_tile, spring_tile_blocks=args.spring_blocks,
                               spring_tensor_cores=args.spring_tensor,
                               **(dict(multigrid=1, coarse_max_iter=args.coarse_iters, coarse_tol=args.coarse_tol)
                                  if args.multigrid else {}))
            sim.advance(1)
            B.ns_reset_stats(sim.ctx)
            h0 = sim.stats()
            sim.advance(2)
            st2 = sim.stats()
            sim.close()
            moved = (st2["h2d_bytes"] - h0["h2d_bytes"]) + (st2["d2h_bytes"] - h0["d2h_bytes"])
            early = st2["h2d_bytes_early"] - h0["h2d_bytes_early"]
            gbs = (moved - early) / (st2["ms_stream_wall"] / 1e3) / 1e9
            best = link["best_GBps"]["bidir"]
            return {"streamed_elems": st2["streamed_elems"], "bytes_per_step": moved / 2,
                    "early_h2d_bytes_per_step": early / 2,
                    "stream_GBps": gbs, "link_GBps_measured": best, "frac_of_link": gbs / best,
                    "frac_of_rated_link": gbs / C2C_RATED_GBPS,
                    "step_ms": st2["ms_advance"] / 2, "resident_step_ms": job_s / args.steps * 1e3,
                    "steps": "steps 2-3 from rest (the link rate does not depend on the strain level)"}

        stream = streamed_run(B.NS_STREAM_RING)
        stream.update({"window": "multi-spring phase start to last D2H; H2D issued at step start (overlapping the "
                                 "solve) excluded from the bytes", "chunk_elems": 100000, "ring_depth": ring,
                       "link_probe": link})
        if args.zero_copy:
            zc = streamed_run(B.NS_STREAM_ZERO_COPY)
            zc["window"] = ("multi-spring phase (the kernel reads and writes the pinned host state in place); "
                            "bytes = 40 B read + 40 B written per streamed spring")
            stream["zero_copy"] = zc

    # small summaries of the other single-GPU configurations (tiny plain-FP64 case, precision form)
    others = None
    if ws == 1 and args.workload == "large" and not args.dims and not args.no_others:
        others = {}
        for name, mk, solver, n_w, n_t in (("tiny_plain_fp64", synth.tiny_two_layer, B.NS_PREC_FP64, 10, 50),
                                           ("precision_form_fp16_tangent", synth.precision_form_model,
                                            B.NS_PREC_FP64_IR16, 3, 5)):
            w2 = mk()
            with B.Simulation(w2, device=local, timing=1, surface_ring_steps=n_t, precision=solver,
                              graphs=1, x0_prev=0) as s2:
                s2.advance(n_w)
                B.ns_reset_stats(s2.ctx)
                s2.advance(n_t)
                st3 = s2.stats()
            others[name] = {"workload": w2.name, "elements": w2.mesh.n_elems, "springs_per_point": w2.n_springs,
                            "solver": {B.NS_PREC_FP64: "fp64-pcg", B.NS_PREC_FP64_IR16: "fp64-ir16"}[solver],
                            "graphs": 1, "steps": [n_w + 1, n_w + n_t],
                            "value": w2.mesh.n_elems * n_t / (st3["ms_advance"] / 1e3), "unit": UNIT,
                            "ms_per_step": st3["ms_advance"] / n_t,
                            "cg_iters_per_step": st3["cg_iters_total"] / n_t}
        # the batched ensemble: 64 members on one shared 201,600-element mesh, 50 springs
        ens2 = synth.ensemble_members(M=64, nt=400)
        n_w, n_t = 3, 3
        with B.BatchSimulation(ens2, shared=True, device=local, timing=1, surface_ring_steps=n_t,
                               precision=B.NS_PREC_FP64_IR, graphs=1, x0_prev=0) as s2:
            s2.advance(n_w)
            B.ns_reset_stats(s2.ctx)
            s2.advance(n_t)
            st3 = s2.stats()
        e2 = ens2.mesh.n_elems * len(ens2.members)
        others["batched_ensemble_shared_mesh"] = {
            "workload": ens2.name, "members": len(ens2.members), "elements": e2,
            "springs_per_point": ens2.member(0).n_springs, "solver": "fp64-ir", "graphs": 1,
            "steps": [n_w + 1, n_w + n_t], "value": e2 * n_t / (st3["ms_advance"] / 1e3), "unit": UNIT,
            "ms_per_step": st3["ms_advance"] / n_t, "cg_iters_per_step": st3["cg_iters_total"] / n_t}
        del ens2
        # a short served trace (config-5 arrivals, soils and spring counts; sizes 50 k-500 k
        # elements, steps scaled to 2.5 %): one context per request, at most 4 in flight
        trace = synth.served_trace(R=8, step_scale=0.025, seed=5, e_lo=5e4, e_hi=5e5)
        srv = B.Server(device=local, pinned_budget=int(32e9), max_active=4, quantum_steps=16, batch=0)
        t0 = time.perf_counter()
        ids = []
        for r in trace:
            delay = r.arrival_s - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(r.workload, r.n_steps, precision=B.NS_PREC_FP64_IR, graphs=1))
        sts = [srv.wait(i, 600.0) for i in ids]
        wall = time.perf_counter() - t0
        srv.close()
        tts = np.array([x["t_done"] - x["t_submit"] for x in sts])
        others["served_short_trace"] = {
            "workload": "served: %d requests, Poisson arrivals 4/s, %d-%d elements, 20-150 springs, steps "
                        "U[1000,4000] x 0.025" % (len(trace), min(r.workload.mesh.n_elems for r in trace),
                                                   max(r.workload.mesh.n_elems for r in trace)),
            "mode": "one context per request, at most 4 in flight", "solver": "fp64-ir", "graphs": 1,
            "value": float(sum(x["elem_steps"] for x in sts)) / wall, "unit": UNIT,
            "time_to_solution_s": {"p50": float(np.percentile(tts, 50)), "p99": float(np.percentile(tts, 99))},
            "makespan_s": wall, "failed": int(sum(x["state"] != B.NS_CASE_DONE for x in sts))}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        v_omp, cores, desc_omp = oracle_sample(steps=2, column=(0, 0, 16, 16), omp=True)
        v_one, _, desc_one = oracle_sample(steps=1, column=(0, 0, 8, 8), omp=False)
        cpu = {"value": v_omp, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc_omp,
               "single_thread": {"value": v_one, "unit": UNIT, "cores": 1, "sample": desc_one}}

    state_gb = B.ns_state_bytes(E, wl.n_springs) / 1e9
    l2_note = ("inputs larger than L2: %.1f GB of spring state read and written per step, no flush needed" % state_gb
               if state_gb > 0.5 else "working set near L2 size (%.3f GB of spring state); no flush" % state_gb)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": job_s / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "arithmetic": ARITHMETIC,
                "data": "synthetic",
                "config": {"workload": wl.name, "elements": E, "nodes": wl.mesh.n_nodes * M, "members": M,
                           "springs_per_point": wl.n_springs, "dt": wl.dt, "cg_tol": 1e-8,
                           "numbering": args.numbering, "state": "resident in HBM (streamed form in state_stream)",
                           "mesh_storage": (None if ens is None else
                                            "disjoint union of member copies" if args.union else
                                            "one shared mesh (connectivity and geometry stored once)"),
                           "l2": l2_note, "parallelism": "replicas" if ws > 1 else "single GPU",
                           "input": "full-length record, 0.2 s taper" if lead else "record with 10% taper"},
                "timed_window": window,
                "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "matvec_roofline": matvec,
                "ebe64": ebe64, "cpu_baseline": cpu,
                "clocks": clocks, "phases_ms_per_step": phases, "cg_iters_per_step": st["cg_iters_total"] / args.steps,
                "inner_iters_last_step": st["inner_iters_last"], "kernels": kernels, "solver": args.solver,
                "graphs": graphs, "staged_operator": args.stage, "inner_iters": args.inner_iters,
                "inner_tol": args.inner_tol, "spring_tensor_cores": args.spring_tensor, "autotune": tuning,
                "multigrid": ({"coarse_max_iter": args.coarse_iters, "coarse_tol": args.coarse_tol}
                              if args.multigrid else None),
                "pair_operator": args.pair_op, "x0": args.x0, "l2_prefetch": args.prefetch,
                "local_gather": args.local_gather,
                "steps_taken": sim_steps, "state_stream": stream, "other_configs": others}
        print(json.dumps(line), flush=True)
    dist.finalize(dd)
    return 0


if __name__ == "__main__":
    sys.exit(main())
