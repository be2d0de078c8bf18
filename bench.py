#!/usr/bin/env python
"""Benchmark of the vertex-patch multigrid solver on one GB300 (or N replicas).

Workload (one "step"): a V-cycle-preconditioned CG solve to a relative
residual of 1e-10 of the 3D Poisson problem with Q4 elements on 32^3 cells
(129^3 nodes, 2,048,383 interior DoFs), seeded random right-hand side in
[-1, 1], colour-multiplicative vertex-patch smoother (1 pre / 1 post step),
FP32 V-cycle inside FP64 CG.  The step runs every row of the hot path:
fused patch smoother, matrix-free operator, transfers, V-cycle (captured as
a CUDA graph) and CG.

Printed (rank 0, one JSON line): value = interior DoFs solved per second
over all ranks; e2e = the same through the host-buffer entry point
(vps_solve_host, host<->device copies included); roofline of the dominant
kernel (the finest-level FP32 smoother colour pass); the time to 1e-10 of
the FP32-multigrid and FP64 solves; the oracle's CPU throughput.

N > 1 (torchrun): every rank solves its own independent problem (replicas,
weak scaling; the path has no data exchange between problems).
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "smoother DoF/s & % FP32/FP64 peak; time-to-1e-10 residual FP32-MG vs FP64; p50/p99"
D, K, L = 3, 4, 5
RTOL = 1e-10
FP32_LANES_PER_SM = 128        # FP32 FMA lanes per SM (Blackwell)
SCHEDULE_NAMES = {0: "colour passes, ordinary launches",
                  1: "colour passes, programmatic dependent launches",
                  2: "dataflow sweep (one launch per smoothing step)"}
CPU_SAMPLE_LEVEL = 4           # oracle sample: the same problem at level 4 (250,047 DoFs)
CPU_SAMPLE_REPEATS = 3         # best of 3 solves
REF_STEP_BUDGET_S = 240.0      # reference arm: whole run within about four minutes
REF_STEP_S_LEVEL4 = 4.0        # one oracle solve at level 4 on the GPU machine's host (3.05 s measured)


def smoother_traffic(variant, schedule):
    """DRAM bytes per launch of the timed smoother kernel on the finest level
    (a colour pass, or a whole step for the dataflow sweep) from the committed
    ncu record (dram__bytes_read.sum + dram__bytes_write.sum of the kernel,
    summarised in profiles/smoother_traffic_3d_q4_l5.md), or None if the
    record is for another variant or schedule or was taken before the kernel
    source last changed."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "smoother_traffic_3d_q4_l5.json")
    src = os.path.join(ROOT, "paper_2405_19004_gb300", "csrc", "kernels_dk.cu")
    try:
        rec = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return None
    if rec.get("kernels_dk.cu sha256") != sha:
        return None
    key = f"{'sweep' if schedule == 2 else 'pass'}:{variant}"
    v = rec.get("traffic_bytes_per_launch", {}).get(key)
    return float(v) if v is not None else None


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the FP64 / additive side measurements")
    p.add_argument("--serving-requests", type=int, default=512,
                   help="requests of the serving measurement (0: skip it)")
    p.add_argument("--tune-cache", default=None,
                   help="autotuner cache file (reused when it holds this workload)")
    p.add_argument("--smoother-variant", type=int, default=None,
                   help="pin the finest level's smoother variant after tuning (profiling runs; "
                        "default: the autotuner's choice)")
    p.add_argument("--colour-schedule", type=int, default=None, choices=[0, 1, 2],
                   help="pin the colour schedule after tuning: 0 ordinary launches, 1 programmatic "
                        "dependent launches, 2 one dataflow sweep per smoothing step (profiling "
                        "runs; default: the autotuner's choice)")
    p.add_argument("--no-graphs", action="store_true",
                   help="launch every kernel directly (no CUDA graphs, host-driven CG iterations): "
                        "the same kernels, for profilers that do not follow graph conditional nodes")
    p.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--repeats", type=int, default=CPU_SAMPLE_REPEATS, help=argparse.SUPPRESS)
    p.add_argument("--cpu-level", type=int, default=CPU_SAMPLE_LEVEL, help=argparse.SUPPRESS)
    return p.parse_args()


# ---------------------------------------------------------------- oracle
def cpu_worker(repeats, level):
    """Times the oracle PCG solve (FP64, multiplicative V-cycle) on the host:
    setup (assembly, patch factorisations) once, then `repeats` solves."""
    import resource
    from oracle import multigrid
    from synthetic import uniform_vector
    t0 = time.perf_counter()
    H = multigrid.Hierarchy(D, K, level)
    setup = time.perf_counter() - t0
    N = H.levels[level].N
    b = uniform_vector(N, 1)
    times, its = [], []
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    w0 = time.perf_counter()
    for _ in range(repeats):
        t0 = time.perf_counter()
        _, it, rel = multigrid.pcg(H.A[level], b, H.precondition, RTOL, 100)
        times.append(time.perf_counter() - t0)
        its.append(it)
    wall = time.perf_counter() - w0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu_s = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    print(json.dumps({"n": N, "level": level, "times": times, "iters": its, "rel": rel,
                      "setup_s": setup, "cpu_s": cpu_s, "wall_s": wall,
                      "nnz": int(H.A[level].nnz)}))


def run_cpu_sample(repeats, level):
    """Runs cpu_worker in a fresh process with every BLAS allowed all host
    threads; returns its record plus the thread count and CPU model."""
    nthreads = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS=str(nthreads), OPENBLAS_NUM_THREADS=str(nthreads),
               MKL_NUM_THREADS=str(nthreads))
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker",
                          "--repeats", str(repeats), "--cpu-level", str(level)],
                         capture_output=True, text=True, env=env, cwd=ROOT, timeout=3600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    rec["threads_available"] = nthreads
    # threads it actually kept busy: CPU time over wall time of the solves
    rec["threads_used"] = max(1, int(round(rec["cpu_s"] / max(rec["wall_s"], 1e-9))))
    rec["cpu_model"] = cpu_model()
    return rec


def cpu_baseline_entry(rec, value, best=True):
    t = min(rec["times"]) if best else statistics.mean(rec["times"])
    return {"value": value, "unit": "DoF/s", "cores": rec["threads_used"], "kind": "oracle",
            "sample": sample_desc(rec, best),
            "threads_available": rec["threads_available"], "cpu_model": rec["cpu_model"],
            "level": rec["level"], "dofs": rec["n"], "seconds_per_solve": t,
            "setup_s": rec["setup_s"]}


def sample_desc(rec, best=True):
    n, lev, reps = rec["n"], rec["level"], len(rec["times"])
    how = f"best of {reps} solves" if best else f"mean of {reps} solves"
    return (f"oracle FP64 PCG (multiplicative V-cycle, 1/1 smoothing, sparse CSR matrices of "
            f"{rec['nnz']} nonzeros on the finest level) of the same 3D Q4 problem at level {lev} "
            f"({n} DoFs; the workload is level {L}: its CSR matrix alone would hold 1.5e9 "
            f"nonzeros), {how}, setup ({rec['setup_s']:.1f} s) excluded, BLAS threads "
            f"{rec['threads_available']} (the sparse products run on one thread), "
            f"CPU {rec['cpu_model']}")


def config(extra=None):
    c = {"workload": f"3D Poisson, Q{K}, 2^{L} cells/dir (129^3 nodes, 2048383 interior DoFs), "
                     f"random RHS U[-1,1] seed 1, V-cycle-preconditioned CG to {RTOL:g}",
         "dim": D, "degree": K, "level": L, "smoother": "multiplicative (8 colours), 1 pre / 1 post",
         "precision": "FP32 V-cycle, FP64 CG", "l2": "flushed between timed steps (256 MB write)"}
    if extra:
        c.update(extra)
    return c


def run_reference(args, rank, world):
    if rank != 0:
        return
    W, Kst = args.warmup, args.steps
    # each step one oracle solve at level 4, unless W + K of them would not
    # finish within about four minutes: then at level 3 (29,791 DoFs)
    level = CPU_SAMPLE_LEVEL if (W + Kst) * REF_STEP_S_LEVEL4 <= REF_STEP_BUDGET_S else 3
    res = run_cpu_sample(W + Kst, level)
    t = res["times"][W:]
    res_t = dict(res, times=t)
    n = res["n"]
    value = n / statistics.mean(t)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s",
            "n_gpus": args.gpus, "steps": Kst, "warmup": W,
            "ms_per_step": 1e3 * statistics.mean(t), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config({"sample": f"level {level} ({n} DoFs)"}),
            "cpu_baseline": cpu_baseline_entry(res_t, value, best=False),
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- replicas
def max_over_ranks(value, dist):
    """The largest of a rank-local number over all ranks (the number itself
    without a process group): the step time every rank waits for."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, t_step, world):
    """Whole-job throughput of `world` replicas that each process
    units_per_rank per step, the step taking t_step (the maximum over ranks)."""
    return world * units_per_rank / t_step


# ---------------------------------------------------------------- serving
def run_serving(vps, n_requests, precision, max_active, budget, closed_loop=False):
    """Replays a seeded Poisson-arrival stream of solve requests in real time;
    closed_loop: submits the same requests all at once, so that the span
    measures the server's capacity (the rate at which it drains a full
    queue) rather than the offered rate."""
    from synthetic import request_stream
    reqs = request_stream(n_requests, 200.0, seed=5)
    srv = vps.Server(budget, max_active=max_active, precision=precision, rtol=RTOL, max_it=200)
    ids, dofs = [], []
    t0 = time.perf_counter()
    for r in reqs:
        delay = t0 + r["t_arrival"] - time.perf_counter()
        if delay > 0 and not closed_loop:
            time.sleep(delay)
        rid, x = srv.submit(r["d"], r["k"], r["level"], r["coef"], r["freq"])
        ids.append(rid)
        dofs.append(len(x))
    srv.wait(0, 3600)
    t_end = time.perf_counter()
    info = [srv.query(i) for i in ids]
    batch = srv.batch_stats()
    host = srv.host_times()
    srv.close()
    lat = sorted(q["latency_s"] for q in info)
    ok = sum(q["state"] == vps.VPS_REQ_DONE for q in info)
    pct = lambda p: lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]
    span = t_end - t0
    if closed_loop:
        return {"requests": len(ids), "completed": ok, "span_s": span,
                "capacity_req_per_s": len(ids) / span, "capacity_dof_per_s": sum(dofs) / span,
                "max_active": max_active, "batching": batch}
    return {"requests": len(ids), "completed": ok, "p50_latency_s": pct(50), "p99_latency_s": pct(99),
            "mean_latency_s": sum(lat) / len(lat), "span_s": span,
            "throughput_req_per_s": len(ids) / span, "throughput_dof_per_s": sum(dofs) / span,
            "offered_req_per_s": len(reqs) / reqs[-1]["t_arrival"],
            "max_active": max_active, "batching": batch, "host_seconds": host}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if self.uuid:
            mine = [r for r in rows if len(r) > 1 and self.uuid in r[1]]
            rows = mine or rows
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[2]))
                mx = float(r[3])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[6:10]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.cpu_worker:
        cpu_worker(args.repeats, args.cpu_level)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    # the oracle's host sample runs first, in a fresh process, before any CUDA call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_sample(CPU_SAMPLE_REPEATS, CPU_SAMPLE_LEVEL)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2405_19004_gb300 as vps
    from paper_2405_19004_gb300.studies import (device_peaks, fp32_peak, mixed_precision_solve,
                                                paper_flops_per_patch,
                                                smem_bandwidth, smoother_flops_executed_per_patch,
                                                smoother_flops_per_patch, smoother_point,
                                                smoother_smem_words_per_patch)
    from synthetic import uniform_vector

    # roofline denominators of this device: SM count, maximum SM clock, and the
    # measured FP32 / FP64 multiply-add throughput (vps_fma_peak)
    peaks = device_peaks(vps, torch)
    props = torch.cuda.get_device_properties(local)
    peaks["sm_count_torch"] = props.multi_processor_count

    P = vps.Poisson(D, K, L, precision=vps.VPS_FP32, smoother=vps.VPS_MULTIPLICATIVE)
    P.vps_autotune(args.tune_cache)  # timed trials on this GPU, before the timed region
    if args.smoother_variant is not None:
        P.vps_set_smooth_variant(L, args.smoother_variant)
    if args.colour_schedule is not None:
        P.vps_set_colour_schedule(args.colour_schedule)
    schedule = P.vps_get_colour_schedule()
    if args.no_graphs:
        P.vps_set_graphs(False)
    tuned = {"coarse_level": P.vps_get_coarse_level(),
             "coarse_solver": (("one cooperative launch" if P.vps_get_coarse_solver() &
                                vps.VPS_COARSE_COOPERATIVE else "one launch per pass") +
                               (", 64-output tiles" if P.vps_get_coarse_solver() &
                                vps.VPS_COARSE_WIDE_TILES else ", 32-output tiles")),
             "smoother_variants": [P.vps_get_smooth_variant(l)[0] for l in range(1, L + 1)],
             "patches_per_block": [P.vps_get_smooth_variant(l)[1] for l in range(1, L + 1)],
             "finest_variant_pinned": args.smoother_variant is not None,
             "colour_schedule": SCHEDULE_NAMES[schedule],
             "colour_schedule_pinned": args.colour_schedule is not None,
             "cuda_graphs": not args.no_graphs}
    N = P.n_interior()
    b = torch.as_tensor(uniform_vector(N, 1 + rank), device="cuda")
    x = torch.zeros_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = P.stream

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def nvtx(name):
        """Push/pop NVTX range (profilers filter the timed region by it); no-op if unavailable."""
        import contextlib
        try:
            return torch.cuda.nvtx.range(name)
        except Exception:
            return contextlib.nullcontext()

    its = []
    for _ in range(args.warmup):
        it, rel = P.vps_solve(b, x, RTOL, 100)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    launches0 = P.vps_kernel_launches()
    barrier()
    times = []
    with nvtx("timed_solves"):
        for _ in range(args.steps):
            flush.zero_()
            stream.wait_stream(torch.cuda.current_stream())
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, rel = P.vps_solve(b, x, RTOL, 100)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            its.append(it)
    barrier()
    launches = P.vps_kernel_launches() - launches0
    clocks = sampler.stop()
    t_step = max_over_ranks(statistics.mean(times), dist)
    value = job_throughput(N, t_step, world)

    # end to end through the host-buffer entry point (copies inside)
    bh = torch.as_tensor(uniform_vector(N, 1 + rank)).pin_memory()
    xh = torch.zeros(N, dtype=torch.float64).pin_memory()
    P.vps_solve_host(bh, xh, RTOL, 100)
    e2e_t = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.vps_solve_host(bh, xh, RTOL, 100)
        e2e_t.append(time.perf_counter() - t0)
    t_e2e = max_over_ranks(statistics.mean(e2e_t), dist)

    # dominant kernel: the finest-level FP32 smoother (same kernel and data sizes
    # as in the solve), CUDA events on the library's stream.  Dataflow sweep: one
    # launch per smoothing step, timed launch by launch.  Colour passes: around
    # each run of the 8 passes of a step, launched back to back as in the V-cycle
    # (programmatic dependent launches: a pass is scheduled while the previous one
    # drains, which an event between two passes would prevent); the average
    # launch duration is the run's time / 8
    lib = vps.lib()
    import ctypes
    bs = P.to_level(b.float())
    xs = P.empty_level()
    torch.cuda.synchronize()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    n_rep = 20
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(n_rep)]
    sweep = schedule == vps.VPS_SCHEDULE_SWEEP

    def smoother_launches():
        if sweep:
            vps._check(lib.vps_smooth(P.h, L, ptr(bs), ptr(xs), 1), P.h)
        else:
            for c in range(8):
                vps._check(lib.vps_smooth_colour(P.h, L, c, ptr(bs), ptr(xs)), P.h)

    smoother_launches()  # warm-up
    with nvtx("smoother_colour_passes"):
        for r in range(n_rep):
            a, z = evs[r]
            a.record(stream)
            smoother_launches()
            z.record(stream)
        torch.cuda.synchronize()
    P.vps_check_waits()
    per_run = 1 if sweep else 8
    launch_ms = [a.elapsed_time(z) / per_run for a, z in evs]
    t_launch = statistics.mean(launch_ms) / 1e3
    n_patches = (2 ** L - 1) ** 3
    var_L = P.vps_get_smooth_variant(L)[0]
    bnd_L = var_L // 3 in vps.BOUNDARY_KINDS
    # algorithmic work per launch: the method's plain sum-factorisation count
    # per patch x the patches of the launch (the kernels' own dense and
    # executed counts are reported beside it)
    flops_per_launch = paper_flops_per_patch(D, K) * n_patches / per_run
    dense_per_launch = smoother_flops_per_patch(D, K, bnd_L) * n_patches / per_run
    # FP32 peak from the unit counts and the device's maximum SM clock; the
    # shared-memory roofline of Section 4.3 at the SM clock sampled under load
    fp32_peak_tflops = fp32_peak(peaks["sm_count"], peaks["sm_max_mhz"]) / 1e12
    smem_mhz = clocks.get("sm_mhz") or peaks["sm_max_mhz"]
    smem_words = smoother_smem_words_per_patch(D, K, bnd_L)
    smem_roof_tflops = smem_bandwidth(peaks["sm_count"], smem_mhz) * smoother_flops_per_patch(
        D, K, bnd_L) / (4.0 * smem_words) / 1e12
    achieved = flops_per_launch / t_launch / 1e12
    achieved_dense = dense_per_launch / t_launch / 1e12
    executed_per_launch = smoother_flops_executed_per_patch(D, K, bnd_L) * n_patches / per_run
    t_smooth_step = per_run * t_launch

    extras = {}
    if not args.no_extras and rank == 0:
        # FP64 V-cycle solve (time to 1e-10 in double precision)
        P64 = vps.Poisson(D, K, L, precision=vps.VPS_FP64)
        P64.vps_autotune(args.tune_cache)
        x64 = torch.zeros_like(b)
        P64.vps_solve(b, x64, RTOL, 100)
        t64 = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it64, rel64 = P64.vps_solve(b, x64, RTOL, 100)
            t64.append(time.perf_counter() - t0)
        # FP64 smoother step for the FP64 fraction of peak
        bs64 = P64.to_level(b)
        xs64 = P64.empty_level()
        P64.vps_smooth(L, bs64, xs64, 1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(P64.stream)
        for _ in range(3):
            vps._check(lib.vps_smooth(P64.h, L, ptr(bs64), ptr(xs64), 1), P64.h)
        e1.record(P64.stream)
        torch.cuda.synchronize()
        t64_step = e0.elapsed_time(e1) / 3e3
        bnd64 = P64.vps_get_smooth_variant(L)[0] // 3 in vps.BOUNDARY_KINDS
        f64 = smoother_flops_per_patch(D, K, bnd64) * n_patches / t64_step / 1e12
        f64x = smoother_flops_executed_per_patch(D, K, bnd64) * n_patches / t64_step / 1e12
        dx = (x64 - x).abs().max().item() / x64.abs().max().item()
        f64_peak = peaks["fp64_fma_measured_flops"] / 1e12
        extras = {
            "time_to_1e-10_s": {"fp32_mg": t_step, "fp64": min(t64), "speedup": min(t64) / t_step},
            "iterations": {"fp32_mg": its[-1], "fp64": it64},
            "fp32_vs_fp64_solution_rel_maxdiff": dx,
            "smoother_fp64": {"dof_per_s": N / t64_step, "tflops": f64,
                              "frac_of_fp64_peak": f64 / f64_peak, "peak_tflops": f64_peak,
                              "tflops_executed": f64x, "frac_of_fp64_peak_executed": f64x / f64_peak,
                              "peak_source": "measured FP64 multiply-add throughput (vps_fma_peak)",
                              "flops_note": "tflops: the method's dense sum-factorised count; "
                                            "executed: what the even/odd kernels issue"},
        }
        # one point of the degree sweep at about 1e8 DoFs (3D Q4 on 2^7 cells,
        # 1.35e8 DoFs), FP32 and FP64, 20 smoothing steps each
        extras["smoother_3d_q4_l7"] = [
            smoother_point(vps, torch, 3, 4, 7, prec, 20, peaks, True, args.tune_cache)
            for prec in (vps.VPS_FP32, vps.VPS_FP64)]
        # the small 2D workload: Q2 on 16 x 16 cells, f from u = sin(pi x) sin(pi y);
        # one FP64 multiplicative smoothing step on a seeded N(0,1) vector, then the
        # FP64 V-cycle-preconditioned CG to 1e-10
        from synthetic import manufactured_sine, normal_vector
        P2 = vps.Poisson(2, 2, 4, precision=vps.VPS_FP64)
        N2 = P2.n_interior()
        coef2, freq2 = manufactured_sine(2)
        b2 = torch.zeros(N2, dtype=torch.float64, device="cuda")
        P2.vps_assemble_rhs_sines(coef2, freq2, b2)
        xs2 = P2.to_level(torch.as_tensor(normal_vector(N2, 0), device="cuda"))
        bs2 = P2.to_level(b2)
        P2.vps_smooth(4, bs2, xs2, 1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(P2.stream)
        for _ in range(20):
            vps._check(lib.vps_smooth(P2.h, 4, ptr(bs2), ptr(xs2), 1), P2.h)
        e1.record(P2.stream)
        torch.cuda.synchronize()
        t2s = e0.elapsed_time(e1) / 20e3
        x2 = torch.zeros_like(b2)
        P2.vps_solve(b2, x2, RTOL, 100)
        t2 = []
        for _ in range(5):
            x2.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it2, rel2 = P2.vps_solve(b2, x2, RTOL, 100)
            t2.append(time.perf_counter() - t0)
        extras["poisson_2d_q2_l4_fp64"] = {
            "dofs": N2, "smoother_step_s": t2s, "smoother_dof_per_s": N2 / t2s,
            "cg_time_to_1e-10_s": min(t2), "iterations": it2, "rel_residual": rel2,
            "l2_error": P2.vps_l2_error_sine(x2)}
        P2.close()
        # the mixed-precision setting: 3D Q3 on 2^7 cells, manufactured sine, 2/2
        # smoothing, FP32 V-cycle in FP64 CG against the FP64 V-cycle, to 1e-10
        extras["mixed_precision_3d_q3_l7"] = mixed_precision_solve(vps, torch, 7, 3,
                                                                   args.tune_cache)
        # full multigrid (Algorithm 2) as a standalone solver, f = 1, tol 1e-9: the
        # setting of the paper's iteration-count tables
        fmg = {}
        for name, Pf in (("fp32_vcycle", P), ("fp64", P64)):
            xf = torch.zeros(N, dtype=torch.float64, device="cuda")
            Pf.vps_fmg([1.0], [0, 0, 0], xf, 1e-9, 100)
            tf = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                itf, relf = Pf.vps_fmg([1.0], [0, 0, 0], xf, 1e-9, 100)
                tf.append(time.perf_counter() - t0)
            fmg[name] = {"v_cycles": itf, "rel_residual": relf, "time_s": min(tf),
                         "coarse_level": Pf.vps_get_coarse_level()}
        extras["fmg_f1_tol1e-9"] = fmg
        # the paper's outer solver: flexible GMRES with the V-cycle of Algorithm 1,
        # u = prod sin(pi x_t), tol 1e-9, FP32 V-cycle / FP64 V-cycle
        from synthetic import manufactured_sine
        coef, freq = manufactured_sine(D)
        bs_ = torch.zeros(N, dtype=torch.float64, device="cuda")
        P.vps_assemble_rhs_sines(coef, freq, bs_)
        gm = {}
        for name, Pg in (("fp32_vcycle", P), ("fp64", P64)):
            xg = torch.zeros_like(bs_)
            Pg.vps_gmres(bs_, xg, 1e-9, 30, 300)
            tg = []
            for _ in range(3):
                xg.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                itg, relg = Pg.vps_gmres(bs_, xg, 1e-9, 30, 300)
                tg.append(time.perf_counter() - t0)
            gm[name] = {"iterations": itg, "rel_residual": relg, "time_s": min(tg),
                        "l2_error": Pg.vps_l2_error_sine(xg)}
        gm["speedup_fp32_vcycle"] = gm["fp64"]["time_s"] / gm["fp32_vcycle"]["time_s"]
        extras["gmres_sine_tol1e-9"] = gm
        # kernel structures of the smoother (Section 3.1): one multiplicative step
        # on the finest level, the tuned fused kernel against Separate, Global and
        # Global with the dense inverse (the "straightforward" implementation)
        abl = {}
        for pname, Pk in (("fp32", P), ("fp64", P64)):
            bk = Pk.to_level(b.to(Pk.dtype))
            xk = Pk.empty_level()
            row = {}
            for kind, kname in ((vps.VPS_KERNEL_FUSED, "fused"), (vps.VPS_KERNEL_SEPARATE, "separate"),
                                (vps.VPS_KERNEL_GLOBAL, "global"),
                                (vps.VPS_KERNEL_GLOBAL_INVERSE, "global_inverse_matrix")):
                Pk.vps_set_smoother_kernel(kind)
                Pk.vps_smooth(L, bk, xk, 2)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(Pk.stream)
                for _ in range(5):
                    vps._check(lib.vps_smooth(Pk.h, L, ptr(bk), ptr(xk), 1), Pk.h)
                e1.record(Pk.stream)
                torch.cuda.synchronize()
                ts = e0.elapsed_time(e1) / 5e3
                row[kname] = {"step_ms": 1e3 * ts, "dof_per_s": N / ts}
            Pk.vps_set_smoother_kernel(vps.VPS_KERNEL_FUSED)
            for kname in ("separate", "global", "global_inverse_matrix"):
                row["fused_speedup_over_" + kname] = row[kname]["step_ms"] / row["fused"]["step_ms"]
            abl[pname] = row
        extras["smoother_kernel_structures"] = abl
        P64.close()
        # additive smoother: damping 0.7 taken literally, and 0.7 of the stability limit
        add = {}
        for om in (0.7, 0.7 * 2 / 8):
            Pa = vps.Poisson(D, K, L, precision=vps.VPS_FP32, smoother=vps.VPS_ADDITIVE, damping=om)
            xa = torch.zeros_like(b)
            try:
                Pa.vps_solve(b, xa, RTOL, 200)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ita, rela = Pa.vps_solve(b, xa, RTOL, 200)
                add[f"omega_{om:g}"] = {"status": "converged", "iterations": ita,
                                        "time_s": time.perf_counter() - t0}
            except vps.VpsError as e:
                add[f"omega_{om:g}"] = {"status": str(e).split(":")[0]}
            Pa.close()
        extras["additive_fp32_mg"] = add

    if not args.no_extras and rank == 0 and args.serving_requests > 0:
        budget = 48 << 30
        extras["serving"] = {
            "workload": f"{args.serving_requests} requests, Poisson arrivals 200/s, d in {{2,3}}, "
                        "k in 2..6, levels with 1e4..2e7 DoFs, 4 sine modes, seed 5, CG to 1e-10",
            "fp32_mg_batched": run_serving(vps, args.serving_requests, vps.VPS_FP32, 16, budget),
            # the same requests queued at once: the rate the server sustains
            # (an open-loop stream cannot complete faster than it arrives)
            "fp32_mg_batched_capacity": run_serving(vps, args.serving_requests, vps.VPS_FP32, 16,
                                                    budget, closed_loop=True),
            "fp64_one_at_a_time": run_serving(vps, args.serving_requests, vps.VPS_FP64, 1, budget),
        }

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": config({"parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                          "autotuned": tuned}),
        "iterations": its[-1], "rel_residual": rel,
        "peaks": peaks,
        "smoother_fp32": {"dof_per_s": N / t_smooth_step, "tflops": achieved,
                          "frac_of_fp32_peak": achieved / fp32_peak_tflops,
                          "frac_of_measured_fma_peak":
                              achieved / (peaks["fp32_fma_measured_flops"] / 1e12),
                          # the kernel's own dense count (the inner mass contraction
                          # shared by two terms, Section 3.1.1)
                          "tflops_kernel_dense_count": achieved_dense,
                          "frac_of_fp32_peak_kernel_dense_count": achieved_dense / fp32_peak_tflops,
                          # shared-memory roofline R = B F / (d_r + d_w) (Section 4.3),
                          # B = SMs x 32 banks x 4 B x the SM clock sampled under load,
                          # F and d_r + d_w = the kernel's dense flops and modelled
                          # shared-memory words per patch
                          "frac_of_smem_roofline": achieved_dense / smem_roof_tflops,
                          "smem_roofline_tflops": smem_roof_tflops,
                          "smem_roofline_clock_mhz": smem_mhz,
                          "smem_words_per_patch_model": smem_words},
        "roofline": {"kernel": ("smooth_sweep_kernel<float> (3D, k=4), finest level, one launch "
                                "per smoothing step (all 8 colours), " if sweep else
                                "smooth_mult_kernel<float> (3D, k=4), finest level, one launch "
                                "per colour pass, ")
                               + ("Boundary" if bnd_L else "fused") + f" variant {var_L}",
                     "bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak_tflops,
                     "traffic": smoother_traffic(var_L, schedule),
                     "peak_source": f"{peaks['sm_count']} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                                    f"flop x {peaks['sm_max_mhz']:g} MHz ({peaks['sm_max_mhz_source']})"
                                    "; measured FMA throughput in peaks.fp32_fma_measured_flops",
                     "avg_launch_us": 1e6 * t_launch, "flops_per_launch": flops_per_launch,
                     "flops_count": "sum-factorisation count of the patch update, "
                                    f"{paper_flops_per_patch(D, K)} flop per patch x "
                                    f"{n_patches / per_run:g} "
                                    "patches per launch",
                     "kernel_dense_flops_per_launch": dense_per_launch,
                     "frac_kernel_dense_count": achieved_dense / fp32_peak_tflops,
                     "executed_flops_per_launch": executed_per_launch,
                     "frac_executed": executed_per_launch / t_launch / 1e12 / fp32_peak_tflops},
        "e2e": {"value": job_throughput(N, t_e2e, world), "unit": "DoF/s", "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 8 * N},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu_baseline_entry(cpu, cpu["n"] / min(cpu["times"]))
    line.update(extras)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
