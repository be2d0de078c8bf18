"""Measurement studies beyond the single-line benchmark.

    python -m paper_2405_19004_gb300.studies sweep [--dims 3 2] [--degrees 1..7]
    python -m paper_2405_19004_gb300.studies mixed

sweep -- smoother-only degree sweep: Q_k for k = 1..7 in 3D and 2D, the mesh
    level whose DoF count is closest (log scale) to 1e8 (3D) or 2.5e8 (2D),
    seeded N(0,1) vectors, FP32 and FP64, 20 multiplicative smoothing steps
    per point timed with CUDA events after two warm-up steps.  Reported:
    DoF/s, algorithmic GFLOP/s and their fraction of the FP32 / FP64 peak
    (measured by vps_fma_peak on the same GPU) and of the shared-memory
    roofline R = B F / (d_r + d_w) of Section 4.3 (Eq. 4.3), B = SMs x 32
    banks x 4 bytes x SM clock, with the kernel's own shared-memory words per
    patch (a model of the kernel's accesses; ncu's shared-memory byte
    counters are recorded beside it under profiles/).
mixed -- mixed precision (Section 4.2): 3D Q3 on 2^7 cells per direction,
    manufactured solution u = prod sin(pi x_t), two pre- and two
    post-smoothing steps, autotuned and graph-captured FP32 V-cycle inside
    FP64 CG to 1e-10, against the same solve with an FP64 V-cycle: time,
    iterations, L2 errors against u and the difference of the solutions.

Every number is measured on the GPU through the library's C ABI; the
arithmetic counts are the method's dense sum-factorised counts.
"""

import argparse
import json
import math
import time

FP32_LANES_PER_SM = 128                  # FP32 FMA lanes per SM


def fp32_peak(sm_count, sm_mhz):
    """FP32 CUDA-core peak in flop/s from the unit counts and the clock."""
    return sm_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6


def smem_bandwidth(sm_count, sm_mhz):
    """Shared-memory bandwidth of Section 4.3: SMs x 32 banks x 4 bytes x clock."""
    return sm_count * 32 * 4 * sm_mhz * 1e6


def device_peaks(vps, torch):
    """SM count, the SM clock the device reports as its maximum (nvidia-smi;
    2070 MHz if unavailable) and the measured FP32 / FP64 multiply-add
    throughput (vps_fma_peak) of the current device."""
    import subprocess
    stream = torch.cuda.current_stream()
    f32, _, sms = vps.vps_fma_peak(vps.VPS_FP32, stream)
    f64, _, _ = vps.vps_fma_peak(vps.VPS_FP64, stream)
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", str(torch.cuda.current_device())],
                             capture_output=True, text=True, timeout=20).stdout
        mhz = float(out.strip().splitlines()[0])
    except Exception:
        mhz = None
    return {"sm_count": sms, "sm_max_mhz": mhz or 2070.0, "sm_max_mhz_source":
            "nvidia-smi clocks.max.sm" if mhz else "assumed 2070 MHz",
            "fp32_fma_measured_flops": f32, "fp64_fma_measured_flops": f64}


def smoother_flops_per_patch(d, k, boundary=False):
    """Sum-factorised flops of one patch update (FMA = 2).

    Fused kernel: local residual on the interior rows from the whole closure,
    fast diagonalisation, x_I += u.
      3D: 4mn^3 + 6m^2n^2 + 4m^3n + 12m^4 + 4m^3;  2D: 4mn^2 + 4m^2n + 8m^3 + 4m^2.
    Boundary kernel (Section 3.2): the first contraction only needs the 8k
    face lines (2 in 2D) in full and 2 end nodes of the m^2 (m) interior
    lines; x_I = u.
      3D: 4m(8kn + 2m^2) + 6m^2n^2 + 4m^3n + 12m^4 + 3m^3;
      2D: 4m(2n + 2m) + 4m^2n + 8m^3 + 3m^2.
    """
    n, m = 2 * k + 1, 2 * k - 1
    if d == 3:
        s0 = 4 * m * (8 * k * n + 2 * m * m) if boundary else 4 * m * n ** 3
        upd = 3 * m ** 3 if boundary else 4 * m ** 3
        return s0 + 6 * m * m * n * n + 4 * m ** 3 * n + 12 * m ** 4 + upd
    s0 = 4 * m * (2 * n + 2 * m) if boundary else 4 * m * n * n
    upd = 3 * m * m if boundary else 4 * m * m
    return s0 + 4 * m * m * n + 8 * m ** 3 + upd


def paper_flops_per_patch(d, k):
    """Flops of one patch update by the plain sum-factorisation count of the
    method (Sections 2.4 and 3.1), the count the reported roofline fractions
    use: the local residual over the whole closure -- along each direction a
    mass and a stiffness contraction of the n-point lines, interior rows m
    for the last direction (3D: 2 (2 n^4) + 3 (2 n^3 m) + 2 (2 n m^3);
    2D: 2 (2 n^3) + 2 (2 n^2 m)) -- the fast diagonalisation (2 d (2 m^(d+1))
    + m^d) and the update (2 m^d).  The kernels execute fewer
    (smoother_flops_per_patch: the inner mass contraction shared by two
    terms; smoother_flops_executed_per_patch: the even/odd halves)."""
    n, m = 2 * k + 1, 2 * k - 1
    if d == 3:
        res = 4 * n ** 4 + 6 * n ** 3 * m + 4 * n * m ** 3
    else:
        res = 4 * n ** 3 + 4 * n * n * m
    return res + 2 * d * 2 * m ** (d + 1) + m ** d + 2 * m ** d


def smoother_flops_executed_per_patch(d, k, boundary=False):
    """Floating-point operations the kernels execute per patch (FMA = 2,
    multiply or add = 1) with the even/odd halves of the 1D matrices.

    A closure line (n = 2k+1 values) against one centrosymmetric patch matrix
    takes 2k^2 multiply-adds on its k+1 even and k odd parts (the dense
    product takes m n = 4k^2 - 1); the parts cost 2k additions, the interior
    outputs 2(k-1) more.  A fast-diagonalisation line (m = 2k-1 values) takes
    k^2 + (k-1)^2 multiply-adds (dense m^2) and 2(k-1) additions.  Stages as
    in the kernels: the first and middle fast-diagonalisation directions in
    registers for k <= 5.  The Boundary kernel's interior lines of the first
    contraction use their two end nodes only (one multiply and one
    multiply-add per output and matrix)."""
    n, m, h = 2 * k + 1, 2 * k - 1, k - 1
    close1 = 4 * k * k + 2 * h                      # one matrix on a split closure line, + combine
    split_n = 2 * k
    fd_line = 2 * (k * k + h * h) + 2 * h           # S or S^T on one interior line
    fuse = k <= 5
    if d == 3:
        full0 = split_n + 2 * close1
        s0 = (8 * k * full0 + m * m * 2 * 3 * m) if boundary else n * n * full0
        s1 = n * m * (2 * split_n + 3 * 4 * k * k + 2 * 2 * h)
        s2 = m * m * (2 * split_n + 2 * 4 * k * k + 2 * h + 2 * m + (fd_line if fuse else 0))
        if fuse:
            fd = m * m * (fd_line + (2 * fd_line + m) + fd_line)
        else:
            fd = m * m * (3 * fd_line + m + 2 * fd_line)
        final = m * m * (fd_line + (1 if boundary else 2) * m)
        return s0 + s1 + s2 + fd + final
    full0 = split_n + 2 * close1
    s0 = (2 * full0 + m * 2 * 3 * m) if boundary else n * full0
    s1 = m * (2 * split_n + 2 * 4 * k * k + 2 * h + 2 * m + (fd_line if fuse else 0))
    fd = m * ((2 * fd_line + m) if fuse else (3 * fd_line + m))
    final = m * (fd_line + (1 if boundary else 2) * m)
    return s0 + s1 + fd + final


def smoother_smem_words_per_patch(d, k, boundary=False):
    """Shared-memory words read + written per patch by the fused kernel (the
    Boundary kernel neither stages nor reads back the interior of x)."""
    n, m = 2 * k + 1, 2 * k - 1
    if d == 3:
        return 4 * n * n * m + 4 * n * m * m + (14 if boundary else 16) * m ** 3
    return 4 * n * m + 4 * m * m + (12 if boundary else 14) * m * m


def level_for(d, k, target):
    best, err = 1, float("inf")
    for L in range(1, 16):
        N = (k * 2 ** L + 1) ** d
        if N > 6e8:
            break
        e = abs(math.log(N / target))
        if e < err:
            best, err = L, e
    return best


def smoother_point(vps, torch, d, k, L, prec, apps, peaks, tune=False, tune_cache=None,
                   seed=None, schedule=None):
    """Times `apps` multiplicative smoothing steps of Q_k on level L (after two
    warm-up steps) and returns the measurement row; `schedule` pins the
    colour schedule (default: the handle's, autotuned with `tune`)."""
    P = vps.Poisson(d, k, L, precision=prec)
    if tune:
        P.vps_autotune(tune_cache)
    if schedule is not None:
        P.vps_set_colour_schedule(schedule)
    N = P.n_interior()
    gen = torch.Generator(device="cuda").manual_seed(2 + k if seed is None else seed)
    b = P.empty_level()
    x = P.empty_level()
    P.vps_pack(L, torch.randn(N, generator=gen, device="cuda", dtype=P.dtype), b)
    P.vps_pack(L, torch.randn(N, generator=gen, device="cuda", dtype=P.dtype), x)
    P.vps_smooth(L, b, x, 2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(P.stream)
    P.vps_smooth(L, b, x, apps)
    e1.record(P.stream)
    torch.cuda.synchronize()
    P.vps_check_waits()
    t = e0.elapsed_time(e1) / 1e3 / apps
    patches = (2 ** L - 1) ** d
    var, ppb = P.vps_get_smooth_variant(L)
    bnd = var // 3 in vps.BOUNDARY_KINDS
    fpp = smoother_flops_per_patch(d, k, bnd)
    flops = fpp * patches
    esz = 4 if prec == vps.VPS_FP32 else 8
    intensity = fpp / (esz * smoother_smem_words_per_patch(d, k, bnd))
    roof_smem = smem_bandwidth(peaks["sm_count"], peaks["sm_max_mhz"]) * intensity
    fp32 = prec == vps.VPS_FP32
    derived = fp32_peak(peaks["sm_count"], peaks["sm_max_mhz"]) if fp32 else None
    measured = peaks["fp32_fma_measured_flops" if fp32 else "fp64_fma_measured_flops"]
    executed = smoother_flops_executed_per_patch(d, k, bnd) * patches
    paper = paper_flops_per_patch(d, k) * patches
    row = {"dim": d, "degree": k, "level": L, "precision": "fp32" if fp32 else "fp64",
           "dofs": N, "ms_per_step": 1e3 * t, "dof_per_s": N / t,
           "gflops_paper_count": paper / t / 1e9,
           "frac_of_measured_fma_peak_paper_count": paper / t / measured,
           "gflops": flops / t / 1e9,
           "gflops_executed": executed / t / 1e9,
           "frac_of_measured_fma_peak": flops / t / measured,
           "frac_of_measured_fma_peak_executed": executed / t / measured,
           "frac_smem_roofline": flops / t / roof_smem, "smem_roofline_tflops": roof_smem / 1e12,
           "kernel": "boundary" if bnd else "fused", "patches_per_block": ppb,
           "colour_schedule": P.vps_get_colour_schedule()}
    if derived:
        row["frac_of_fp32_peak"] = flops / t / derived
        row["frac_of_fp32_peak_paper_count"] = paper / t / derived
    P.close()
    del b, x
    torch.cuda.empty_cache()
    return row


def sweep(args):
    import torch
    import paper_2405_19004_gb300 as vps
    peaks = device_peaks(vps, torch)
    print(json.dumps({"peaks": peaks}), flush=True)
    rows = []
    for d in args.dims:
        target = 1e8 if d == 3 else 2.5e8
        for k in args.degrees:
            L = level_for(d, k, target)
            for prec in (vps.VPS_FP32, vps.VPS_FP64):
                row = smoother_point(vps, torch, d, k, L, prec, args.apps, peaks, args.tune,
                                     args.tune_cache)
                rows.append(row)
                print(json.dumps(row), flush=True)
    return rows


def mixed_precision_solve(vps, torch, level=7, repeats=3, tune_cache=None):
    """The mixed-precision setting of Section 4.2 on 3D Q3 (see the module
    docstring); returns the record."""
    from synthetic import manufactured_sine
    d, k, L = 3, 3, level
    coef, freq = manufactured_sine(d)
    out = {"workload": f"3D Q{k}, 2^{L} cells per direction, u = prod sin(pi x_t), 2 pre / 2 post "
                       "smoothing, CG to 1e-10"}
    sols = {}
    for prec, name in ((vps.VPS_FP32, "fp32_mg"), (vps.VPS_FP64, "fp64")):
        P = vps.Poisson(d, k, L, precision=prec, n_pre=2, n_post=2)
        P.vps_autotune(tune_cache)
        N = P.n_interior()
        b = torch.zeros(N, dtype=torch.float64, device="cuda")
        P.vps_assemble_rhs_sines(coef, freq, b)
        x = torch.zeros_like(b)
        P.vps_solve(b, x, 1e-10, 100)  # warm-up (captures the graph)
        ts = []
        for _ in range(repeats):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, rel = P.vps_solve(b, x, 1e-10, 100)
            ts.append(time.perf_counter() - t0)
        out[name] = {"dofs": N, "time_to_1e-10_s": min(ts), "iterations": it, "rel_residual": rel,
                     "l2_error": P.vps_l2_error_sine(x), "coarse_level": P.vps_get_coarse_level()}
        sols[name] = x.clone()
        P.close()
        del b, x
        torch.cuda.empty_cache()
    diff = (sols["fp32_mg"] - sols["fp64"]).abs().max().item() / sols["fp64"].abs().max().item()
    out["solution_rel_maxdiff"] = diff
    out["speedup_fp32_mg_over_fp64"] = out["fp64"]["time_to_1e-10_s"] / out["fp32_mg"]["time_to_1e-10_s"]
    return out


def mixed(args):
    import torch
    import paper_2405_19004_gb300 as vps
    out = mixed_precision_solve(vps, torch, args.level, args.repeats, args.tune_cache)
    print(json.dumps(out), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    s = sub.add_parser("sweep")
    s.add_argument("--dims", type=int, nargs="+", default=[3, 2])
    s.add_argument("--degrees", type=int, nargs="+", default=list(range(1, 8)))
    s.add_argument("--apps", type=int, default=20)
    s.add_argument("--tune", action="store_true")
    s.add_argument("--tune-cache", default=None)
    m = sub.add_parser("mixed")
    m.add_argument("--level", type=int, default=7)
    m.add_argument("--repeats", type=int, default=3)
    m.add_argument("--tune-cache", default=None)
    a = ap.parse_args()
    if a.cmd == "sweep":
        sweep(a)
    else:
        mixed(a)


if __name__ == "__main__":
    main()
