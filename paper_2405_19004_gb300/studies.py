"""Measurement studies beyond the single-line benchmark.

    python -m paper_2405_19004_gb300.studies sweep [--dims 3 2] [--degrees 1..7]
    python -m paper_2405_19004_gb300.studies mixed

sweep -- smoother-only degree sweep: Q_k for k = 1..7 in 3D and 2D, the mesh
    level whose DoF count is closest (log scale) to 1e8 (3D) or 2.5e8 (2D),
    seeded N(0,1) vectors, FP32 and FP64, 20 multiplicative smoothing steps
    per point timed with CUDA events after two warm-up steps.  Reported:
    DoF/s, algorithmic GFLOP/s and their fraction of the FP32 / FP64 peak and
    of the shared-memory roofline R = B F / (d_r + d_w) of Section 4.3 (Eq.
    4.3), B = 152 SMs x 32 banks x 4 bytes x 2.07 GHz, with the kernel's own
    shared-memory words per patch.
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

FP32_PEAK = 152 * 128 * 2 * 2.07e9      # flop/s, FP32 pipe at the maximum SM clock
FP64_PEAK = 1.25e12                      # flop/s, nominal GB300 FP64
SMEM_BW = 152 * 32 * 4 * 2.07e9          # bytes/s, shared memory (banks x word x clock)


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


def sweep(args):
    import torch
    import paper_2405_19004_gb300 as vps
    from synthetic import normal_vector
    rows = []
    for d in args.dims:
        target = 1e8 if d == 3 else 2.5e8
        for k in args.degrees:
            L = level_for(d, k, target)
            for prec, name in ((vps.VPS_FP32, "fp32"), (vps.VPS_FP64, "fp64")):
                P = vps.Poisson(d, k, L, precision=prec)
                if args.tune:
                    P.vps_autotune(args.tune_cache)
                N = P.n_interior()
                gen = torch.Generator(device="cuda").manual_seed(2 + k)
                b = P.empty_level()
                x = P.empty_level()
                P.vps_pack(L, torch.randn(N, generator=gen, device="cuda", dtype=P.dtype), b)
                P.vps_pack(L, torch.randn(N, generator=gen, device="cuda", dtype=P.dtype), x)
                P.vps_smooth(L, b, x, 2)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(P.stream)
                P.vps_smooth(L, b, x, args.apps)
                e1.record(P.stream)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / 1e3 / args.apps
                patches = (2 ** L - 1) ** d
                var, ppb = P.vps_get_smooth_variant(L)
                bnd = var // 3 >= 1
                fpp = smoother_flops_per_patch(d, k, bnd)
                flops = fpp * patches
                esz = 4 if prec == vps.VPS_FP32 else 8
                intensity = fpp / (esz * smoother_smem_words_per_patch(d, k, bnd))
                roof_smem = SMEM_BW * intensity
                peak = FP32_PEAK if prec == vps.VPS_FP32 else FP64_PEAK
                row = {"dim": d, "degree": k, "level": L, "precision": name, "dofs": N,
                       "ms_per_step": 1e3 * t, "dof_per_s": N / t, "gflops": flops / t / 1e9,
                       "frac_fp_peak": flops / t / peak, "frac_smem_roofline": flops / t / roof_smem,
                       "smem_roofline_tflops": roof_smem / 1e12,
                       "kernel": "boundary" if bnd else "fused", "patches_per_block": ppb}
                rows.append(row)
                print(json.dumps(row), flush=True)
                P.close()
                del b, x
                torch.cuda.empty_cache()
    return rows


def mixed(args):
    import torch
    import paper_2405_19004_gb300 as vps
    from synthetic import manufactured_sine
    d, k, L = 3, 3, args.level
    coef, freq = manufactured_sine(d)
    out = {"workload": f"3D Q{k}, 2^{L} cells per direction, u = prod sin(pi x_t), 2 pre / 2 post "
                       "smoothing, CG to 1e-10"}
    sols = {}
    for prec, name in ((vps.VPS_FP32, "fp32_mg"), (vps.VPS_FP64, "fp64")):
        P = vps.Poisson(d, k, L, precision=prec, n_pre=2, n_post=2)
        P.vps_autotune(args.tune_cache)
        N = P.n_interior()
        b = torch.zeros(N, dtype=torch.float64, device="cuda")
        P.vps_assemble_rhs_sines(coef, freq, b)
        x = torch.zeros_like(b)
        P.vps_solve(b, x, 1e-10, 100)  # warm-up (captures the graph)
        ts = []
        for _ in range(args.repeats):
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, rel = P.vps_solve(b, x, 1e-10, 100)
            ts.append(time.perf_counter() - t0)
        out[name] = {"dofs": N, "time_to_1e-10_s": min(ts), "iterations": it, "rel_residual": rel,
                     "l2_error": P.vps_l2_error_sine(x), "coarse_level": P.vps_get_coarse_level()}
        sols[name] = x.clone()
        P.close()
    diff = (sols["fp32_mg"] - sols["fp64"]).abs().max().item() / sols["fp64"].abs().max().item()
    out["solution_rel_maxdiff"] = diff
    out["speedup_fp32_mg_over_fp64"] = out["fp64"]["time_to_1e-10_s"] / out["fp32_mg"]["time_to_1e-10_s"]
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
