"""Shared helpers of the GPU parity tests (test infrastructure)."""

import functools

import numpy as np

from oracle import assembly, fe, smoothers

TOL = {0: 1e-12, 1: 1e-5}   # relative 2-norm error: FP64 / FP32 smoother applications


@functools.lru_cache(maxsize=None)
def oracle_level(d, k, l):
    lv = fe.Level(d, k, l)
    A = assembly.stiffness(lv)
    ps = smoothers.PatchSolver(lv, A) if l >= 1 else None
    return lv, A, ps


@functools.lru_cache(maxsize=None)
def oracle_prolongation(d, k, l):
    return assembly.prolongation(fe.Level(d, k, l))


def rel_err(got, ref):
    """The larger of the relative 2-norm error and the largest element error
    relative to the largest element of ref: a single bad element cannot hide
    under the norm of a long vector."""
    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    if ref.size == 0:
        return 0.0 if got.size == 0 else np.inf
    den2 = np.linalg.norm(ref)
    deninf = np.max(np.abs(ref))
    e = got - ref
    if not np.all(np.isfinite(e)):
        return np.inf
    r2 = np.linalg.norm(e) / (den2 if den2 > 0 else 1.0)
    rinf = np.max(np.abs(e)) / (deninf if deninf > 0 else 1.0)
    return max(r2, rinf)


def as_prec(v, prec):
    """Round an FP64 input to the working precision (FP32 inputs feed both sides)."""
    return np.asarray(v, dtype=np.float32).astype(np.float64) if prec == 1 else np.asarray(v)


def to_dev(P, compact, level):
    import torch
    t = torch.as_tensor(np.asarray(compact), dtype=P.dtype, device="cuda")
    return P.to_level(t, level)


def to_host(P, lev, level):
    return P.to_compact(lev, level).double().cpu().numpy()
