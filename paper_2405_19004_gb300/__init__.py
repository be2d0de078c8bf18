"""GB300 vertex-patch multigrid for Q_k Poisson problems -- Python binding.

A thin ctypes binding over the C ABI of ``libvps.so`` (``include/vps.h``):
the functions below carry the same names as the C entry points and only
marshal arguments; every numerical step runs in the library's CUDA kernels.
PyTorch provides device memory and streams.

There is no CPU path: importing works without a GPU (so the library can be
inspected), but every call that computes needs the compiled library and a
CUDA device, and raises ``VpsError`` otherwise.
"""

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libvps.so")

VPS_OK = 0
VPS_EINVAL = -1
VPS_ENOMEM = -2
VPS_ECUDA = -3
VPS_ENOCONV = -4
VPS_EBREAKDOWN = -5
VPS_ETIMEOUT = -6
VPS_FP64 = 0
VPS_FP32 = 1
VPS_MULTIPLICATIVE = 0
VPS_ADDITIVE = 1
VPS_MAX_DEGREE = 7
VPS_KERNEL_FUSED, VPS_KERNEL_SEPARATE, VPS_KERNEL_GLOBAL, VPS_KERNEL_GLOBAL_INVERSE = 0, 1, 2, 3
VPS_OUTER_FP64 = 0
VPS_OUTER_DOUBLE_FLOAT = 1
VPS_SCHEDULE_PLAIN, VPS_SCHEDULE_PDL, VPS_SCHEDULE_SWEEP = 0, 1, 2
VPS_COARSE_PASSES, VPS_COARSE_COOPERATIVE, VPS_COARSE_WIDE_TILES = 0, 1, 2
VPS_REQ_QUEUED, VPS_REQ_RUNNING, VPS_REQ_DONE, VPS_REQ_FAILED = 0, 1, 2, 3
# smoother variants (vps_set_smooth_variant): variant = 3 * kind + block shape
VPS_SMOOTH_VARIANTS = 18
BOUNDARY_KINDS = (1, 2, 4)   # kinds whose kernel is the Boundary kernel of Section 3.2

# C signatures: name -> (restype, argtypes)
_i, _d, _p, _i64p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "vps_create": (_i, [_i, _i, _i, _i, _i, _d, _i, _i, _p, ctypes.POINTER(_p)]),
    "vps_destroy": (_i, [_p]),
    "vps_sizes": (_i, [_p, _i64p, _i64p, ctypes.POINTER(ctypes.c_size_t)]),
    "vps_level_layout": (_i, [_p, _i, _i64p, _i64p, _i64p]),
    "vps_pack": (_i, [_p, _i, _p, _p]),
    "vps_unpack": (_i, [_p, _i, _p, _p]),
    "vps_smooth": (_i, [_p, _i, _p, _p, _i]),
    "vps_smooth_colour": (_i, [_p, _i, _i, _p, _p]),
    "vps_apply": (_i, [_p, _i, _p, _p]),
    "vps_restrict": (_i, [_p, _i, _p, _p]),
    "vps_prolongate_add": (_i, [_p, _i, _p, _p]),
    "vps_vcycle": (_i, [_p, _p, _p]),
    "vps_solve": (_i, [_p, _p, _p, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "vps_solve_host": (_i, [_p, _p, _p, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "vps_gmres": (_i, [_p, _p, _p, _d, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "vps_assemble_rhs_sines": (_i, [_p, _i, _p, _p, _p]),
    "vps_l2_error_sine": (_i, [_p, _p, ctypes.POINTER(_d)]),
    "vps_fmg": (_i, [_p, _i, _p, _p, _d, _i, _p, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "vps_set_graphs": (_i, [_p, _i]),
    "vps_set_outer_operator": (_i, [_p, _i]),
    "vps_get_outer_operator": (_i, [_p, ctypes.POINTER(_i)]),
    "vps_apply_outer": (_i, [_p, _p, _p]),
    "vps_get_solve_info": (_i, [_p, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "vps_set_smoother_kernel": (_i, [_p, _i]),
    "vps_get_smoother_kernel": (_i, [_p, ctypes.POINTER(_i)]),
    "vps_kernel_launches": (_i, [_p, _i64p]),
    "vps_set_coarse_level": (_i, [_p, _i]),
    "vps_autotune": (_i, [_p, ctypes.c_char_p, ctypes.POINTER(_i)]),
    "vps_set_smooth_variant": (_i, [_p, _i, _i]),
    "vps_get_smooth_variant": (_i, [_p, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "vps_set_operator_variant": (_i, [_p, _i, _i]),
    "vps_get_operator_variant": (_i, [_p, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "vps_set_colour_schedule": (_i, [_p, _i]),
    "vps_get_colour_schedule": (_i, [_p, ctypes.POINTER(_i)]),
    "vps_check_waits": (_i, [_p]),
    "vps_set_coarse_solver": (_i, [_p, _i]),
    "vps_get_coarse_solver": (_i, [_p, ctypes.POINTER(_i)]),
    "vps_skip_sweep_tiles": (_i, [_p, _i, ctypes.c_int64]),
    "vps_get_coarse_level": (_i, [_p, ctypes.POINTER(_i)]),
    "vps_smooth_additive_static": (_i, [_i, _i, _i, _i, _d, _p, _p, _p]),
    "vps_server_create": (_i, [ctypes.c_size_t, _i, _i, _d, _i, ctypes.POINTER(_p)]),
    "vps_server_submit": (_i, [_p, _i, _i, _i, _i, _p, _p, _p, _i64p]),
    "vps_server_query": (_i, [_p, ctypes.c_int64, ctypes.POINTER(_i), ctypes.POINTER(_i),
                              ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(_d),
                              ctypes.POINTER(_d)]),
    "vps_server_wait": (_i, [_p, ctypes.c_int64, _d]),
    "vps_server_stats": (_i, [_p, _i64p, _i64p, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "vps_server_last_error": (ctypes.c_char_p, [_p]),
    "vps_server_batch_stats": (_i, [_p, _i64p, _i64p, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "vps_server_host_times": (_i, [_p, ctypes.POINTER(_d)]),
    "vps_server_destroy": (_i, [_p]),
    "vps_last_error": (ctypes.c_char_p, [_p]),
    "vps_status_string": (ctypes.c_char_p, [_i]),
    "vps_check_fp_conversions": (_i, [_p, ctypes.c_int64, _i64p, _p]),
    "vps_fma_peak": (_i, [_i, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_i), _p]),
}

_lib = None


class VpsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_status_name(code)} ({code}): {msg}")
        self.code = code


def _status_name(code):
    names = {0: "VPS_OK", -1: "VPS_EINVAL", -2: "VPS_ENOMEM", -3: "VPS_ECUDA",
             -4: "VPS_ENOCONV", -5: "VPS_EBREAKDOWN", -6: "VPS_ETIMEOUT"}
    return names.get(code, "VPS_UNKNOWN")


def lib():
    """The loaded library (raises VpsError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise VpsError(VPS_ECUDA, f"{LIB_PATH} missing: run __graft_entry__.build() first "
                                      "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _check(rc, handle=None):
    if rc != VPS_OK:
        msg = lib().vps_last_error(handle)
        raise VpsError(rc, msg.decode() if msg else "")
    return rc


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def vps_smooth_additive_static(dim, degree, level, precision, damping, b, x, stream):
    """One additive smoothing step without a handle and without allocating.

    b, x: CUDA tensors in the level layout of ``level`` (float32 for VPS_FP32,
    float64 for VPS_FP64); stream: a torch CUDA stream the call runs on.  The
    step's scratch lives in a fixed 32 MiB device array inside the library
    (larger levels are rejected); calls that overlap on one GPU race on it.
    """
    rc = lib().vps_smooth_additive_static(dim, degree, level, precision, float(damping), _ptr(b),
                                          _ptr(x), ctypes.c_void_p(stream.cuda_stream))
    return _check(rc, None)


def vps_fma_peak(precision, stream):
    """Measured FP32 / FP64 multiply-add throughput: (flop/s, seconds of the
    timed launch, multiprocessor count)."""
    f = ctypes.c_double()
    t = ctypes.c_double()
    sm = ctypes.c_int()
    rc = lib().vps_fma_peak(precision, ctypes.byref(f), ctypes.byref(t), ctypes.byref(sm),
                            ctypes.c_void_p(stream.cuda_stream))
    _check(rc, None)
    return f.value, t.value, sm.value


def vps_check_fp_conversions(patterns, stream):
    """Mismatch counts (f2d, d2f_rn, split) of the library's float/double
    conversions against the hardware ones on a CUDA int64 tensor of bit
    patterns (see vps.h)."""
    out = (ctypes.c_int64 * 3)()
    rc = lib().vps_check_fp_conversions(_ptr(patterns), patterns.numel(), out,
                                        ctypes.c_void_p(stream.cuda_stream))
    _check(rc, None)
    return list(out)


class Poisson:
    """One level hierarchy of -Laplace u = f on (0,1)^dim with Q_degree elements.

    Owns a ``vps_handle``; all its work runs on ``self.stream`` (a torch CUDA
    stream).  Each method makes the stream wait for the caller's current
    stream before the call and the current stream wait for it afterwards.
    """

    def __init__(self, dim, degree, level, precision=VPS_FP64, smoother=VPS_MULTIPLICATIVE,
                 damping=1.0, n_pre=1, n_post=1, stream=None, graphs=True, coarse_level=0):
        import torch
        self.torch = torch
        if not torch.cuda.is_available():
            raise VpsError(VPS_ECUDA, "no CUDA device (there is no CPU fallback)")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.dim, self.degree, self.level = dim, degree, level
        self.precision, self.smoother = precision, smoother
        h = ctypes.c_void_p()
        rc = lib().vps_create(dim, degree, level, precision, smoother, float(damping), n_pre, n_post,
                              ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != VPS_OK:
            raise VpsError(rc, lib().vps_last_error(None).decode())
        self.h = h
        if not graphs:
            _check(lib().vps_set_graphs(self.h, 0), self.h)
        if coarse_level:
            _check(lib().vps_set_coarse_level(self.h, int(coarse_level)), self.h)
        self.dtype = torch.float64 if precision == VPS_FP64 else torch.float32

    def close(self):
        if getattr(self, "h", None):
            lib().vps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- ordering with torch's current stream
    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream())

    def _leave(self):
        self.torch.cuda.current_stream().wait_stream(self.stream)

    def _call(self, fn, *args):
        self._enter()
        try:
            return _check(fn(self.h, *args), self.h)
        finally:
            self._leave()

    # --- sizes and layouts
    def sizes(self):
        n, p, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(lib().vps_sizes(self.h, ctypes.byref(n), ctypes.byref(p), ctypes.byref(b)), self.h)
        return n.value, p.value, b.value

    def layout(self, level=None):
        level = self.level if level is None else level
        n1, px, tot = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().vps_level_layout(self.h, level, ctypes.byref(n1), ctypes.byref(px),
                                      ctypes.byref(tot)), self.h)
        return n1.value, px.value, tot.value

    def empty_level(self, level=None, dtype=None):
        n1, px, tot = self.layout(level)
        return self.torch.zeros(tot, dtype=dtype or self.dtype, device="cuda")

    def n_interior(self, level=None):
        n1, _, _ = self.layout(level)
        return (n1 - 2) ** self.dim

    # --- entry points (same names as the C ABI)
    def vps_pack(self, level, compact, lev):
        self._call(lib().vps_pack, level, _ptr(compact), _ptr(lev))

    def vps_unpack(self, level, lev, compact):
        self._call(lib().vps_unpack, level, _ptr(lev), _ptr(compact))

    def vps_smooth(self, level, b, x, n_steps=1):
        self._call(lib().vps_smooth, level, _ptr(b), _ptr(x), n_steps)

    def vps_smooth_colour(self, level, colour, b, x):
        self._call(lib().vps_smooth_colour, level, colour, _ptr(b), _ptr(x))

    def vps_apply(self, level, x, y):
        self._call(lib().vps_apply, level, _ptr(x), _ptr(y))

    def vps_restrict(self, fine_level, rf, rc):
        self._call(lib().vps_restrict, fine_level, _ptr(rf), _ptr(rc))

    def vps_prolongate_add(self, fine_level, xc, xf):
        self._call(lib().vps_prolongate_add, fine_level, _ptr(xc), _ptr(xf))

    def vps_vcycle(self, b, x):
        self._call(lib().vps_vcycle, _ptr(b), _ptr(x))

    def vps_solve(self, b, x, rtol=1e-10, max_it=100):
        it, rel = ctypes.c_int(), ctypes.c_double()
        self._call(lib().vps_solve, _ptr(b), _ptr(x), float(rtol), int(max_it), ctypes.byref(it),
                   ctypes.byref(rel))
        return it.value, rel.value

    def vps_gmres(self, b, x, rtol=1e-9, restart=30, max_it=300):
        it, rel = ctypes.c_int(), ctypes.c_double()
        self._call(lib().vps_gmres, _ptr(b), _ptr(x), float(rtol), int(restart), int(max_it),
                   ctypes.byref(it), ctypes.byref(rel))
        return it.value, rel.value

    def vps_solve_host(self, b_host, x_host, rtol=1e-10, max_it=100):
        """b_host, x_host: CPU float64 tensors (pinned for full-speed copies)."""
        it, rel = ctypes.c_int(), ctypes.c_double()
        self._call(lib().vps_solve_host, _ptr(b_host), _ptr(x_host), float(rtol), int(max_it),
                   ctypes.byref(it), ctypes.byref(rel))
        return it.value, rel.value

    def vps_assemble_rhs_sines(self, coef, freq, b):
        import numpy as np
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        freq = np.ascontiguousarray(freq, dtype=np.int32)
        self._call(lib().vps_assemble_rhs_sines, len(coef), coef.ctypes.data_as(ctypes.c_void_p),
                   freq.ctypes.data_as(ctypes.c_void_p), _ptr(b))

    def vps_fmg(self, coef, freq, x, tol=1e-9, max_it=100):
        """Full multigrid (Algorithm 2) for f = sum coef prod sin(pi freq x_t)
        (freq 0: constant 1); x: compact float64 device output.  -> (V-cycles, rel)."""
        import numpy as np
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        freq = np.ascontiguousarray(freq, dtype=np.int32)
        it, rel = ctypes.c_int(), ctypes.c_double()
        self._call(lib().vps_fmg, len(coef), coef.ctypes.data_as(ctypes.c_void_p),
                   freq.ctypes.data_as(ctypes.c_void_p), float(tol), int(max_it), _ptr(x),
                   ctypes.byref(it), ctypes.byref(rel))
        return it.value, rel.value

    def vps_l2_error_sine(self, x):
        err = ctypes.c_double()
        self._call(lib().vps_l2_error_sine, _ptr(x), ctypes.byref(err))
        return err.value

    def vps_autotune(self, cache_path=None):
        """Tune smoother variants and the coarsest level; returns True if the
        settings came from the cache file."""
        fc = ctypes.c_int()
        path = cache_path.encode() if cache_path else None
        self._call(lib().vps_autotune, path, ctypes.byref(fc))
        return bool(fc.value)

    def vps_set_smooth_variant(self, level, variant):
        self._call(lib().vps_set_smooth_variant, int(level), int(variant))

    def vps_get_smooth_variant(self, level):
        v, p = ctypes.c_int(), ctypes.c_int()
        _check(lib().vps_get_smooth_variant(self.h, int(level), ctypes.byref(v), ctypes.byref(p)),
               self.h)
        return v.value, p.value

    def vps_set_operator_variant(self, level, variant):
        self._call(lib().vps_set_operator_variant, int(level), int(variant))

    def vps_get_operator_variant(self, level):
        v, n = ctypes.c_int(), ctypes.c_int()
        _check(lib().vps_get_operator_variant(self.h, int(level), ctypes.byref(v), ctypes.byref(n)),
               self.h)
        return v.value, n.value

    def vps_set_colour_schedule(self, schedule):
        self._call(lib().vps_set_colour_schedule, int(schedule))

    def vps_get_colour_schedule(self):
        e = ctypes.c_int()
        _check(lib().vps_get_colour_schedule(self.h, ctypes.byref(e)), self.h)
        return e.value

    def vps_check_waits(self):
        self._call(lib().vps_check_waits)

    def vps_set_coarse_solver(self, solver):
        self._call(lib().vps_set_coarse_solver, int(solver))

    def vps_get_coarse_solver(self):
        e = ctypes.c_int()
        _check(lib().vps_get_coarse_solver(self.h, ctypes.byref(e)), self.h)
        return e.value

    def vps_skip_sweep_tiles(self, level, tiles):
        self._call(lib().vps_skip_sweep_tiles, int(level), int(tiles))

    def vps_set_coarse_level(self, level):
        self._call(lib().vps_set_coarse_level, int(level))

    def vps_get_coarse_level(self):
        c = ctypes.c_int()
        _check(lib().vps_get_coarse_level(self.h, ctypes.byref(c)), self.h)
        return c.value

    def vps_kernel_launches(self):
        c = ctypes.c_int64()
        _check(lib().vps_kernel_launches(self.h, ctypes.byref(c)), self.h)
        return c.value

    def vps_set_graphs(self, enable):
        _check(lib().vps_set_graphs(self.h, int(bool(enable))), self.h)

    def vps_set_outer_operator(self, mode):
        _check(lib().vps_set_outer_operator(self.h, int(mode)), self.h)

    def vps_apply_outer(self, x, y):
        assert x.dtype == self.torch.float64 and y.dtype == self.torch.float64
        self._call(lib().vps_apply_outer, _ptr(x), _ptr(y))

    def vps_set_smoother_kernel(self, kind):
        _check(lib().vps_set_smoother_kernel(self.h, int(kind)), self.h)

    def vps_get_smoother_kernel(self):
        c = ctypes.c_int()
        _check(lib().vps_get_smoother_kernel(self.h, ctypes.byref(c)), self.h)
        return c.value

    def vps_get_solve_info(self):
        """(restarts, at_rounding_bound) of the last solve."""
        r, f = ctypes.c_int(), ctypes.c_int()
        _check(lib().vps_get_solve_info(self.h, ctypes.byref(r), ctypes.byref(f)), self.h)
        return r.value, f.value

    def vps_get_outer_operator(self):
        c = ctypes.c_int()
        _check(lib().vps_get_outer_operator(self.h, ctypes.byref(c)), self.h)
        return c.value

    # --- conveniences on compact vectors
    def to_level(self, compact, level=None):
        level = self.level if level is None else level
        lev = self.empty_level(level)
        self.vps_pack(level, compact.to(device="cuda", dtype=self.dtype).contiguous(), lev)
        return lev

    def to_compact(self, lev, level=None):
        level = self.level if level is None else level
        out = self.torch.empty(self.n_interior(level), dtype=lev.dtype, device="cuda")
        self.vps_unpack(level, lev, out)
        return out


class Server:
    """Continuous-batching solve server (vps_server_* of the C ABI).

    ``submit`` returns a request id and the numpy array that receives the
    solution (compact layout, float64); results arrive asynchronously.
    """

    def __init__(self, memory_budget, max_active=8, precision=VPS_FP32, rtol=1e-10, max_it=100):
        s = ctypes.c_void_p()
        rc = lib().vps_server_create(int(memory_budget), int(max_active), int(precision),
                                     float(rtol), int(max_it), ctypes.byref(s))
        if rc != VPS_OK:
            raise VpsError(rc, lib().vps_last_error(None).decode())
        self.s = s
        self._bufs = {}

    def submit(self, dim, degree, level, coef, freq):
        import numpy as np
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        freq = np.ascontiguousarray(freq, dtype=np.int32)
        n = (degree * 2 ** level - 1) ** dim
        # no host buffer for sizes the library rejects anyway (it checks the
        # level before anything else)
        x = np.zeros(n, dtype=np.float64) if n < 2 ** 31 else None
        rid = ctypes.c_int64()
        rc = lib().vps_server_submit(self.s, dim, degree, level, len(coef),
                                     coef.ctypes.data_as(ctypes.c_void_p),
                                     freq.ctypes.data_as(ctypes.c_void_p),
                                     None if x is None else x.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(rid))
        if rc != VPS_OK:
            raise VpsError(rc, "vps_server_submit")
        self._bufs[rid.value] = (x, coef, freq)
        return rid.value, x

    def query(self, rid):
        st, status, it = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rel, qs, lat = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        rc = lib().vps_server_query(self.s, int(rid), ctypes.byref(st), ctypes.byref(status),
                                    ctypes.byref(it), ctypes.byref(rel), ctypes.byref(qs),
                                    ctypes.byref(lat))
        if rc != VPS_OK:
            raise VpsError(rc, "vps_server_query")
        return dict(state=st.value, status=status.value, iters=it.value, rel_res=rel.value,
                    queue_s=qs.value, latency_s=lat.value)

    def wait(self, rid=0, timeout_s=600.0):
        rc = lib().vps_server_wait(self.s, int(rid), float(timeout_s))
        if rc != VPS_OK:
            raise VpsError(rc, "vps_server_wait")

    def stats(self):
        sub, done = ctypes.c_int64(), ctypes.c_int64()
        act, q = ctypes.c_int(), ctypes.c_int()
        lib().vps_server_stats(self.s, ctypes.byref(sub), ctypes.byref(done), ctypes.byref(act),
                               ctypes.byref(q))
        return dict(submitted=sub.value, done=done.value, active=act.value, queued=q.value)

    def batch_stats(self):
        """Cohort V-cycle steps, batched launches, and the largest number of
        requests in one batched launch / one step."""
        t, bl = ctypes.c_int64(), ctypes.c_int64()
        ml, mt = ctypes.c_int(), ctypes.c_int()
        _check(lib().vps_server_batch_stats(self.s, ctypes.byref(t), ctypes.byref(bl),
                                            ctypes.byref(ml), ctypes.byref(mt)), None)
        return dict(ticks=t.value, batched_launches=bl.value, max_requests_per_launch=ml.value,
                    max_requests_per_tick=mt.value)

    def host_times(self):
        """Host seconds of the engine's admission, cohort steps and polling,
        and of the helper threads' hierarchy building and result copies."""
        t = (ctypes.c_double * 5)()
        _check(lib().vps_server_host_times(self.s, t), None)
        return dict(admit_s=t[0], tick_s=t[1], poll_s=t[2], create_s=t[3], copy_s=t[4])

    def last_error(self):
        return lib().vps_server_last_error(self.s).decode()

    def close(self):
        if getattr(self, "s", None):
            lib().vps_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
