"""Thin ctypes binding of ``include/mgrit.h``: argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays may
be numpy arrays (host) or torch tensors (host or CUDA); the library detects
device pointers itself.  PyTorch supplies the CUDA stream and, when a CUDA
device is present, the device memory of the library's state: importing this
module routes the library's allocations through PyTorch's caching allocator
(``use_default_allocator`` switches back to the library's cudaMallocAsync).

There is no fallback: if ``libmgrit_gb300.so`` is missing the import fails
and says how to build it.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgrit_gb300.so")

MGRIT_OK, MGRIT_PENDING = 0, 1
STATUS = {0: "OK", 1: "PENDING", -1: "ERR_INVALID", -2: "ERR_UNSTABLE", -3: "ERR_PSI_ILLCOND",
          -4: "ERR_NOT_CONVERGED", -5: "ERR_DIVERGED", -6: "ERR_OVER_BUDGET", -7: "ERR_OOM",
          -8: "ERR_TIMEOUT", -9: "ERR_CUDA", -10: "ERR_UNSUPPORTED", -11: "ERR_UNKNOWN_TICKET"}
ERK, SDIRK = 0, 1
BC_PERIODIC, BC_INFLOW = 0, 1
PREC_FP64, PREC_MIXED, PREC_MIXED_DF = 0, 1, 2
PSI_AUTO, PSI_HALFWIDTH, PSI_THRESHOLD, PSI_USER, PSI_IDEAL, PSI_REDISC = 0, 1, 2, 3, 4, 5
OUT_FINAL, OUT_CPOINTS, OUT_FULL = 0, 1, 2
CYCLE_V, CYCLE_F = 0, 1
RELAX_FCF, RELAX_F = 0, 1
INIT_ZERO, INIT_RANDOM = 0, 1
MAX_INFLIGHT = 64
MAX_HISTORY = 128
MAX_LEVELS = 8
FLAG_TIME_KERNELS = 1
FLAG_NO_AUTOTUNE = 2
FLAG_HOST_LOOP = 4
FLAG_NO_DIVERGENCE_STOP = 8
KERNEL_KINDS = ["fcf", "fcf_coarse", "march", "correct", "norm", "add", "propagate", "other"]
K_KINDS = len(KERNEL_KINDS)

EXPORTED = ["mgrit_opts_default", "mgrit_set_allocator", "mgrit_phi_taps", "mgrit_phi_boundary", "mgrit_psi_plan",
            "mgrit_setup", "mgrit_solve", "mgrit_solve_async", "mgrit_solve_wait", "mgrit_solve_from", "mgrit_relax", "mgrit_sequential", "mgrit_propagate",
            "mgrit_psi_info",
            "mgrit_device_bytes", "mgrit_destroy", "mgrit_server_create", "mgrit_submit",
            "mgrit_poll", "mgrit_server_stats", "mgrit_server_destroy", "mgrit_fcf_residual_static", "mgrit_last_error",
            "mgrit_abi_version", "mgrit_check_conversions"]


class MgritProblem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nt", C.c_int32), ("family", C.c_int32), ("rk_order", C.c_int32),
                ("upwind_order", C.c_int32), ("boundary", C.c_int32), ("cfl", C.c_double),
                ("alpha", C.c_double), ("xmin", C.c_double), ("xmax", C.c_double)]


class MgritOpts(C.Structure):
    _fields_ = [("m", C.c_int32), ("levels", C.c_int32), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("psi_rule", C.c_int32), ("psi_halfwidth", C.c_int32), ("output", C.c_int32),
                ("min_coarse", C.c_int32), ("flags", C.c_int32), ("cycle", C.c_int32), ("relax", C.c_int32),
                ("init_guess", C.c_int32), ("tol", C.c_double), ("psi_eta", C.c_double),
                ("psi_rho", C.c_double), ("seed", C.c_uint64), ("psi_user_nnz", C.POINTER(C.c_int32)),
                ("psi_user_offsets", C.POINTER(C.c_int32)), ("psi_user_coeffs", C.POINTER(C.c_double))]


class MgritResult(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("n_levels", C.c_int32), ("converged", C.c_int32),
                ("n_history", C.c_int32), ("rel_residual", C.c_double), ("r0_norm", C.c_double),
                ("setup_s", C.c_double), ("solve_s", C.c_double), ("dof_per_s", C.c_double),
                ("op_complexity", C.c_double), ("history", C.c_double * MAX_HISTORY),
                ("launches", C.c_int32), ("fine_tile", C.c_int32), ("fine_threads", C.c_int32),
                ("graph", C.c_int32), ("fine_collapsed", C.c_int32), ("fine_fourier", C.c_int32),
                ("kernel_count", C.c_int32 * K_KINDS),
                ("kernel_ms", C.c_double * K_KINDS), ("dx", C.c_double), ("dt", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("history", "kernel_count", "kernel_ms")}
        d["history"] = list(self.history[: self.n_history])
        d["kernel_count"] = {KERNEL_KINDS[i]: self.kernel_count[i] for i in range(K_KINDS)}
        d["kernel_ms"] = {KERNEL_KINDS[i]: self.kernel_ms[i] for i in range(K_KINDS)}
        return d


class MgritServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("cycles", C.c_uint64), ("admit_s", C.c_double), ("plan_s", C.c_double), ("tune_s", C.c_double),
                ("cycle_s", C.c_double),
                ("retire_s", C.c_double), ("mean_active", C.c_double), ("peak_resident_bytes", C.c_double),
                ("gpu_fcf_ms", C.c_double), ("gpu_norm_ms", C.c_double), ("gpu_coarse_ms", C.c_double),
                ("gpu_gap_ms", C.c_double), ("first_cycle_s", C.c_double), ("fft_coarse_solves", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MgritServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("max_active", C.c_int32), ("reserved", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_1910_03726_gb300.build` "
                          "(needs nvcc); there is no CPU fallback")
    return C.CDLL(LIB_PATH)


_lib = _load()
_vp, _i32, _f64 = C.c_void_p, C.c_int32, C.c_double
_P = C.POINTER


def _sig(name, res, *args):
    f = getattr(_lib, name, None)
    if f is not None:
        f.restype = res
        f.argtypes = list(args)
    return f


_sig("mgrit_opts_default", None, _P(MgritOpts))
ALLOC_FN = C.CFUNCTYPE(_vp, C.c_size_t, _vp, _vp)
FREE_FN = C.CFUNCTYPE(None, _vp, _vp, _vp)
_sig("mgrit_set_allocator", None, ALLOC_FN, FREE_FN, _vp)
_sig("mgrit_phi_taps", _i32, _P(MgritProblem), _i32, _P(_i32), _P(_i32), _P(_f64))
_sig("mgrit_phi_boundary", _i32, _P(MgritProblem), _i32, _i32, _P(_i32), _P(_f64))
_sig("mgrit_psi_plan", _i32, _P(MgritProblem), _P(MgritOpts), _i32, _P(_i32), _P(_i32), _P(_f64), _P(_f64))
_sig("mgrit_setup", _i32, _P(MgritProblem), _P(MgritOpts), _vp, _P(_vp))
_sig("mgrit_solve", _i32, _vp, _vp, _vp, _P(MgritResult))
_sig("mgrit_solve_async", _i32, _vp, _vp, _vp)
_sig("mgrit_solve_wait", _i32, _vp, _P(MgritResult))
_sig("mgrit_solve_from", _i32, _vp, _vp, _f64, _vp, _P(MgritResult))
_sig("mgrit_relax", _i32, _vp, _i32, _P(_f64))
_sig("mgrit_sequential", _i32, _vp, _vp, _vp, _P(_f64))
_sig("mgrit_propagate", _i32, _vp, _i32, _i32, _i32, _vp, _vp)
_sig("mgrit_psi_info", _i32, _vp, _i32, _i32, _P(_i32), _P(_i32), _P(_f64))
_sig("mgrit_device_bytes", C.c_size_t, _vp)
_sig("mgrit_destroy", None, _vp)
_sig("mgrit_server_create", _i32, _P(MgritServerOpts), _vp, _P(_vp))
_sig("mgrit_submit", _i32, _vp, _P(MgritProblem), _P(MgritOpts), _vp, _P(C.c_uint64))
_sig("mgrit_poll", _i32, _vp, C.c_uint64, _vp, _P(MgritResult))
_sig("mgrit_server_stats", _i32, _vp, _P(MgritServerStats))
_sig("mgrit_server_destroy", None, _vp)
_sig("mgrit_fcf_residual_static", _i32, _vp, _vp, _vp, _vp, _i32, _i32, _i32, _i32, _P(_i32), _P(_f64), _i32, _vp)
_sig("mgrit_last_error", C.c_char_p)
_sig("mgrit_abi_version", _i32)
_sig("mgrit_check_conversions", _i32, C.c_uint64, C.c_uint64, _P(C.c_uint64))


class MgritError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status, allow=(MGRIT_OK,)):
    if status not in allow:
        raise MgritError(status, mgrit_last_error())
    return status


def _ptr(x):
    """Raw pointer of a numpy array or torch tensor (contiguous float64)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise TypeError("arrays must be C-contiguous float64")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return x.data_ptr()
    raise TypeError(type(x))


# ------------------------------------------------------------------ helpers

def problem(nx, nt, family="ERK", rk_order=1, upwind_order=None, cfl=0.85, boundary=BC_PERIODIC, alpha=1.0,
            xmin=-1.0, xmax=1.0):
    fam = ERK if family in ("ERK", ERK) else SDIRK
    bc = BC_INFLOW if boundary in ("inflow", BC_INFLOW) else BC_PERIODIC
    return MgritProblem(nx, nt, fam, rk_order, upwind_order or rk_order, bc, float(cfl), float(alpha),
                        float(xmin), float(xmax))


def mgrit_opts_default(**overrides):
    o = MgritOpts()
    _lib.mgrit_opts_default(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def user_psi(opts, ops):
    """Attach caller-supplied coarse operators (list of (offsets, coeffs)) to
    opts; returns the ctypes arrays, which must stay alive with opts."""
    nnz = (C.c_int32 * len(ops))(*[len(o[0]) for o in ops])
    offs = [int(i) for o in ops for i in o[0]]
    cfs = [float(c) for o in ops for c in o[1]]
    off_arr = (C.c_int32 * max(1, len(offs)))(*offs)
    cf_arr = (C.c_double * max(1, len(cfs)))(*cfs)
    opts.psi_rule = PSI_USER
    opts.psi_user_nnz = C.cast(nnz, _P(C.c_int32))
    opts.psi_user_offsets = C.cast(off_arr, _P(C.c_int32))
    opts.psi_user_coeffs = C.cast(cf_arr, _P(C.c_double))
    return (nnz, off_arr, cf_arr)


# ----------------------------------------------------------- entry points

def mgrit_last_error():
    s = _lib.mgrit_last_error()
    return s.decode() if s else ""


def mgrit_abi_version():
    return int(_lib.mgrit_abi_version())


def mgrit_check_conversions(n, seed=0):
    """Patterns (of 2n) on which the kernels' integer-pipe binary32 -> binary64
    conversion differs from the GPU's conversion instruction (0 expected)."""
    bad = C.c_uint64()
    _check(_lib.mgrit_check_conversions(int(n), int(seed), C.byref(bad)))
    return int(bad.value)


def mgrit_phi_taps(prob, cap=1024):
    n = C.c_int32()
    offs = (C.c_int32 * cap)()
    cfs = (C.c_double * cap)()
    _check(_lib.mgrit_phi_taps(C.byref(prob), cap, C.byref(n), offs, cfs))
    return list(offs[: n.value]), list(cfs[: n.value])


def mgrit_phi_boundary(prob, m=1, cap=1 << 18):
    """Boundary rows of an inflow/outflow problem's Phi^m: (left block
    (nl, cl), right block (nr, cr)) as numpy arrays."""
    dims = (C.c_int32 * 4)()
    w = (C.c_double * cap)()
    _check(_lib.mgrit_phi_boundary(C.byref(prob), m, cap, dims, w))
    nl, cl, nr, cr = (int(v) for v in dims)
    a = np.array(w[: nl * cl + nr * cr])
    return a[: nl * cl].reshape(nl, cl), a[nl * cl:].reshape(nr, cr)


def mgrit_psi_plan(prob, opts, cap=1 << 16):
    L = opts.levels - 1
    nnz = (C.c_int32 * L)()
    offs = (C.c_int32 * cap)()
    cfs = (C.c_double * cap)()
    diag = (C.c_double * (3 * L))()
    st = _lib.mgrit_psi_plan(C.byref(prob), C.byref(opts), cap, nnz, offs, cfs, diag)
    _check(st)
    out, pos = [], 0
    for l in range(L):
        n = nnz[l]
        out.append((list(offs[pos:pos + n]), list(cfs[pos:pos + n])))
        pos += n
    return out, [tuple(diag[3 * l:3 * l + 3]) for l in range(L)]


def _stream_ptr(stream):
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # noqa: BLE001
        pass
    return None


def mgrit_setup(prob, opts, stream=None):
    h = C.c_void_p()
    _check(_lib.mgrit_setup(C.byref(prob), C.byref(opts), _stream_ptr(stream), C.byref(h)))
    return h


def mgrit_solve(h, u0, out=None, allow_not_converged=False):
    r = MgritResult()
    allow = (MGRIT_OK, -4) if allow_not_converged else (MGRIT_OK,)
    st = _check(_lib.mgrit_solve(h, _ptr(u0), _ptr(out), C.byref(r)), allow)
    return r, st


def mgrit_solve_async(h, u0, out=None):
    """Enqueue a solve (out: device tensor or None); finish it with mgrit_solve_wait."""
    _check(_lib.mgrit_solve_async(h, _ptr(u0), _ptr(out)))


def mgrit_solve_wait(h, allow_not_converged=False):
    """Wait for the oldest queued solve of h; returns (result, status)."""
    r = MgritResult()
    allow = (MGRIT_OK, -4) if allow_not_converged else (MGRIT_OK,)
    st = _check(_lib.mgrit_solve_wait(h, C.byref(r)), allow)
    return r, st


def mgrit_solve_from(h, c_init, r0_norm=0.0, out=None, allow_not_converged=False):
    r = MgritResult()
    allow = (MGRIT_OK, -4) if allow_not_converged else (MGRIT_OK,)
    st = _check(_lib.mgrit_solve_from(h, _ptr(c_init), C.c_double(r0_norm), _ptr(out), C.byref(r)), allow)
    return r, st


def mgrit_relax(h, sweeps):
    """Level-1 FCF sweeps on the last solve's C-points; returns the relative residual."""
    rel = C.c_double()
    _check(_lib.mgrit_relax(h, int(sweeps), C.byref(rel)))
    return rel.value


def mgrit_sequential(h, u0, out=None):
    t = C.c_double()
    _check(_lib.mgrit_sequential(h, _ptr(u0), _ptr(out), C.byref(t)))
    return t.value


def mgrit_propagate(h, level, k, count, inp, out):
    _check(_lib.mgrit_propagate(h, level, k, count, _ptr(inp), _ptr(out)))


def mgrit_psi_info(h, level, cap=4096):
    n = C.c_int32()
    offs = (C.c_int32 * cap)()
    cfs = (C.c_double * cap)()
    _check(_lib.mgrit_psi_info(h, level, cap, C.byref(n), offs, cfs))
    return list(offs[: n.value]), list(cfs[: n.value])


def mgrit_device_bytes(h):
    return int(_lib.mgrit_device_bytes(h))


def mgrit_destroy(h):
    _lib.mgrit_destroy(h)


def mgrit_server_create(budget_bytes, max_active=0, stream=None):
    so = MgritServerOpts(float(budget_bytes), int(max_active), 0)
    s = C.c_void_p()
    _check(_lib.mgrit_server_create(C.byref(so), _stream_ptr(stream), C.byref(s)))
    return s


def mgrit_submit(s, prob, opts, u0):
    t = C.c_uint64()
    _check(_lib.mgrit_submit(s, C.byref(prob), C.byref(opts), _ptr(u0), C.byref(t)))
    return t.value


def mgrit_poll(s, ticket, out=None):
    """Returns (status, result); status PENDING (1) while running."""
    r = MgritResult()
    st = _lib.mgrit_poll(s, C.c_uint64(ticket), _ptr(out), C.byref(r))
    return st, r


def mgrit_server_stats(s):
    st = MgritServerStats()
    _check(_lib.mgrit_server_stats(s, C.byref(st)))
    return st.as_dict()


def mgrit_server_destroy(s):
    _lib.mgrit_server_destroy(s)


def mgrit_fcf_residual_static(c_old, c_new, r, norm2, nx, m, n_intervals, offsets, coeffs, precision=PREC_FP64,
                              stream=None):
    """No-allocation FCF + residual (device tensors in/out, host taps)."""
    n = len(offsets)
    offs = (C.c_int32 * max(1, n))(*[int(o) for o in offsets])
    cfs = (C.c_double * max(1, n))(*[float(v) for v in coeffs])
    return _check(_lib.mgrit_fcf_residual_static(_ptr(c_old), _ptr(c_new), _ptr(r), _ptr(norm2), nx, m,
                                                 n_intervals, n, offs, cfs, precision, _stream_ptr(stream)))


# ------------------------------------------------------------ torch memory

_KEEP = []


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching
    allocator on the stream of the allocating call (the default once this
    module is imported on a machine with a CUDA device).  The device is the
    calling thread's current one, so a server's worker thread allocates on
    the server's device."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=torch.cuda.current_device(),
                                                          stream=int(stream or 0)))
        except Exception:  # noqa: BLE001  (the C side reports OOM)
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _KEEP[:] = [a, f]
    _lib.mgrit_set_allocator(a, f, None)


def use_default_allocator():
    _lib.mgrit_set_allocator(ALLOC_FN(), FREE_FN(), None)
    _KEEP[:] = []


def _torch_memory_by_default():
    try:
        import torch
        if torch.cuda.is_available():
            use_torch_allocator()
    except ImportError:
        pass


_torch_memory_by_default()
