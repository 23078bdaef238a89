"""Thin ctypes binding of the CUDA registration library (``include/reg.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels. Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they must
be float64 and contiguous. There is no CPU fallback: if the library cannot be
built or loaded, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

REG_OK, REG_EINVAL, REG_ENOMEM, REG_ECUDA, REG_ENOTREADY = 0, 1, 2, 3, 4
REG_ENONFINITE, REG_ECFL, REG_ELINESEARCH, REG_EMAXIT, REG_ETIMEOUT = 5, 6, 7, 8, 9
REG_H1, REG_H2 = 1, 2
REG_FP64, REG_MIXED = 0, 1
REG_QUAD_TRAPEZOID, REG_QUAD_DISCRETE = 0, 1
REG_HESS_GN, REG_HESS_NEWTON = 0, 1
REG_METHOD_KRYLOV, REG_METHOD_PICARD = 0, 1
REG_STOP_GRAD_REL, REG_STOP_C1C5 = 0, 1

_STATUS = {0: "REG_OK", 1: "REG_EINVAL", 2: "REG_ENOMEM", 3: "REG_ECUDA", 4: "REG_ENOTREADY",
           5: "REG_ENONFINITE", 6: "REG_ECFL", 7: "REG_ELINESEARCH", 8: "REG_EMAXIT", 9: "REG_ETIMEOUT"}


class SolveOpts(ctypes.Structure):
    _fields_ = [
        ("grad_rtol", ctypes.c_double),
        ("max_outer", ctypes.c_int),
        ("armijo_c1", ctypes.c_double),
        ("backtrack", ctypes.c_double),
        ("max_backtracks", ctypes.c_int),
        ("pcg_maxit", ctypes.c_long),
        ("cfl_max", ctypes.c_double),
        ("detF_substeps", ctypes.c_int),
        ("method", ctypes.c_int),
        ("step_memory", ctypes.c_int),
        ("stop_rule", ctypes.c_int),
        ("tau_J", ctypes.c_double),
        ("detF_refine", ctypes.c_int),
    ]

    @classmethod
    def make(cls, L, opts):
        """Library defaults overridden by the keyword options (unknown names raise)."""
        o = cls()
        L.reg_solve_opts_default(ctypes.byref(o))
        names = {f for f, _ in cls._fields_}
        for k, val in opts.items():
            if k not in names:
                raise TypeError(f"unknown solve option {k!r}")
            setattr(o, k, val)
        return o


class SolveReport(ctypes.Structure):
    _fields_ = [
        ("outer", ctypes.c_int),
        ("pcg_iters", ctypes.c_long),
        ("matvecs", ctypes.c_long),
        ("n_pde", ctypes.c_long),
        ("ls_trials", ctypes.c_int),
        ("cfl_halvings", ctypes.c_int),
        ("status", ctypes.c_int),
        ("J0", ctypes.c_double),
        ("J", ctypes.c_double),
        ("g0_inf", ctypes.c_double),
        ("g_inf", ctypes.c_double),
        ("dist_rel", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("detF", ctypes.c_double * 4),
        ("seconds", ctypes.c_double),
        ("stop_flags", ctypes.c_int),
        ("alpha_mem", ctypes.c_double),
        ("J_prev", ctypes.c_double),
        ("dv_inf", ctypes.c_double),
        ("v_inf", ctypes.c_double),
        ("device_loops", ctypes.c_int),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            val = getattr(self, name)
            out[name] = list(val) if name == "detF" else val
        return out


class ProblemC(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
        ("n_t", ctypes.c_int),
        ("n_c", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("reg_type", ctypes.c_int),
        ("stokes", ctypes.c_int),
        ("m_T", ctypes.c_void_p),
        ("m_R", ctypes.c_void_p),
        ("v", ctypes.c_void_p),
    ]


class ContOpts(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in
                ("beta0", "beta_min", "eps_F", "eps_theta", "beta_rtol", "dist_rtol", "cfl_target")] + [
        ("detF_substeps", ctypes.c_int), ("max_solves", ctypes.c_int)]


CONT_TRACE = 64


class ContReport(ctypes.Structure):
    _fields_ = [
        ("found", ctypes.c_int),
        ("stop", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("beta_breach", ctypes.c_double),
        ("solves", ctypes.c_int),
        ("n_t", ctypes.c_int),
        ("outer", ctypes.c_long),
        ("pcg_iters", ctypes.c_long),
        ("matvecs", ctypes.c_long),
        ("detF_min", ctypes.c_double),
        ("angle_min", ctypes.c_double),
        ("dist_rel", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("n_trace", ctypes.c_int),
        ("trace_beta", ctypes.c_double * CONT_TRACE),
        ("trace_detF", ctypes.c_double * CONT_TRACE),
        ("trace_angle", ctypes.c_double * CONT_TRACE),
        ("trace_dist", ctypes.c_double * CONT_TRACE),
        ("trace_ok", ctypes.c_int * CONT_TRACE),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            val = getattr(self, name)
            out[name] = list(val)[:self.n_trace] if name.startswith("trace_") else val
        return out


class RegError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_SIGNATURES = {
    "reg_create": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int,
                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp],
    "reg_destroy": [_vp],
    "reg_set_quadrature": [_vp, ctypes.c_int],
    "reg_set_hessian": [_vp, ctypes.c_int],
    "reg_set_images": [_vp, _vp, _vp],
    "reg_objective": [_vp, _vp, _vp, _vp],
    "reg_gradient": [_vp, _vp, _vp, _vp],
    "reg_linearize": [_vp, _vp],
    "reg_hessvec": [_vp, _vp, _vp],
    "reg_precond": [_vp, _vp, _vp],
    "reg_regularization": [_vp, _vp, _vp],
    "reg_transport": [_vp, _vp, _vp, _vp],
    "reg_transport_adjoint": [_vp, _vp, _vp, _vp, _vp, _vp],
    "reg_detF": [_vp, _vp, ctypes.c_int, _vp, _vp],
    "reg_detF_refined": [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp],
    "reg_cfl": [_vp, _vp, _vp],
    "reg_grid_angle": [_vp, _vp, ctypes.c_int, _vp, _vp],
    "reg_displacement": [_vp, _vp, _vp],
    "reg_smooth": [_vp, ctypes.c_double, _vp, _vp],
    "reg_lanczos": [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.POINTER(ctypes.c_int), _vp],
    "reg_set_beta": [_vp, ctypes.c_double],
    "reg_selftest_copy_timeout": [ctypes.POINTER(ctypes.c_int)],
    "reg_set_time_steps": [_vp, ctypes.c_int],
    "reg_continuation": [_vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(ContOpts), ctypes.POINTER(ContReport)],
    "reg_solve": [_vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport)],
    "reg_precond_noalloc": [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                            _vp, _vp, _vp],
    "reg_solve_batched": [ctypes.POINTER(ProblemC), ctypes.c_int, ctypes.c_int, ctypes.POINTER(SolveOpts),
                          ctypes.POINTER(SolveReport), ctypes.c_int],
    "reg_solve_lockstep": [ctypes.POINTER(ProblemC), ctypes.c_int, ctypes.c_int, ctypes.POINTER(SolveOpts),
                           ctypes.POINTER(SolveReport), ctypes.c_int],
    "reg_profile_begin": [_vp, ctypes.c_uint],
    "reg_profile_end": [_vp, _vp, _vp, _vp],
    "reg_profile_flops": [_vp, _vp],
    "reg_fp64_peak": [ctypes.POINTER(ctypes.c_double)],
}

EXPORTED = tuple(_SIGNATURES) + ("reg_last_error", "reg_solve_opts_default", "reg_launch_count",
                                  "reg_cont_opts_default")
KIND_NAMES = ("rows_r2c", "rows_c2r", "cols", "mult", "stage", "force", "other")


def selftest_copy_timeout():
    """Number of timeouts counted by the bounded-wait self-test (1 expected)."""
    L = load()
    n = ctypes.c_int(0)
    st = L.reg_selftest_copy_timeout(ctypes.byref(n))
    if st != REG_OK:
        raise RegError(st, L.reg_last_error(None).decode())
    return n.value


def launch_count():
    return int(load().reg_launch_count())


def fp64_peak_gflops():
    """Measured double-precision FMA throughput of the current device (GFLOP/s)."""
    L = load()
    g = ctypes.c_double(0.0)
    st = L.reg_fp64_peak(ctypes.byref(g))
    if st != REG_OK:
        raise RegError(st, L.reg_last_error(None).decode())
    return g.value


def precond_noalloc(n, n_c, beta, reg, r, z, stream=None):
    """z = P^{-1} r like Registration.precond, without a context and without
    allocating (fixed device scratch; r and z must be CUDA tensors). Returns
    once the work is enqueued on `stream`."""
    L = load()
    n = tuple(int(k) for k in n)
    arr = (ctypes.c_int64 * len(n))(*n)
    count = int(n_c) * len(n) * int(np.prod(n))
    a, ka = _addr(r, count)
    b, kb = _addr(z, count)
    st = L.reg_precond_noalloc(len(n), arr, int(n_c), float(beta), int(reg), a, b, stream)
    if st != REG_OK:
        raise RegError(st, L.reg_last_error(None).decode())


def _problem_array(problems):
    arr = (ProblemC * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        n = tuple(int(k) for k in p["n"])
        N = int(np.prod(n))
        a, ka = _addr(p["mT"], N)
        b, kb = _addr(p["mR"], N)
        c, kc = _addr(p["v"], int(p.get("n_c", 1)) * len(n) * N)
        keep += [ka, kb, kc]
        arr[i] = ProblemC(len(n), (ctypes.c_int64 * 3)(*(list(n) + [1] * (3 - len(n)))), int(p["n_t"]),
                          int(p.get("n_c", 1)), float(p["beta"]), int(p.get("reg", REG_H1)),
                          int(bool(p.get("stokes", False))), a, b, c)
    return arr, keep


def solve_batched(problems, precision=REG_MIXED, workers=8, **opts):
    """Solve independent problems concurrently (reg_solve_batched).

    problems: list of dicts with keys n, n_t, n_c, beta, reg, stokes, mT, mR, v
    (arrays as accepted by Registration; v is updated in place). Returns the
    list of report dicts in the order of `problems`."""
    L = load()
    arr, keep = _problem_array(problems)
    o = SolveOpts.make(L, opts)
    reps = (SolveReport * len(problems))()
    st = L.reg_solve_batched(arr, len(problems), int(precision), ctypes.byref(o), reps, int(workers))
    if st not in (REG_OK, REG_EMAXIT):
        raise RegError(st, L.reg_last_error(None).decode())
    return [r.as_dict() for r in reps]


def solve_lockstep(problems, precision=REG_MIXED, max_stack=0, **opts):
    """Lockstep batched solve (reg_solve_lockstep): problems of one shape are
    stacked and iterated together. Same arguments and result as solve_batched;
    a failed stack raises, with the reports of the others lost."""
    L = load()
    arr, keep = _problem_array(problems)
    o = SolveOpts.make(L, opts)
    reps = (SolveReport * len(problems))()
    st = L.reg_solve_lockstep(arr, len(problems), int(precision), ctypes.byref(o), reps, int(max_stack))
    if st not in (REG_OK, REG_EMAXIT):
        raise RegError(st, L.reg_last_error(None).decode())
    return [r.as_dict() for r in reps]


def library_path():
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load (building first if needed) the CUDA library; raise if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"registration CUDA library missing at {path}")
            L = ctypes.CDLL(path)
            for name, args in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.reg_last_error.argtypes = [_vp]
            L.reg_last_error.restype = ctypes.c_char_p
            L.reg_solve_opts_default.argtypes = [ctypes.POINTER(SolveOpts)]
            L.reg_solve_opts_default.restype = None
            L.reg_cont_opts_default.argtypes = [ctypes.POINTER(ContOpts)]
            L.reg_cont_opts_default.restype = None
            L.reg_launch_count.argtypes = []
            L.reg_launch_count.restype = ctypes.c_long
            _lib = L
    return _lib


def _addr(a, count=None):
    """(address, keepalive) of a contiguous float64 torch tensor or numpy array.

    count: the number of float64 values the library will read or write
    through this pointer; a different element count raises ValueError before
    any library call (the C side cannot know the size of the array). A CUDA
    tensor must live on the current device, where the kernels run."""
    if a is None:
        return None, None
    n = None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise TypeError("tensors passed to the registration library must be contiguous float64")
            if a.is_cuda and a.device.index != torch.cuda.current_device():
                raise ValueError(f"tensor on {a.device} but cuda:{torch.cuda.current_device()} is current")
            n, out = a.numel(), (a.data_ptr(), a)
    except ImportError:
        pass
    if n is None:
        if not isinstance(a, np.ndarray):
            raise TypeError(f"unsupported array type {type(a)}")
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("arrays passed to the registration library must be C-contiguous float64")
        n, out = a.size, (a.ctypes.data, a)
    if count is not None and n != int(count):
        raise ValueError(f"array of {n} float64 values where {int(count)} are expected")
    return out


class Registration:
    """One library context: grid, time discretisation and regulariser fixed at creation."""

    def __init__(self, n, n_t, n_c=1, beta=1e-2, reg=REG_H1, stokes=False, precision=REG_FP64, ckpt_every=0,
                 stream=None, quadrature=REG_QUAD_TRAPEZOID, hessian=REG_HESS_GN):
        self.L = load()
        self.n = tuple(int(k) for k in n)
        self.d = len(self.n)
        self.n_t, self.n_c = int(n_t), int(n_c)
        self.ckpt_every = int(ckpt_every)
        ctx = _vp()
        arr = (ctypes.c_int64 * self.d)(*self.n)
        st = self.L.reg_create(ctypes.byref(ctx), self.d, arr, self.n_t, self.n_c, float(beta), int(reg),
                               int(bool(stokes)), int(precision), int(ckpt_every), stream)
        if st != REG_OK:
            raise RegError(st, self.L.reg_last_error(None).decode())
        self.ctx = ctx
        if quadrature != REG_QUAD_TRAPEZOID:
            self._check(self.L.reg_set_quadrature(self.ctx, int(quadrature)))
        if hessian != REG_HESS_GN:
            self.set_hessian(hessian)

    @property
    def N(self):
        return int(np.prod(self.n))

    @property
    def ncdN(self):
        """values of a coefficient vector: n_c * d * N"""
        return self.n_c * self.d * self.N

    def coef_shape(self):
        return (self.n_c, self.d) + self.n

    def close(self):
        if getattr(self, "ctx", None):
            self.L.reg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != REG_OK:
            raise RegError(st, self.L.reg_last_error(self.ctx).decode())

    # each method passes raw pointers through; outputs are caller-allocated
    def set_hessian(self, kind):
        """REG_HESS_GN (default) or REG_HESS_NEWTON for hessvec and solve."""
        self._check(self.L.reg_set_hessian(self.ctx, int(kind)))

    def set_images(self, mT, mR):
        a, ka = _addr(mT, self.N)
        b, kb = _addr(mR, self.N)
        self._check(self.L.reg_set_images(self.ctx, a, b))

    def objective(self, v):
        a, ka = _addr(v, self.ncdN)
        J = ctypes.c_double()
        parts = (ctypes.c_double * 2)()
        self._check(self.L.reg_objective(self.ctx, a, ctypes.byref(J), parts))
        return J.value, (parts[0], parts[1])

    def gradient(self, v, g):
        a, ka = _addr(v, self.ncdN)
        b, kb = _addr(g, self.ncdN)
        J = ctypes.c_double()
        self._check(self.L.reg_gradient(self.ctx, a, b, ctypes.byref(J)))
        return J.value

    def linearize(self, v):
        a, ka = _addr(v, self.ncdN)
        self._check(self.L.reg_linearize(self.ctx, a))

    def hessvec(self, vt, out):
        a, ka = _addr(vt, self.ncdN)
        b, kb = _addr(out, self.ncdN)
        self._check(self.L.reg_hessvec(self.ctx, a, b))

    def precond(self, r, z):
        a, ka = _addr(r, self.ncdN)
        b, kb = _addr(z, self.ncdN)
        self._check(self.L.reg_precond(self.ctx, a, b))

    def regularization(self, v, out):
        a, ka = _addr(v, self.ncdN)
        b, kb = _addr(out, self.ncdN)
        self._check(self.L.reg_regularization(self.ctx, a, b))

    def transport(self, v, m0, m1):
        a, ka = _addr(v, self.ncdN)
        b, kb = _addr(m0, self.N)
        c, kc = _addr(m1, self.N)
        self._check(self.L.reg_transport(self.ctx, a, b, c))

    def transport_adjoint(self, v, m0, G, grad_v=None, grad_m0=None):
        a, ka = _addr(v, self.ncdN)
        b, kb = _addr(m0, self.N)
        c, kc = _addr(G, self.N)
        d, kd = _addr(grad_v, self.ncdN)
        e, ke = _addr(grad_m0, self.N)
        self._check(self.L.reg_transport_adjoint(self.ctx, a, b, c, d, e))

    def detF(self, v, substeps=1, out=None):
        a, ka = _addr(v, self.ncdN)
        b, kb = _addr(out, self.N)
        st = (ctypes.c_double * 4)()
        self._check(self.L.reg_detF(self.ctx, a, int(substeps), st, b))
        return tuple(st)

    def detF_refined(self, v, substeps=1, refine=2, out=None):
        """det F_1 statistics (min, max, mean, std) on a grid refined `refine`
        times per axis; out (optional): the fine-grid field (N * refine^d values)."""
        a, ka = _addr(v, self.ncdN)
        b, kb = _addr(out, self.N * int(refine) ** self.d)
        st = (ctypes.c_double * 4)()
        self._check(self.L.reg_detF_refined(self.ctx, a, int(substeps), int(refine), st, b))
        return tuple(st)

    def cfl(self, v):
        a, ka = _addr(v, self.ncdN)
        c = ctypes.c_double()
        self._check(self.L.reg_cfl(self.ctx, a, ctypes.byref(c)))
        return c.value

    def grid_angle(self, v, substeps=1, out=None):
        """Smallest acute angle between deformed grid edges: (min, max, mean, std)."""
        a, ka = _addr(v, self.ncdN)
        b, kb = _addr(out, self.N)
        st = (ctypes.c_double * 4)()
        self._check(self.L.reg_grid_angle(self.ctx, a, int(substeps), st, b))
        return tuple(st)

    def displacement(self, v, u):
        """u_1 of the deformation map into u (d fields)."""
        a, ka = _addr(v, self.ncdN)
        b, kb = _addr(u, self.d * self.N)
        self._check(self.L.reg_displacement(self.ctx, a, b))

    def smooth(self, sigma, m, out):
        """Gaussian presmoothing of m (N values) into out."""
        a, ka = _addr(m, self.N)
        b, kb = _addr(out, self.N)
        self._check(self.L.reg_smooth(self.ctx, float(sigma), a, b))

    def lanczos(self, q0, k, precond=False):
        """(alpha, beta, ritz) of k Lanczos steps on H (or P^{-1} H) at the linearisation point."""
        a, ka = _addr(q0, self.ncdN)
        al = (ctypes.c_double * k)()
        be = (ctypes.c_double * k)()
        rz = (ctypes.c_double * k)()
        m = ctypes.c_int(0)
        self._check(self.L.reg_lanczos(self.ctx, a, int(k), int(bool(precond)), al, be, ctypes.byref(m), rz))
        m = m.value
        return np.array(al[:m]), np.array(be[:m]), np.array(rz[:m])

    def set_beta(self, beta):
        self._check(self.L.reg_set_beta(self.ctx, float(beta)))

    def set_time_steps(self, n_t):
        self._check(self.L.reg_set_time_steps(self.ctx, int(n_t)))
        self.n_t = int(n_t)

    def continuation(self, v, solve_opts=None, **cont):
        """Beta continuation in place on v; returns the report dict."""
        a, ka = _addr(v, self.ncdN)
        so = SolveOpts.make(self.L, solve_opts or {})
        co = ContOpts()
        self.L.reg_cont_opts_default(ctypes.byref(co))
        names = {f for f, _ in ContOpts._fields_}
        for k, val in cont.items():
            if k not in names:
                raise TypeError(f"unknown continuation option {k!r}")
            setattr(co, k, val)
        rep = ContReport()
        self._check(self.L.reg_continuation(self.ctx, a, ctypes.byref(so), ctypes.byref(co), ctypes.byref(rep)))
        out = rep.as_dict()
        self.n_t = out["n_t"]
        return out

    def profile_begin(self, mask=(1 << 7) - 1):
        self._check(self.L.reg_profile_begin(self.ctx, int(mask)))

    def profile_end(self):
        ms = (ctypes.c_double * 7)()
        by = (ctypes.c_double * 7)()
        cnt = (ctypes.c_long * 7)()
        self._check(self.L.reg_profile_end(self.ctx, ms, by, cnt))
        fl = (ctypes.c_double * 7)()
        self._check(self.L.reg_profile_flops(self.ctx, fl))
        return {KIND_NAMES[k]: dict(ms=ms[k], bytes=by[k], launches=cnt[k], flops=fl[k]) for k in range(7)}

    def solve(self, v, **opts):
        """Solve in place on v; returns the report dict (raises on a failed solve)."""
        a, ka = _addr(v, self.ncdN)
        o = SolveOpts.make(self.L, opts)
        rep = SolveReport()
        st = self.L.reg_solve(self.ctx, a, ctypes.byref(o), ctypes.byref(rep))
        out = rep.as_dict()
        out["status"] = st
        if st not in (REG_OK, REG_EMAXIT):
            self._check(st)
        return out
