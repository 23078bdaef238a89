"""ctypes front end of the FP64 CPU oracle (``oracle.c``).

Test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module. The product path (the CUDA
library under ``paper_1408_6299_gb300``) never does, and shares no code with it.

Every array is float64, row-major with the last grid axis fastest. Velocity
coefficient vectors have shape ``(n_c, d, *n)`` (the Chebyshev expansion in time
of Sec. 3.3.2); images have shape ``n``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Prob(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("n_t", ctypes.c_int),
        ("n_c", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("reg", ctypes.c_int),
        ("stokes", ctypes.c_int),
        ("dto", ctypes.c_int),
    ]


class Opts(ctypes.Structure):
    _fields_ = [
        ("grad_rtol", ctypes.c_double),
        ("max_outer", ctypes.c_int),
        ("armijo_c1", ctypes.c_double),
        ("backtrack", ctypes.c_double),
        ("max_backtracks", ctypes.c_int),
        ("pcg_maxit", ctypes.c_int),
        ("newton", ctypes.c_int),
        ("picard", ctypes.c_int),
        ("step_memory", ctypes.c_int),
        ("stop_rule", ctypes.c_int),
        ("tau_J", ctypes.c_double),
        ("cfl_max", ctypes.c_double),
    ]


class Report(ctypes.Structure):
    _fields_ = [
        ("outer", ctypes.c_int),
        ("pcg_iters", ctypes.c_int),
        ("matvecs", ctypes.c_int),
        ("n_pde", ctypes.c_int),
        ("ls_trials", ctypes.c_int),
        ("status", ctypes.c_int),
        ("J0", ctypes.c_double),
        ("J", ctypes.c_double),
        ("g0_inf", ctypes.c_double),
        ("g_inf", ctypes.c_double),
        ("g0_2", ctypes.c_double),
        ("g_2", ctypes.c_double),
        ("stop_flags", ctypes.c_int),
        ("cfl_halvings", ctypes.c_int),
        ("alpha_mem", ctypes.c_double),
        ("J_prev", ctypes.c_double),
        ("dv_inf", ctypes.c_double),
        ("v_inf", ctypes.c_double),
    ]


class ContOpts(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in
                ("beta0", "beta_min", "eps_F", "eps_theta", "beta_rtol", "dist_rtol", "cfl_target")] + [
        ("max_solves", ctypes.c_int)]


class ContReport(ctypes.Structure):
    _fields_ = [
        ("found", ctypes.c_int),
        ("stop", ctypes.c_int),
        ("solves", ctypes.c_int),
        ("n_t", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("beta_breach", ctypes.c_double),
        ("detF_min", ctypes.c_double),
        ("angle_min", ctypes.c_double),
        ("dist", ctypes.c_double),
        ("n_trace", ctypes.c_int),
        ("trace_beta", ctypes.c_double * 64),
        ("trace_detF", ctypes.c_double * 64),
        ("trace_angle", ctypes.c_double * 64),
        ("trace_dist", ctypes.c_double * 64),
        ("trace_ok", ctypes.c_int * 64),
    ]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER(Prob)
            dp = ctypes.POINTER(ctypes.c_double)
            for name, args in {
                "orc_fft": [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, ctypes.c_int],
                "orc_grad": [P, dp, dp],
                "orc_div": [P, dp, dp],
                "orc_apply_A": [P, dp, dp],
                "orc_leray": [P, dp, dp],
                "orc_precond": [P, dp, dp],
                "orc_reg_apply": [P, dp, dp],
                "orc_state": [P, dp, dp, dp, dp],
                "orc_adjoint": [P, dp, dp, dp, dp],
                "orc_objective": [P, dp, dp, dp, dp],
                "orc_gradient": [P, dp, dp, dp, dp, dp],
                "orc_hessvec": [P, dp, dp, dp, dp],
                "orc_hessvec_newton": [P, dp, dp, dp, dp, dp],
                "orc_detF": [P, dp, dp],
                "orc_defgrad": [P, dp, dp],
                "orc_grid_angle": [P, dp, dp],
                "orc_displacement": [P, dp, dp],
                "orc_smooth": [P, ctypes.c_double, dp, dp],
                "orc_lanczos": [P, dp, dp, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, dp,
                                ctypes.POINTER(ctypes.c_int)],
                "orc_solve": [P, ctypes.POINTER(Opts), dp, dp, dp, ctypes.POINTER(Report)],
                "orc_continuation": [P, ctypes.POINTER(Opts), ctypes.POINTER(ContOpts), dp, dp, dp,
                                     ctypes.POINTER(ContReport)],
            }.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.orc_cfl.argtypes = [P, dp]
            L.orc_cfl.restype = ctypes.c_double
            L.orc_cheb_eval.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            L.orc_cheb_eval.restype = None
            L.orc_cheb_gram.argtypes = [ctypes.c_int, dp]
            L.orc_cheb_gram.restype = None
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """Discrete problem description (grid, time steps, regulariser)."""

    def __init__(self, n, n_t, n_c=1, beta=1e-2, reg=1, stokes=False, dto=False):
        n = tuple(int(x) for x in n)
        self.n, self.d, self.n_t, self.n_c = n, len(n), int(n_t), int(n_c)
        self.beta, self.reg, self.stokes, self.dto = float(beta), int(reg), bool(stokes), bool(dto)
        nn = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
        self._p = Prob(self.d, nn, self.n_t, self.n_c, self.beta, self.reg, int(self.stokes), int(self.dto))

    @property
    def N(self):
        return int(np.prod(self.n))

    @property
    def hd(self):
        return float(np.prod([2 * np.pi / k for k in self.n]))

    def coef_shape(self):
        return (self.n_c, self.d) + self.n

    def _call(self, name, *args):
        st = getattr(lib(), name)(ctypes.byref(self._p), *args)
        if st != 0:
            raise RuntimeError(f"{name} failed with status {st}")

    # -- spectral operators --------------------------------------------
    def grad(self, u):
        u = _f64(u)
        out = np.empty((self.d,) + self.n)
        self._call("orc_grad", _ptr(u), _ptr(out))
        return out

    def div(self, w):
        w = _f64(w)
        out = np.empty(self.n)
        self._call("orc_div", _ptr(w), _ptr(out))
        return out

    def apply_A(self, u):
        u = _f64(u)
        out = np.empty(self.n)
        self._call("orc_apply_A", _ptr(u), _ptr(out))
        return out

    def leray(self, w):
        w = _f64(w)
        out = np.empty((self.d,) + self.n)
        self._call("orc_leray", _ptr(w), _ptr(out))
        return out

    def precond(self, r):
        r = _f64(r).reshape(self.coef_shape())
        out = np.empty(self.coef_shape())
        self._call("orc_precond", _ptr(r), _ptr(out))
        return out

    def reg_apply(self, v):
        v = _f64(v).reshape(self.coef_shape())
        out = np.empty(self.coef_shape())
        self._call("orc_reg_apply", _ptr(v), _ptr(out))
        return out

    # -- transport ------------------------------------------------------
    def state(self, v, m0, stages=False):
        v = _f64(v).reshape(self.coef_shape())
        m0 = _f64(m0)
        traj = np.empty((self.n_t + 1,) + self.n)
        mh = np.zeros((self.n_t + 1,) + self.n) if stages else None
        self._call("orc_state", _ptr(v), _ptr(m0), _ptr(traj), _ptr(mh))
        return (traj, mh) if stages else traj

    def adjoint(self, v, lam_end, stages=False):
        v = _f64(v).reshape(self.coef_shape())
        lam_end = _f64(lam_end)
        traj = np.empty((self.n_t + 1,) + self.n)
        lh = np.zeros((self.n_t + 1,) + self.n) if stages else None
        self._call("orc_adjoint", _ptr(v), _ptr(lam_end), _ptr(traj), _ptr(lh))
        return (traj, lh) if stages else traj

    # -- reduced-space operators ---------------------------------------
    def objective(self, v, mT, mR):
        v = _f64(v).reshape(self.coef_shape())
        out = np.empty(3)
        self._call("orc_objective", _ptr(v), _ptr(_f64(mT)), _ptr(_f64(mR)), _ptr(out))
        return float(out[0]), float(out[1]), float(out[2])

    def gradient(self, v, mT, mR):
        v = _f64(v).reshape(self.coef_shape())
        g = np.empty(self.coef_shape())
        J = np.empty(1)
        self._call("orc_gradient", _ptr(v), _ptr(_f64(mT)), _ptr(_f64(mR)), _ptr(g), _ptr(J))
        return g, float(J[0])

    def hessvec(self, v, mT, vt):
        v = _f64(v).reshape(self.coef_shape())
        vt = _f64(vt).reshape(self.coef_shape())
        out = np.empty(self.coef_shape())
        self._call("orc_hessvec", _ptr(v), _ptr(_f64(mT)), _ptr(vt), _ptr(out))
        return out

    def hessvec_newton(self, v, mT, mR, vt):
        """Full Newton Hessian matvec (trapezoid quadrature)."""
        v = _f64(v).reshape(self.coef_shape())
        vt = _f64(vt).reshape(self.coef_shape())
        out = np.empty(self.coef_shape())
        self._call("orc_hessvec_newton", _ptr(v), _ptr(_f64(mT)), _ptr(_f64(mR)), _ptr(vt), _ptr(out))
        return out

    def detF(self, v):
        v = _f64(v).reshape(self.coef_shape())
        out = np.empty(self.n)
        self._call("orc_detF", _ptr(v), _ptr(out))
        return out

    def detF_refined(self, v, refine, substeps=1):
        """det F_1 of App. D Eq. def-grad on the grid refined `refine` times per
        axis with substeps * n_t Heun steps: the velocity coefficients are
        carried to the fine grid by trigonometric interpolation without their
        Nyquist modes (trig_interp, nyquist="drop": the coarse first
        derivatives, reading R1, do not see those) and the oracle's own
        F-equation solve runs there."""
        v = _f64(v).reshape(self.coef_shape())
        nf = tuple(refine * k for k in self.n)
        vf = np.stack([np.stack([trig_interp(v[l, i], nf, "drop") for i in range(self.d)])
                       for l in range(self.n_c)])
        Pf = Problem(nf, self.n_t * substeps, self.n_c, self.beta, self.reg, self.stokes)
        return Pf.detF(vf)

    def defgrad(self, v):
        """F_1 of App. D Eq. def-grad, shape (d, d, *n)."""
        v = _f64(v).reshape(self.coef_shape())
        out = np.empty((self.d, self.d) + self.n)
        self._call("orc_defgrad", _ptr(v), _ptr(out))
        return out

    def grid_angle(self, v):
        """Per point, the smallest acute angle between deformed grid edges."""
        v = _f64(v).reshape(self.coef_shape())
        out = np.empty(self.n)
        self._call("orc_grid_angle", _ptr(v), _ptr(out))
        return out

    def displacement(self, v):
        """u_1 of App. D Eq. displacement, shape (d, *n); the map is y = x - u_1."""
        v = _f64(v).reshape(self.coef_shape())
        out = np.empty((self.d,) + self.n)
        self._call("orc_displacement", _ptr(v), _ptr(out))
        return out

    def smooth(self, m, sigma):
        """Gaussian presmoothing with standard deviation sigma."""
        out = np.empty(self.n)
        self._call("orc_smooth", float(sigma), _ptr(_f64(m)), _ptr(out))
        return out

    def lanczos(self, v, mT, q0, k, precond=False, mR=None, newton=False):
        """k Lanczos steps on H (or P^{-1} H); returns (alpha, beta, ritz) with the
        Ritz values (eigenvalues of the tridiagonal matrix) ascending."""
        from scipy.linalg import eigvalsh_tridiagonal
        v = _f64(v).reshape(self.coef_shape())
        q0 = _f64(q0).reshape(self.coef_shape())
        a, b = np.zeros(k), np.zeros(k)
        steps = ctypes.c_int(0)
        self._call("orc_lanczos", _ptr(v), _ptr(_f64(mT)), _ptr(None if mR is None else _f64(mR)), int(newton),
                   _ptr(q0), int(k), int(bool(precond)), _ptr(a), _ptr(b), ctypes.byref(steps))
        m = steps.value
        a, b = a[:m], b[:m]
        ritz = eigvalsh_tridiagonal(a, b[:m - 1]) if m > 1 else a.copy()
        return a, b, ritz

    def cfl(self, v):
        v = _f64(v).reshape(self.coef_shape())
        return float(lib().orc_cfl(ctypes.byref(self._p), _ptr(v)))

    def solve(self, mT, mR, v0=None, grad_rtol=1e-2, max_outer=50, armijo_c1=1e-4, backtrack=0.5,
              max_backtracks=20, pcg_maxit=0, newton=False, picard=False, step_memory=True, stop_rule=0,
              tau_J=1e-3, cfl_max=0.0):
        """Outer solve (Alg. 1). Returns (v, report dict); report["status"] is
        0, 6 (CFL halvings exhausted), 7 (line search failed) or 8 (iteration cap)."""
        v = np.zeros(self.coef_shape()) if v0 is None else _f64(v0).reshape(self.coef_shape()).copy()
        if newton and self.dto:
            raise ValueError("the full Newton Hessian uses the trapezoid quadrature")
        opts = Opts(grad_rtol, max_outer, armijo_c1, backtrack, max_backtracks, pcg_maxit, int(bool(newton)),
                    int(bool(picard)), int(bool(step_memory)), int(stop_rule), float(tau_J), float(cfl_max))
        rep = Report()
        st = lib().orc_solve(ctypes.byref(self._p), ctypes.byref(opts), _ptr(_f64(mT)), _ptr(_f64(mR)),
                             _ptr(v), ctypes.byref(rep))
        out = {f: getattr(rep, f) for f, _ in Report._fields_}
        out["status"] = st
        return v, out


def continuation(problem, mT, mR, v0=None, beta0=1.0, beta_min=1e-6, eps_F=0.1, eps_theta=0.0, beta_rtol=0.05,
                 dist_rtol=1e-2, cfl_target=0.0, max_solves=50, **solve_kw):
    """Beta continuation (Sec. 3.3.5) on `problem` (its beta is the start of
    nothing: beta0 is). Returns (v, report dict with the trace as lists)."""
    v = np.zeros(problem.coef_shape()) if v0 is None else _f64(v0).reshape(problem.coef_shape()).copy()
    so = dict(grad_rtol=1e-2, max_outer=50, armijo_c1=1e-4, backtrack=0.5, max_backtracks=20, pcg_maxit=0,
              newton=False, picard=False, step_memory=True, stop_rule=0, tau_J=1e-3, cfl_max=0.0)
    so.update(solve_kw)
    opts = Opts(so["grad_rtol"], so["max_outer"], so["armijo_c1"], so["backtrack"], so["max_backtracks"],
                so["pcg_maxit"], int(bool(so["newton"])), int(bool(so["picard"])), int(bool(so["step_memory"])),
                int(so["stop_rule"]), float(so["tau_J"]), float(so["cfl_max"]))
    co = ContOpts(beta0, beta_min, eps_F, eps_theta, beta_rtol, dist_rtol, cfl_target, max_solves)
    rep = ContReport()
    st = lib().orc_continuation(ctypes.byref(problem._p), ctypes.byref(opts), ctypes.byref(co), _ptr(_f64(mT)),
                                _ptr(_f64(mR)), _ptr(v), ctypes.byref(rep))
    if st != 0:
        raise RuntimeError(f"orc_continuation failed with status {st}")
    out = {}
    for f, _ in ContReport._fields_:
        val = getattr(rep, f)
        out[f] = list(val)[:rep.n_trace] if f.startswith("trace_") else val
    return v, out


def fft(a, inverse=False):
    """Complex FFT over all axes of ``a`` (oracle's own radix-2 transform)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    buf = a.view(np.float64).copy()
    n = (ctypes.c_int * a.ndim)(*a.shape)
    st = lib().orc_fft(a.ndim, n, _ptr(buf), int(bool(inverse)))
    if st != 0:
        raise RuntimeError(f"orc_fft failed with status {st}")
    return buf.view(np.complex128).reshape(a.shape)


def cheb_eval(n_c, t):
    b = np.empty(n_c)
    lib().orc_cheb_eval(int(n_c), float(t), _ptr(b))
    return b


def cheb_gram(n_c):
    C = np.empty((n_c, n_c))
    lib().orc_cheb_gram(int(n_c), _ptr(C))
    return C


def trig_interp(u, nf, nyquist="split"):
    """The trigonometric interpolant of the periodic grid values u (shape n) at
    the nodes of the grid nf (nf_a a multiple of n_a): per axis, the DFT
    coefficients of |k| < n_a/2 are kept and every finer mode is zero. The
    Nyquist coefficient k = n_a/2 is split in halves between +n_a/2 and -n_a/2
    (nyquist="split": the real interpolant of the samples) or dropped
    (nyquist="drop": the part of u that the masked first derivatives of the
    Nyquist reading R1 differentiate). numpy's FFT is the transform; the result
    is scaled by nf_a / n_a so that it holds point values."""
    out = np.asarray(u, dtype=np.float64)
    for a, m in enumerate(nf):
        n = out.shape[a]
        if m == n:
            continue
        U = np.moveaxis(np.fft.fft(out, axis=a), a, 0)
        W = np.zeros((m,) + U.shape[1:], dtype=np.complex128)
        h = n // 2
        W[:h] = U[:h]
        W[m - h + 1:] = U[h + 1:]
        if nyquist == "split":
            W[h] = 0.5 * U[h]
            W[m - h] = 0.5 * U[h]
        out = np.real(np.fft.ifft(np.moveaxis(W, 0, a), axis=a)) * (m / n)
    return out


def num_threads():
    return int(lib().orc_num_threads())
