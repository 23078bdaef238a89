"""Parity of the full Newton Hessian matvec (Eq. sec-order-opt-cond with the
pressure eliminated; trapezoid quadrature) with the oracle's
``hessvec_newton``.

The linearisation point is half the true velocity, so the residual
m_R - m_1 and with it the adjoint lambda are far from zero and the two Newton
terms (the source div(v~ lambda) of the incremental adjoint and the body force
lambda grad m~) are a sizeable part of the result. Tolerances as for the
Gauss-Newton matvec: FP64 relative 1e-10, mixed precision relative 1e-5.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1408_6299_gb300 import lib, synth
from gpu_util import cuda, empty, host, pair, rel, relmax

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def cases():
    out = [
        (synth.sinusoid_2d(32), "sin32"),
        (dict(synth.blobs_2d(64, n_t=8), n=(64, 64)), "blobs64"),
        (synth.stokes_3d(16, n_t=6, n_c=3), "stokes16"),
    ]
    for c, _ in out:
        P = O.Problem(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], c["stokes"])
        c["mR"] = P.state(c["v_true"], c["mT"])[-1]
    return out


@pytest.mark.parametrize("precision,ckpt", [
    (lib.REG_FP64, 0), (lib.REG_FP64, 2), (lib.REG_MIXED, 0), (lib.REG_MIXED, 2)])
def test_newton_hessvec(cases, precision, ckpt):
    tol = FP64_TOL if precision == lib.REG_FP64 else MIXED_TOL
    for c, label in cases:
        R, P = pair(c, precision=precision, ckpt=ckpt)
        R.set_hessian(lib.REG_HESS_NEWTON)
        R.set_images(cuda(c["mT"]), cuda(c["mR"]))
        v = 0.5 * c["v_true"]
        R.linearize(cuda(v))
        Hv = empty(R.coef_shape())
        R.hessvec(cuda(c["vt"]), Hv)
        ref = P.hessvec_newton(v, c["mT"], c["mR"], c["vt"])
        err = rel(host(Hv), ref)
        assert err < tol, (label, err)
        assert relmax(host(Hv), ref) < 10 * tol, label
        # the Newton terms are exercised: the result is far from Gauss-Newton
        assert rel(P.hessvec(v, c["mT"], c["vt"]), ref) > 1e-4, label


def test_newton_equals_gn_at_zero_residual(cases):
    # m_R = m_1(v): lambda = 0, so both Hessians coincide
    c, _ = cases[0]
    R, _ = pair(c)
    R.set_images(cuda(c["mT"]), cuda(c["mR"]))
    R.linearize(cuda(c["v_true"]))
    gn = empty(R.coef_shape())
    R.hessvec(cuda(c["vt"]), gn)
    R.set_hessian(lib.REG_HESS_NEWTON)
    R.linearize(cuda(c["v_true"]))
    nw = empty(R.coef_shape())
    R.hessvec(cuda(c["vt"]), nw)
    assert rel(host(nw), host(gn)) < 1e-12


def test_newton_switch_and_quadrature_rules(cases):
    c, _ = cases[0]
    R, _ = pair(c)
    R.set_images(cuda(c["mT"]), cuda(c["mR"]))
    R.linearize(cuda(0.5 * c["v_true"]))
    R.set_hessian(lib.REG_HESS_NEWTON)  # invalidates the linearisation point
    with pytest.raises(lib.RegError) as e:
        R.hessvec(cuda(c["vt"]), empty(R.coef_shape()))
    assert e.value.status == lib.REG_ENOTREADY
    assert R.L.reg_set_quadrature(R.ctx, lib.REG_QUAD_DISCRETE) == lib.REG_EINVAL
    with pytest.raises(lib.RegError) as e:
        R.set_hessian(7)
    assert e.value.status == lib.REG_EINVAL
    Rd, _ = pair(c, quad=1)
    with pytest.raises(lib.RegError) as e:
        Rd.set_hessian(lib.REG_HESS_NEWTON)
    assert e.value.status == lib.REG_EINVAL


def test_newton_solve_matches_oracle():
    # N-PCG (Sec. 4): iterate by iterate as the oracle's Newton solve, and
    # fewer outer iterations than Gauss-Newton to the same tolerance
    c = synth.sinusoid_2d(32)
    mR = O.Problem(c["n"], 16).state(c["v_true"], c["mT"])[-1]  # not reachable exactly with n_t = 8
    R = lib.Registration(c["n"], 8, 1, c["beta"], c["reg"], False, lib.REG_FP64, hessian=lib.REG_HESS_NEWTON)
    P = O.Problem(c["n"], 8, 1, c["beta"], c["reg"], False)
    R.set_images(cuda(c["mT"]), cuda(mR))
    v = cuda(np.zeros(R.coef_shape()))
    rep = R.solve(v, grad_rtol=1e-6, max_outer=30)
    vo, repo = P.solve(c["mT"], mR, grad_rtol=1e-6, max_outer=30, newton=True)
    _, repg = P.solve(c["mT"], mR, grad_rtol=1e-6, max_outer=30)
    assert rep["status"] == 0 and repo["status"] == 0
    assert (rep["outer"], rep["pcg_iters"], rep["ls_trials"]) == (repo["outer"], repo["pcg_iters"], repo["ls_trials"])
    assert rel(host(v), vo) < 1e-8
    assert rep["outer"] < repg["outer"]
    # mixed precision Krylov matvecs reach the same tolerance
    Rm = lib.Registration(c["n"], 8, 1, c["beta"], c["reg"], False, lib.REG_MIXED, hessian=lib.REG_HESS_NEWTON)
    Rm.set_images(cuda(c["mT"]), cuda(mR))
    vm = cuda(np.zeros(R.coef_shape()))
    repm = Rm.solve(vm, grad_rtol=1e-4, max_outer=30)
    assert repm["status"] == 0 and repm["g_inf"] <= 1e-4 * repm["g0_inf"]
    assert rel(host(vm), vo) < 1e-4
