"""GPU parity of the rows around the solver (Sec. 3.3.5, App. D): Gaussian
presmoothing, the deformation map, the grid-angle measure, the Lanczos
spectrum estimate, beta / n_t changes of a context, and the beta
continuation, each against the oracle on the same seeded inputs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1408_6299_gb300 import lib, synth
from gpu_util import cuda, empty, host, pair, rel, relmax

pytestmark = pytest.mark.gpu


def cases():
    return [
        (synth.sinusoid_2d(32), "sin32"),
        (dict(synth.blobs_2d(64, n_t=8), n=(64, 64)), "blobs64"),
        (synth.stokes_3d(16, n_t=6, n_c=3), "stokes16"),
    ]


def test_smooth_matches_oracle():
    for c, label in cases():
        R, P = pair(c)
        for sigma in (0.0, 2 * np.pi / min(c["n"]), 0.5):
            out = empty(c["n"])
            R.smooth(sigma, cuda(c["mT"]), out)
            assert relmax(host(out), P.smooth(c["mT"], sigma)) < 1e-13, (label, sigma)
    # in place, host arrays
    c, _ = cases()[0]
    R, P = pair(c)
    m = np.ascontiguousarray(c["mT"]).copy()
    R.smooth(0.3, m, m)
    assert relmax(m, P.smooth(c["mT"], 0.3)) < 1e-13


def test_displacement_matches_oracle():
    for c, label in cases():
        R, P = pair(c)
        u = empty((len(c["n"]),) + tuple(c["n"]))
        R.displacement(cuda(c["v_true"]), u)
        ref = P.displacement(c["v_true"])
        assert rel(host(u), ref) < 1e-12, label


def test_grid_angle_and_detF_match_oracle():
    for c, label in cases():
        R, P = pair(c)
        ang = empty(c["n"])
        st = R.grid_angle(cuda(2.0 * c["v_true"]), 1, ang)
        ref = P.grid_angle(2.0 * c["v_true"])
        assert np.abs(host(ang) - ref).max() < 1e-10, label
        assert abs(st[0] - ref.min()) < 1e-10 and abs(st[1] - ref.max()) < 1e-10, label


def test_lanczos_matches_oracle():
    for c, label in cases()[:2]:
        R, P = pair(c)
        R.set_images(cuda(c["mT"]), cuda(c["mR"] if "mR" in c else c["mT"]))
        R.linearize(cuda(c["v_true"]))
        q0 = np.random.default_rng(8).standard_normal(R.coef_shape())
        for pre in (False, True):
            a, b, ritz = R.lanczos(cuda(q0), 12, precond=pre)
            ao, bo, ro = P.lanczos(c["v_true"], c["mT"], q0, 12, precond=pre)
            assert len(a) == 12
            assert np.abs(a[:6] - ao[:6]).max() < 1e-9 * np.abs(ao).max(), (label, pre)
            assert np.abs(b[:6] - bo[:6]).max() < 1e-9 * np.abs(bo).max(), (label, pre)
            assert abs(ritz[-1] - ro[-1]) < 1e-8 * abs(ro[-1]), (label, pre)
            # the library's own tridiagonal eigenvalues of its own coefficients
            from scipy.linalg import eigvalsh_tridiagonal
            assert np.abs(ritz - eigvalsh_tridiagonal(a, b[:-1])).max() < 1e-12 * np.abs(ritz).max()


def test_lanczos_reproduces_the_printed_beta_1e6_maxima():
    # Tab. 5.2: the largest eigenvalue at beta = 1e6 on 64^2
    c = synth.blobs_2d(64, n_t=8)
    for reg, stokes, value in ((2, False, 4.194304e12), (1, True, 2.048000e9)):
        R = lib.Registration((64, 64), 8, 1, 1e6, reg, stokes, lib.REG_FP64)
        R.set_images(cuda(c["mT"]), cuda(c["mT"]))
        R.linearize(cuda(c["v_true"]))
        q0 = np.random.default_rng(63).standard_normal(R.coef_shape())
        _, _, ritz = R.lanczos(cuda(q0), 40)
        assert float(f"{ritz[-1]:.6e}") == value, (reg, ritz[-1])


def test_lanczos_requires_a_point():
    c, _ = cases()[0]
    R, _ = pair(c)
    R.set_images(cuda(c["mT"]), cuda(c["mT"]))
    with pytest.raises(lib.RegError) as e:
        R.lanczos(cuda(np.ones(R.coef_shape())), 4)
    assert e.value.status == lib.REG_ENOTREADY


def test_set_beta_and_time_steps_with_graph_replay():
    # a context with its own stream replays its matvec as a CUDA graph: a new
    # beta, n_t or Hessian kind must be seen by the next matvec
    import torch
    c = synth.sinusoid_2d(32)
    mR = O.Problem(c["n"], 16).state(c["v_true"], c["mT"])[-1]
    s = torch.cuda.Stream()
    R = lib.Registration(c["n"], 8, 1, c["beta"], c["reg"], False, lib.REG_FP64, stream=s.cuda_stream)
    R.set_images(cuda(c["mT"]), cuda(mR))
    v = 0.5 * c["v_true"]
    R.linearize(cuda(v))
    out = empty(R.coef_shape())
    for beta, nt, hess in ((c["beta"], 8, 0), (0.3, 8, 0), (0.3, 8, 1), (0.3, 12, 1), (0.3, 12, 0)):
        R.set_beta(beta)
        if nt != R.n_t:
            R.set_time_steps(nt)
        R.set_hessian(hess)
        R.linearize(cuda(v))
        R.hessvec(cuda(c["vt"]), out)
        R.hessvec(cuda(c["vt"]), out)  # the replayed graph
        s.synchronize()
        P = O.Problem(c["n"], nt, 1, beta, c["reg"], False)
        ref = P.hessvec_newton(v, c["mT"], mR, c["vt"]) if hess else P.hessvec(v, c["mT"], c["vt"])
        assert rel(host(out), ref) < 1e-10, (beta, nt, hess)


def continuation_setup(precision=lib.REG_FP64):
    c = synth.sinusoid_2d(32)
    mR = O.Problem(c["n"], 16).state(2 * c["v_true"], c["mT"])[-1]
    R = lib.Registration(c["n"], 8, 1, 1.0, 1, False, precision)
    R.set_images(cuda(c["mT"]), cuda(mR))
    P = O.Problem(c["n"], 8, 1, 1.0, 1, False)
    return c, mR, R, P


@pytest.mark.parametrize("kw", [dict(eps_F=0.8), dict(eps_F=0.0, eps_theta=1.2), dict(eps_F=0.8, cfl_target=0.05),
                                dict(eps_F=0.99)], ids=["detF", "angle", "cfl", "none"])
def test_continuation_matches_oracle(kw):
    c, mR, R, P = continuation_setup()
    v = cuda(np.zeros(R.coef_shape()))
    rep = R.continuation(v, solve_opts=dict(max_outer=20, pcg_maxit=100), **kw)
    vo, repo = O.continuation(P, c["mT"], mR, max_outer=20, pcg_maxit=100, **kw)
    for k in ("found", "stop", "solves", "n_t", "n_trace", "trace_ok"):
        assert rep[k] == repo[k], (k, rep[k], repo[k])
    assert np.allclose(rep["trace_beta"], repo["trace_beta"], rtol=1e-14)
    assert np.allclose(rep["trace_detF"], repo["trace_detF"], rtol=1e-8)
    assert abs(rep["beta"] - repo["beta"]) <= 1e-14 * repo["beta"]
    assert rel(host(v), vo) < 1e-7


def test_continuation_mixed_precision_reaches_the_same_beta():
    c, mR, R, P = continuation_setup(lib.REG_MIXED)
    v = cuda(np.zeros(R.coef_shape()))
    rep = R.continuation(v, solve_opts=dict(max_outer=20, pcg_maxit=100), eps_F=0.8)
    _, repo = O.continuation(P, c["mT"], mR, eps_F=0.8, max_outer=20, pcg_maxit=100)
    assert rep["found"] and rep["trace_ok"] == repo["trace_ok"]
    assert abs(rep["beta"] - repo["beta"]) <= 1e-12 * repo["beta"]
