"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Inputs are seeded synthetic workloads (paper_1408_6299_gb300.synth); the
reference image is the template transported by the true velocity with the
oracle's own solver, and both sides take that same m_R. Tolerances: FP64 path
relative 1e-10, mixed-precision Hessian matvec relative 1e-5 (per result,
relative 2-norm over the whole coefficient vector, plus an elementwise bound
against the largest entry).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1408_6299_gb300 import lib, synth
from gpu_util import cuda, empty, host, pair, rel, relmax

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-5


def small_cases():
    # (workload, label): grids chosen to cover 2D/3D, non-square shapes, several
    # FFT tiles per axis, partial row blocks, n_c > 1 and the Stokes scheme
    return [
        (synth.sinusoid_2d(32), "sin32"),
        (dict(synth.blobs_2d(64, n_t=8), n=(64, 64)), "blobs64"),
        (synth.stokes_3d(16, n_t=6, n_c=3), "stokes16"),
    ]


def nonsquare_case():
    r = np.random.default_rng(77)
    n = (8, 32, 16)
    mT = synth.random_spectral_field(n, r, 6.0)
    v = np.stack([synth.velocity_field(n, r, 3, 0.3)])
    vt = np.stack([synth.velocity_field(n, r, 3, 1.0)])
    return dict(name="nonsquare", n=n, n_t=4, n_c=1, beta=2e-2, reg=2, stokes=False, mT=mT, v_true=v, vt=vt)


@pytest.fixture(scope="module")
def cases():
    out = small_cases() + [(nonsquare_case(), "nonsq")]
    for c, _ in out:
        P = O.Problem(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], c["stokes"])
        c["mR"] = P.state(c["v_true"], c["mT"])[-1]
    return out


def test_spectral_operators(cases):
    for c, label in cases:
        R, P = pair(c)
        r = np.random.default_rng(5).standard_normal(R.coef_shape())
        out = empty(R.coef_shape())
        R.regularization(cuda(r), out)
        assert rel(host(out), P.reg_apply(r)) < 1e-12, label
        R.precond(cuda(r), out)
        assert rel(host(out), P.precond(r)) < 1e-12, label


def test_transport_and_objective(cases):
    for c, label in cases:
        R, P = pair(c)
        m1 = empty(c["n"])
        R.transport(cuda(c["v_true"]), cuda(c["mT"]), m1)
        ref = P.state(c["v_true"], c["mT"])[-1]
        assert rel(host(m1), ref) < FP64_TOL, label
        R.set_images(cuda(c["mT"]), cuda(c["mR"]))
        v = 0.5 * c["v_true"]
        J, parts = R.objective(cuda(v))
        Jo, do, ro = P.objective(v, c["mT"], c["mR"])
        assert abs(J - Jo) < FP64_TOL * Jo, label
        assert abs(parts[0] - do) < FP64_TOL * Jo and abs(parts[1] - ro) < FP64_TOL * Jo, label


@pytest.mark.parametrize("quad", [0, 1])
def test_gradient_fp64(cases, quad):
    for c, label in cases:
        R, P = pair(c, quad=quad)
        R.set_images(cuda(c["mT"]), cuda(c["mR"]))
        v = 0.5 * c["v_true"]
        g = empty(R.coef_shape())
        J = R.gradient(cuda(v), g)
        go, Jo = P.gradient(v, c["mT"], c["mR"])
        assert rel(host(g), go) < FP64_TOL, (label, rel(host(g), go))
        assert relmax(host(g), go) < 10 * FP64_TOL, label
        assert abs(J - Jo) < FP64_TOL * Jo, label


@pytest.mark.parametrize("precision,ckpt,quad", [
    (lib.REG_FP64, 0, 0), (lib.REG_FP64, 2, 0), (lib.REG_FP64, 0, 1), (lib.REG_FP64, 2, 1),
    (lib.REG_MIXED, 0, 0), (lib.REG_MIXED, 2, 0), (lib.REG_MIXED, 0, 1)])
def test_hessvec(cases, precision, ckpt, quad):
    tol = FP64_TOL if precision == lib.REG_FP64 else MIXED_TOL
    for c, label in cases:
        R, P = pair(c, precision=precision, ckpt=ckpt, quad=quad)
        R.set_images(cuda(c["mT"]), cuda(c["mR"]))
        v = c["v_true"]
        R.linearize(cuda(v))
        Hv = empty(R.coef_shape())
        R.hessvec(cuda(c["vt"]), Hv)
        ref = P.hessvec(v, c["mT"], c["vt"])
        err = rel(host(Hv), ref)
        assert err < tol, (label, err)
        assert relmax(host(Hv), ref) < 10 * tol, label


def test_hessvec_host_buffers_and_aliasing(cases):
    c, label = cases[0]
    R, P = pair(c)
    R.set_images(c["mT"], c["mR"])  # host numpy arrays: staged by the library
    R.linearize(c["v_true"])
    buf = np.ascontiguousarray(c["vt"], dtype=np.float64).copy()
    R.hessvec(buf, buf)  # aliasing input and output
    ref = P.hessvec(c["v_true"], c["mT"], c["vt"])
    assert rel(buf, ref) < FP64_TOL


def test_hessvec_before_point_is_rejected(cases):
    c, _ = cases[0]
    R, _ = pair(c)
    R.set_images(cuda(c["mT"]), cuda(c["mR"]))
    with pytest.raises(lib.RegError) as e:
        R.hessvec(cuda(c["vt"]), empty(R.coef_shape()))
    assert e.value.status == lib.REG_ENOTREADY


def test_transport_adjoint(cases):
    for c, label in cases:
        R, P = pair(c, quad=1)
        G = np.random.default_rng(3).standard_normal(c["n"])
        gv, gm0 = empty(R.coef_shape()), empty(c["n"])
        R.transport_adjoint(cuda(c["v_true"]), cuda(c["mT"]), cuda(G), gv, gm0)
        # oracle: with m_R = m_1 + G the adjoint starts from lambda_1 = -G
        Pn = O.Problem(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], False, dto=True)
        m1 = Pn.state(c["v_true"], c["mT"])[-1]
        g, _ = Pn.gradient(c["v_true"], c["mT"], m1 - G)
        f = g - Pn.reg_apply(c["v_true"])
        assert rel(host(gv), f) < FP64_TOL, label
        lam0 = Pn.adjoint(c["v_true"], -G)[0]
        assert rel(host(gm0), -lam0) < FP64_TOL, label


def test_detF_and_cfl(cases):
    for c, label in cases:
        R, P = pair(c)
        det = empty(c["n"])
        st = R.detF(cuda(c["v_true"]), 1, det)
        ref = P.detF(c["v_true"])
        assert relmax(host(det), ref) < 1e-12, label
        assert abs(st[0] - ref.min()) < 1e-12 and abs(st[1] - ref.max()) < 1e-12
        assert abs(st[2] - ref.mean()) < 1e-12 and abs(st[3] - ref.std()) < 1e-10
        assert abs(R.cfl(cuda(c["v_true"])) - P.cfl(c["v_true"])) < 1e-13


def test_solve_matches_oracle():
    c = synth.sinusoid_2d()
    R, P = pair(c)
    c["mR"] = P.state(c["v_true"], c["mT"])[-1]
    R.set_images(cuda(c["mT"]), cuda(c["mR"]))
    v = cuda(np.zeros(R.coef_shape()))
    rep = R.solve(v, grad_rtol=1e-2, detF_substeps=4)
    vo, repo = P.solve(c["mT"], c["mR"], grad_rtol=1e-2)
    assert rep["status"] == 0 and repo["status"] == 0
    assert rep["outer"] == repo["outer"] and rep["pcg_iters"] == repo["pcg_iters"]
    assert rep["ls_trials"] == repo["ls_trials"]
    assert rel(host(v), vo) < 1e-8
    assert abs(rep["J"] - repo["J"]) < 1e-8 * repo["J"]
    assert rep["g_inf"] <= 1e-2 * rep["g0_inf"]


def test_mixed_solve_reaches_tolerance():
    c = synth.blobs_2d(128)
    R, P = pair(c, precision=lib.REG_MIXED)
    c["mR"] = P.state(c["v_true"], c["mT"])[-1]
    R.set_images(cuda(c["mT"]), cuda(c["mR"]))
    v = cuda(np.zeros(R.coef_shape()))
    rep = R.solve(v, grad_rtol=1e-2)
    assert rep["status"] == 0
    assert rep["g_inf"] <= 1e-2 * rep["g0_inf"]
    vo, repo = P.solve(c["mT"], c["mR"], grad_rtol=1e-2)
    assert abs(rep["outer"] - repo["outer"]) <= 1
    assert rel(host(v), vo) < 1e-3


def test_bad_arguments_are_rejected():
    with pytest.raises(lib.RegError) as e:
        lib.Registration((12, 16), 4)
    assert e.value.status == lib.REG_EINVAL
    with pytest.raises(lib.RegError):
        lib.Registration((16, 16), 6, ckpt_every=4)
    with pytest.raises(lib.RegError):
        lib.Registration((16, 16), 4, beta=-1.0)


@pytest.mark.parametrize("n", [(512, 512), (512, 8), (8, 512), (8, 16, 512), (512, 8, 8)],
                         ids=["512x512", "512x8", "8x512", "8x16x512", "512x8x8"])
def test_extreme_grid_shapes(n):
    # the largest and smallest admissible axis lengths (8 and 512) on rows and on strided axes; the
    # speed keeps the CFL number below 0.2 with n_t = 2 on the 512-point axis (Heun is unstable above 1)
    r = np.random.default_rng(91)
    mT = synth.random_spectral_field(n, r, 3.0)
    v = np.stack([synth.velocity_field(n, r, 2, 0.004)])
    vt = np.stack([synth.velocity_field(n, r, 2, 1.0)])
    c = dict(n=n, n_t=2, n_c=1, beta=1e-2, reg=1, stokes=False)
    P = O.Problem(n, 2, 1, 1e-2, 1, False)
    mR = P.state(v, mT)[-1]
    for precision, tol in ((lib.REG_FP64, FP64_TOL), (lib.REG_MIXED, MIXED_TOL)):
        R, _ = pair(c, precision=precision)
        R.set_images(cuda(mT), cuda(mR))
        g = empty(R.coef_shape())
        R.gradient(cuda(0.5 * v), g)
        go, _ = P.gradient(0.5 * v, mT, mR)
        assert rel(host(g), go) < FP64_TOL, (n, precision)  # the gradient is FP64 in both precisions
        Hv = empty(R.coef_shape())
        R.hessvec(cuda(vt), Hv)
        assert rel(host(Hv), P.hessvec(0.5 * v, mT, vt)) < tol, (n, precision)


# ---------------------------------------------------------------------------
# Checkpointed contexts: the gradient and the transport adjoint recompute the
# state segment by segment from every K-th state (Alg. 1 with time
# checkpointing); the result must not depend on K.
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def ckpt_cases():
    out = [(synth.sinusoid_2d(32), "sin32"), (synth.stokes_3d(16, n_t=8, n_c=3), "stokes16-nc3")]
    for c, _ in out:
        P = O.Problem(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], c["stokes"])
        c["mR"] = P.state(c["v_true"], c["mT"])[-1]
    return out


@pytest.mark.parametrize("ckpt", [2, 4])
@pytest.mark.parametrize("quad", [0, 1])
def test_gradient_checkpointed(ckpt_cases, ckpt, quad):
    for c, label in ckpt_cases:
        R, P = pair(c, ckpt=ckpt, quad=quad)
        R.set_images(cuda(c["mT"]), cuda(c["mR"]))
        v = 0.5 * c["v_true"]
        g = empty(R.coef_shape())
        J = R.gradient(cuda(v), g)
        go, Jo = P.gradient(v, c["mT"], c["mR"])
        assert rel(host(g), go) < FP64_TOL, (label, ckpt, rel(host(g), go))
        assert relmax(host(g), go) < 10 * FP64_TOL, (label, ckpt, relmax(host(g), go))
        assert abs(J - Jo) < FP64_TOL * Jo, label


@pytest.mark.parametrize("ckpt", [2, 4])
@pytest.mark.parametrize("quad", [0, 1])
def test_transport_adjoint_checkpointed(ckpt_cases, ckpt, quad):
    for c, label in ckpt_cases:
        R, _ = pair(c, ckpt=ckpt, quad=quad)
        G = np.random.default_rng(3).standard_normal(c["n"])
        gv, gm0 = empty(R.coef_shape()), empty(c["n"])
        R.transport_adjoint(cuda(c["v_true"]), cuda(c["mT"]), cuda(G), gv, gm0)
        Pn = O.Problem(c["n"], c["n_t"], c["n_c"], c["beta"], c["reg"], False, dto=bool(quad))
        m1 = Pn.state(c["v_true"], c["mT"])[-1]
        g, _ = Pn.gradient(c["v_true"], c["mT"], m1 - G)  # lambda_1 = -G
        f = g - Pn.reg_apply(c["v_true"])
        assert rel(host(gv), f) < FP64_TOL, (label, ckpt, rel(host(gv), f))
        lam0 = Pn.adjoint(c["v_true"], -G)[0]
        assert rel(host(gm0), -lam0) < FP64_TOL, (label, ckpt)


# ---------------------------------------------------------------------------
# Full-spectrum inputs: white-noise template, velocity and direction carry
# every Fourier mode, the Nyquist modes included, through the packed DC /
# Nyquist slot of the row transforms, the masked first derivatives (reading
# R1) and the Leray projection.
# ---------------------------------------------------------------------------

def white_case(n):
    r = np.random.default_rng(404 + sum(n))
    n_t = max(4, max(n) // 16)  # CFL <= 0.25 for the speed 0.1 below
    if len(n) == 2:
        c = dict(n=n, n_t=n_t, n_c=1, beta=1e-2, reg=2, stokes=False)
    else:
        c = dict(n=n, n_t=n_t, n_c=2, beta=1e-2, reg=1, stokes=True)
    c["mT"] = synth.white_noise(n, r)
    c["v_true"] = synth.white_noise_velocity(n, r, c["n_c"], 0.1)
    c["vt"] = synth.white_noise_velocity(n, r, c["n_c"], 1.0)
    P = O.Problem(n, c["n_t"], c["n_c"], c["beta"], c["reg"], c["stokes"])
    c["mR"] = synth.white_noise(n, r)  # unrelated to m_T: a large adjoint everywhere
    return c, P


# Last axes of 64, 128 and 256 points run the edge-stage row kernels (pack and
# unpack partners over warp shuffles): every butterfly's partner modes and the
# packed DC/Nyquist slot carry content here, and 8 rows per field leave the
# divergence pass's row blocks (32 rows in single precision) partly empty.
FULL_SPECTRUM_SHAPES = [(16, 16), (8, 16, 32), (8, 64), (8, 256), (8, 8, 128), (8, 8, 256)]


@pytest.mark.parametrize("n", FULL_SPECTRUM_SHAPES, ids=["x".join(map(str, n)) for n in FULL_SPECTRUM_SHAPES])
@pytest.mark.parametrize("precision,ckpt", [(lib.REG_FP64, 0), (lib.REG_MIXED, 0), (lib.REG_MIXED, 2)])
def test_full_spectrum_inputs(n, precision, ckpt):
    c, P = white_case(n)
    tol = FP64_TOL if precision == lib.REG_FP64 else MIXED_TOL
    R, _ = pair(c, precision=precision, ckpt=ckpt)
    m1 = empty(n)
    R.transport(cuda(c["v_true"]), cuda(c["mT"]), m1)
    assert rel(host(m1), P.state(c["v_true"], c["mT"])[-1]) < FP64_TOL
    R.set_images(cuda(c["mT"]), cuda(c["mR"]))
    g = empty(R.coef_shape())
    J = R.gradient(cuda(c["v_true"]), g)
    go, Jo = P.gradient(c["v_true"], c["mT"], c["mR"])
    assert rel(host(g), go) < FP64_TOL, rel(host(g), go)  # the gradient is FP64 in both precisions
    assert abs(J - Jo) < FP64_TOL * Jo
    Hv = empty(R.coef_shape())
    R.hessvec(cuda(c["vt"]), Hv)
    ref = P.hessvec(c["v_true"], c["mT"], c["vt"])
    assert rel(host(Hv), ref) < tol, rel(host(Hv), ref)
    assert relmax(host(Hv), ref) < 10 * tol, relmax(host(Hv), ref)


# ---------------------------------------------------------------------------
# Large single-precision fields (over 16 MB per spectrum) take the paired
# column kernel: all strided passes of a stage in one persistent launch. The
# second shape has different x and y lengths (128 and 256): one launch per
# length. n_t = 2 and a slow velocity keep Heun's amplification of the top
# modes small (CFL <= 0.41).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [(256, 256, 128), (128, 256, 256)], ids=["256x256x128", "128x256x256"])
def test_mixed_matvec_with_paired_column_passes(n):
    r = np.random.default_rng(606)
    mT = synth.random_spectral_field(n, r, 24.0)
    mT /= mT.std()
    v = np.stack([synth.velocity_field(n, r, 4, 0.02)])
    vt = np.stack([synth.velocity_field(n, r, 4, 1.0)])
    c = dict(n=n, n_t=2, n_c=1, beta=1e-3, reg=2, stokes=False)
    P = O.Problem(n, 2, 1, 1e-3, 2, False)
    mR = P.state(v, mT)[-1]
    ref = P.hessvec(v, mT, vt)
    for ckpt in (0, 2):
        R, _ = pair(c, precision=lib.REG_MIXED, ckpt=ckpt)
        R.set_images(cuda(mT), cuda(mR))
        R.linearize(cuda(v))
        Hv = empty(R.coef_shape())
        R.hessvec(cuda(vt), Hv)
        err = rel(host(Hv), ref)
        assert err < MIXED_TOL, (ckpt, err)
        assert relmax(host(Hv), ref) < 10 * MIXED_TOL, ckpt
        R.close()


# ---------------------------------------------------------------------------
# det F_1 on a refined grid (reg_detF_refined): trigonometric interpolation of
# the velocity, with Nyquist content (white noise) and n_c = 2, then Eq.
# def-grad on the finer grid
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,refine,n_c", [((16, 16), 2, 1), ((16, 16), 4, 2), ((8, 16, 16), 2, 2)],
                         ids=["16x16-r2", "16x16-r4-nc2", "8x16x16-r2-nc2"])
def test_refined_detF_matches_oracle(n, refine, n_c):
    r = np.random.default_rng(808)
    v = synth.white_noise_velocity(n, r, n_c, 0.05)
    c = dict(n=n, n_t=4, n_c=n_c, beta=1e-2, reg=1, stokes=False)
    R, P = pair(c)
    out = empty(tuple(refine * k for k in n))
    st = R.detF_refined(cuda(v), 2, refine, out)
    ref = P.detF_refined(v, refine, 2)
    assert relmax(host(out), ref) < 1e-12
    assert abs(st[0] - ref.min()) < 1e-12 and abs(st[1] - ref.max()) < 1e-12
    assert abs(st[2] - ref.mean()) < 1e-12 and abs(st[3] - ref.std()) < 1e-10
    # refine = 1 is the plain evaluation
    assert R.detF_refined(cuda(v), 1, 1) == R.detF(cuda(v), 1)
