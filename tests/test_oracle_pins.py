"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself.

Each test cites the passage of Mang & Biros (arXiv:1408.6299) it follows and
checks the oracle against one of: a brute-force O(N^2) DFT, numpy's FFT (an
independent transform), closed forms of the discrete scheme, dense-matrix
brute force of the whole discrete method on tiny grids, exact identities of
the discretisation (skew-adjointness, adjoint transport, mass conservation,
Gauss-Newton energy identity), finite differences, and values printed in the
paper (Tab. 5.2 eigenvalue maxima, tests/golden/).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1408_6299_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed):
    return np.random.default_rng(seed)


def hd(n):
    return float(np.prod([2 * np.pi / k for k in n]))


# ---------------------------------------------------------------------------
# P1 FFT (Sec. 3.3.1 "Fourier spectral methods"): brute-force DFT, inverse, Parseval
# ---------------------------------------------------------------------------

def brute_dft(a, inverse=False):
    out = a.astype(np.complex128)
    sign = 1.0 if inverse else -1.0
    for ax, n in enumerate(a.shape):
        j = np.arange(n)
        W = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
        out = np.moveaxis(np.tensordot(W, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
        if inverse:
            out = out / n
    return out


@pytest.mark.parametrize("shape", [(2,), (8,), (32,), (8, 8), (4, 16), (4, 4, 4), (2, 8, 4)])
def test_fft_matches_bruteforce_dft(shape):
    r = rng(sum(shape))
    a = r.standard_normal(shape) + 1j * r.standard_normal(shape)
    F = O.fft(a)
    ref = brute_dft(a)
    assert np.abs(F - ref).max() <= 1e-13 * np.abs(ref).max()
    back = O.fft(F, inverse=True)
    assert np.abs(back - a).max() <= 1e-14 * np.abs(a).max() * 10
    assert np.abs(O.fft(a, inverse=True) - brute_dft(a, inverse=True)).max() <= 1e-13 * np.abs(a).max()
    # Parseval: sum |a|^2 = (1/N) sum |F|^2
    N = a.size
    assert abs((np.abs(a) ** 2).sum() - (np.abs(F) ** 2).sum() / N) <= 1e-12 * (np.abs(a) ** 2).sum()


def test_fft_larger_against_numpy():
    a = rng(3).standard_normal((16, 32, 8)) + 0j
    assert np.abs(O.fft(a) - np.fft.fftn(a)).max() <= 1e-12 * np.abs(np.fft.fftn(a)).max()


# ---------------------------------------------------------------------------
# P2 spectral derivatives, A and K on trigonometric polynomials (Sec. 3.3.1,
# Eq. first-variation-H1/H2, Eq. eliminated-control)
# ---------------------------------------------------------------------------

def test_gradient_of_sin2_template_is_exact():
    n = (32, 32)
    P = O.Problem(n, 4)
    X = synth.coords(n)
    u = 0.5 * (np.sin(X[0]) ** 2 + np.sin(X[1]) ** 2)
    g = P.grad(u)
    assert np.abs(g[0] - 0.5 * np.sin(2 * X[0])).max() < 1e-13
    assert np.abs(g[1] - 0.5 * np.sin(2 * X[1])).max() < 1e-13


def test_gradient_divergence_3d_trig():
    n = (8, 16, 8)
    P = O.Problem(n, 4)
    X = synth.coords(n)
    u = np.sin(2 * X[0] + X[1]) * np.cos(3 * X[2]) + np.cos(X[1] - X[0])
    g = P.grad(u)
    ex = [2 * np.cos(2 * X[0] + X[1]) * np.cos(3 * X[2]) + np.sin(X[1] - X[0]),
          np.cos(2 * X[0] + X[1]) * np.cos(3 * X[2]) - np.sin(X[1] - X[0]),
          -3 * np.sin(2 * X[0] + X[1]) * np.sin(3 * X[2])]
    for i in range(3):
        assert np.abs(g[i] - ex[i]).max() < 1e-13
    w = np.stack([np.sin(X[1]), np.cos(X[0] + X[2]), np.sin(2 * X[2])])
    assert np.abs(P.div(w) - 2 * np.cos(2 * X[2])).max() < 1e-13


def test_nyquist_reading():
    """Reading R1: first derivatives drop the Nyquist mode; a(k) keeps it."""
    n = (16, 8)
    X = synth.coords(n)
    u = np.cos(8 * X[0])  # pure Nyquist mode on axis 0
    for reg in (1, 2):
        P = O.Problem(n, 4, reg=reg)
        assert np.abs(P.grad(u)).max() < 1e-14
        assert np.abs(P.apply_A(u) - (64.0 ** reg) * u).max() < 1e-9 * 64.0 ** reg


@pytest.mark.parametrize("reg", [1, 2])
def test_apply_A_symbol(reg):
    n = (16, 16, 16)
    P = O.Problem(n, 4, reg=reg)
    X = synth.coords(n)
    u = np.cos(3 * X[0] - 2 * X[1] + 5 * X[2]) + 2.0
    kk = 9 + 4 + 25
    assert np.abs(P.apply_A(u) - kk ** reg * (u - 2.0)).max() < 1e-10 * kk ** reg


def test_leray_on_gradient_and_solenoidal_fields():
    n = (16, 16)
    P = O.Problem(n, 4)
    X = synth.coords(n)
    phi = np.sin(2 * X[0]) * np.cos(X[1])
    gphi = P.grad(phi)
    assert np.abs(P.leray(gphi)).max() < 1e-13
    psi = np.cos(X[0] + 3 * X[1])
    sol = np.stack([-3 * np.sin(X[0] + 3 * X[1]), np.sin(X[0] + 3 * X[1])])  # curl of psi: div = 0
    assert np.abs(P.leray(sol) - sol).max() < 1e-13
    const = np.ones((2,) + n)
    assert np.abs(P.leray(const) - const).max() < 1e-14


# ---------------------------------------------------------------------------
# P3 skew/self-adjointness, projector identities
# ---------------------------------------------------------------------------

def test_skew_and_projector_identities():
    n = (8, 16, 8)
    P = O.Problem(n, 4)
    r = rng(5)
    a, b = r.standard_normal(n), r.standard_normal(n)
    ga, gb = P.grad(a), P.grad(b)
    for i in range(3):
        assert abs((ga[i] * b).sum() + (a * gb[i]).sum()) < 1e-12 * np.abs(ga[i] * b).sum()
    w, z = r.standard_normal((3,) + n), r.standard_normal((3,) + n)
    Kw, Kz = P.leray(w), P.leray(z)
    assert abs((Kw * z).sum() - (w * Kz).sum()) < 1e-12 * np.abs(w * z).sum()
    assert np.abs(P.leray(Kw) - Kw).max() < 1e-13 * np.abs(Kw).max()
    assert np.abs(P.div(Kw)).max() < 1e-12 * np.abs(w).max()
    Aa = P.apply_A(a)
    assert abs((Aa * b).sum() - (a * P.apply_A(b)).sum()) < 1e-12 * np.abs(Aa * b).sum()


# ---------------------------------------------------------------------------
# Chebyshev basis and Gram matrix (Sec. 3.3.2, App. A; reading R3)
# ---------------------------------------------------------------------------

def test_chebyshev_basis_and_gram():
    from numpy.polynomial import chebyshev as C
    for nc in (1, 2, 5):
        for t in (0.0, 0.3, 1.0):
            ref = [C.chebval(2 * t - 1, [0] * l + [1]) for l in range(nc)]
            assert np.allclose(O.cheb_eval(nc, t), ref, atol=1e-15)
        x, w = np.polynomial.legendre.leggauss(40)
        t = 0.5 * (x + 1)
        B = np.stack([C.chebval(2 * t - 1, [0] * l + [1]) for l in range(nc)])
        ref = 0.5 * (B * w) @ B.T
        assert np.abs(O.cheb_gram(nc) - ref).max() < 1e-14


# ---------------------------------------------------------------------------
# P4 preconditioner (Sec. 3.3.3; Sec. 3.2.1 left preconditioner beta A)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nc,reg", [(1, 1), (1, 2), (3, 1)])
def test_preconditioner_inverts_regularisation(nc, reg):
    n = (16, 8)
    P = O.Problem(n, 4, n_c=nc, beta=3e-3, reg=reg)
    r = rng(7)
    u = r.standard_normal(P.coef_shape())
    u -= u.mean(axis=(2, 3), keepdims=True)
    back = P.precond(P.reg_apply(u))
    assert np.abs(back - u).max() < 1e-12 * np.abs(u).max()
    # k = 0 mode: identity (times C^-1 across coefficients)
    c = np.ones(P.coef_shape()) * r.standard_normal((nc, 2, 1, 1))
    Cinv = np.linalg.inv(O.cheb_gram(nc))
    assert np.abs(P.precond(c) - np.einsum("lm,mi...->li...", Cinv, c)).max() < 1e-13


def test_reg_apply_against_numpy():
    n = (16, 16)
    P = O.Problem(n, 4, n_c=2, beta=0.7, reg=2)
    r = rng(8)
    v = r.standard_normal(P.coef_shape())
    k = np.fft.fftfreq(16, 1 / 16)
    k[8] = -8
    K = np.meshgrid(k, k, indexing="ij")
    a = (K[0] ** 2 + K[1] ** 2) ** 2
    Av = np.real(np.fft.ifftn(a * np.fft.fftn(v, axes=(2, 3)), axes=(2, 3)))
    ref = 0.7 * np.einsum("lm,mi...->li...", O.cheb_gram(2), Av)
    assert np.abs(P.reg_apply(v) - ref).max() < 1e-10 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# P5 constant velocity: closed form of the Heun scheme (Sec. 3.3.1)
# ---------------------------------------------------------------------------

def test_constant_velocity_closed_form():
    n = (16, 8)
    nt = 8
    P = O.Problem(n, nt)
    c = np.array([0.37, -0.8])
    v = np.ones((1, 2) + n) * c[None, :, None, None]
    m0 = rng(9).standard_normal(n)
    mt = P.state(v, m0)
    k = [np.fft.fftfreq(m, 1 / m) for m in n]
    for i, m in enumerate(n):
        k[i][m // 2] = 0.0  # masked first-derivative wavenumber
    K = np.meshgrid(*k, indexing="ij")
    z = (1.0 / nt) * (-1j) * (c[0] * K[0] + c[1] * K[1])
    R = 1 + z + z * z / 2
    ref = np.real(np.fft.ifftn(R ** nt * np.fft.fftn(m0)))
    assert np.abs(mt[-1] - ref).max() < 1e-13 * np.abs(m0).max() * 10
    det = P.detF(v)
    assert np.abs(det - 1).max() < 1e-14


# ---------------------------------------------------------------------------
# P6 mass conservation (div-free v) and adjoint mass conservation (any v)
# ---------------------------------------------------------------------------

def test_mass_conservation():
    c = synth.stokes_3d(16, n_t=8, n_c=2)
    P = O.Problem(c["n"], 8, n_c=2)
    mt = P.state(c["v_true"], c["mT"])
    s0 = c["mT"].sum()
    assert np.abs(mt.reshape(9, -1).sum(axis=1) - s0).max() < 1e-12 * np.abs(c["mT"]).sum()
    v = rng(10).standard_normal(P.coef_shape()) * 0.1  # not divergence-free
    lam = P.adjoint(v, c["mT"])
    assert np.abs(lam.reshape(9, -1).sum(axis=1) - s0).max() < 1e-12 * np.abs(c["mT"]).sum()


# ---------------------------------------------------------------------------
# P7 exact discrete transport adjoint: <Phi m0, w> = <m0, Phi^T w> (Eq.
# first-order-forward / first-order-adjoint; one Heun step transposes into the
# backward Heun step because L^T = D)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nc", [1, 3])
def test_transport_adjoint_identity(nc):
    n = (8, 16)
    P = O.Problem(n, 6, n_c=nc)
    r = rng(11 + nc)
    v = 0.3 * r.standard_normal(P.coef_shape())
    m0, w = r.standard_normal(n), r.standard_normal(n)
    lhs = (P.state(v, m0)[-1] * w).sum()
    rhs = (m0 * P.adjoint(v, w)[0]).sum()
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + np.abs(m0 * w).sum())


# ---------------------------------------------------------------------------
# P8 zero velocity closed forms (Eq. first-order-control, Eq. gauss-newton)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("stokes", [False, True])
def test_zero_velocity_gradient_and_hessian(stokes):
    n = (16, 16)
    X = synth.coords(n)
    mT = 0.5 * (np.sin(X[0]) ** 2 + np.sin(X[1]) ** 2)
    gmT = np.stack([0.5 * np.sin(2 * X[0]), 0.5 * np.sin(2 * X[1])])
    mR = np.cos(X[0] + X[1]) * 0.3 + mT
    P = O.Problem(n, 4, beta=0.05, reg=1, stokes=stokes)
    v0 = np.zeros(P.coef_shape())
    g, J = P.gradient(v0, mT, mR)
    f = (mR - mT) * gmT
    if stokes:  # independent Leray projection via numpy
        k = np.fft.fftfreq(16, 1 / 16)
        k[8] = 0
        K = np.meshgrid(k, k, indexing="ij")
        kk = K[0] ** 2 + K[1] ** 2
        kk[kk == 0] = 1.0  # numerator vanishes there too: identity on those modes
        F = np.fft.fftn(f, axes=(1, 2))
        dotk = K[0] * F[0] + K[1] * F[1]
        f = np.real(np.fft.ifftn(np.stack([F[0] - K[0] * dotk / kk, F[1] - K[1] * dotk / kk]), axes=(1, 2)))
    assert np.abs(g[0] - f).max() < 1e-13
    assert abs(J - 0.5 * hd(n) * ((mR - mT) ** 2).sum()) < 1e-13 * J
    vt = np.stack([np.cos(X[1]), np.sin(2 * X[0] + X[1])])[None]
    H = P.hessvec(v0, mT, vt)
    s = (gmT * vt[0]).sum(axis=0)
    data = s * gmT
    if stokes:
        F = np.fft.fftn(data, axes=(1, 2))
        dotk = K[0] * F[0] + K[1] * F[1]
        data = np.real(np.fft.ifftn(np.stack([F[0] - K[0] * dotk / kk, F[1] - K[1] * dotk / kk]), axes=(1, 2)))
    reg = 0.05 * np.stack([vt[0, 0] * 1.0, vt[0, 1] * 5.0])  # |k|^2 of each component
    assert np.abs(H[0] - (reg + data)).max() < 1e-13


# ---------------------------------------------------------------------------
# P9 printed eigenvalue maxima at beta = 1e6 (Tab. 5.2)
# ---------------------------------------------------------------------------

def test_beta_1e6_eigenvalue_maxima_match_paper():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "eigen_beta1e6_64.txt")) if not ln.startswith("#")]
    c = synth.blobs_2d(64, n_t=8)
    for reg_name, stokes, value, digits in rows:
        reg = 1 if reg_name == "H1" else 2
        P = O.Problem((64, 64), 8, beta=1e6, reg=reg, stokes=bool(int(stokes)))
        j = np.arange(64)
        e = np.zeros(P.coef_shape())
        e[0, 0] = np.outer((-1.0) ** j, (-1.0) ** j)  # Nyquist corner mode, the top of a(k)
        x = e
        for _ in range(3):  # a few power steps from the corner mode
            Hx = P.hessvec(c["v_true"], c["mT"], x)
            lam = (x * Hx).sum() / (x * x).sum()
            x = Hx / np.abs(Hx).max()
        assert float(f"{lam:.{int(digits) - 1}e}") == float(value)


# ---------------------------------------------------------------------------
# Dense brute force of the whole discrete method on a tiny grid (Sec. 3.3.1,
# Alg. 1-2, Eq. gauss-newton, App. A): every operator is an explicit matrix
# built from numpy's FFT, the Heun steps are matrix products.
# ---------------------------------------------------------------------------

class Dense:
    def __init__(self, n, nt, nc, beta, reg, stokes):
        self.n, self.nt, self.nc, self.beta = n, nt, nc, beta
        N = int(np.prod(n))
        self.N, self.d = N, len(n)
        I = np.eye(N).reshape((N,) + n)
        axes = tuple(range(1, self.d + 1))
        FI = np.fft.fftn(I, axes=axes)
        ks = []
        for i, m in enumerate(n):
            k = np.fft.fftfreq(m, 1 / m)
            k[m // 2] = -m // 2
            ks.append(k)
        Kf = np.meshgrid(*ks, indexing="ij")
        Km = [np.where(np.abs(k) == m // 2, 0.0, k) for k, m in zip(Kf, n)]
        def op(sym):
            return np.real(np.fft.ifftn(FI * sym[None], axes=axes)).reshape(N, N).T
        self.D = [op(1j * Km[i]) for i in range(self.d)]
        a = sum(k ** 2 for k in Kf) ** reg
        self.A = op(a)
        kk = sum(k ** 2 for k in Km)
        kk1 = np.where(kk == 0, 1.0, kk)
        self.K = None
        if stokes:
            blocks = [[op((1.0 if i == j else 0.0) - np.where(kk == 0, 0.0, Km[i] * Km[j] / kk1)) for j in range(self.d)]
                      for i in range(self.d)]
            self.K = np.block(blocks)
        self.C = O.cheb_gram(nc)
        self.h = 1.0 / nt

    def b(self, t):
        from numpy.polynomial import chebyshev as C
        return np.array([C.chebval(2 * t - 1, [0] * l + [1]) for l in range(self.nc)])

    def vel(self, v, t):
        return np.einsum("l,lix->ix", self.b(t), v.reshape(self.nc, self.d, self.N))

    def L(self, v, t):
        vt = self.vel(v, t)
        return -sum(vt[i][:, None] * self.D[i] for i in range(self.d))

    def state(self, v, m0):
        ms = [m0.reshape(-1)]
        h = self.h
        for j in range(self.nt):
            La, Lb = self.L(v, j * h), self.L(v, (j + 1) * h)
            step = np.eye(self.N) + h / 2 * (La + Lb) + h * h / 2 * Lb @ La
            ms.append(step @ ms[-1])
        return ms

    def adjoint(self, v, lend):
        h = self.h
        ls = [None] * (self.nt + 1)
        ls[-1] = lend
        for j in range(self.nt - 1, -1, -1):
            La, Lb = self.L(v, j * h), self.L(v, (j + 1) * h)
            step = np.eye(self.N) + h / 2 * (La + Lb) + h * h / 2 * Lb @ La
            ls[j] = step.T @ ls[j + 1]
        return ls

    def force(self, ms, ls):
        h = self.h
        f = np.zeros((self.nc, self.d, self.N))
        for j in range(self.nt + 1):
            w = h / 2 if j in (0, self.nt) else h
            gm = np.stack([D @ ms[j] for D in self.D])
            f += w * self.b(j * h)[:, None, None] * (ls[j] * gm)[None]
        return f

    def tail(self, v, f):
        v = v.reshape(self.nc, self.d, self.N)
        out = self.beta * np.einsum("lm,mix->lix", self.C, np.einsum("xy,miy->mix", self.A, v))
        for l in range(self.nc):
            out[l] += (self.K @ f[l].reshape(-1)).reshape(self.d, self.N) if self.K is not None else f[l]
        return out

    def hessvec(self, v, mT, vt):
        ms = self.state(v, mT)
        h = self.h
        y = np.zeros(self.N)
        for j in range(self.nt):
            La, Lb = self.L(v, j * h), self.L(v, (j + 1) * h)
            sa = -(np.stack([D @ ms[j] for D in self.D]) * self.vel(vt, j * h)).sum(0)
            sb = -(np.stack([D @ ms[j + 1] for D in self.D]) * self.vel(vt, (j + 1) * h)).sum(0)
            k1 = La @ y + sa
            k2 = Lb @ (y + h * k1) + sb
            y = y + h / 2 * (k1 + k2)
        ls = self.adjoint(v, -y)
        return self.tail(vt, self.force(ms, ls))

    def gradient(self, v, mT, mR):
        ms = self.state(v, mT)
        ls = self.adjoint(v, mR.reshape(-1) - ms[-1])
        return self.tail(v, self.force(ms, ls))


@pytest.mark.parametrize("nc,reg,stokes", [(1, 1, False), (2, 2, False), (2, 1, True)])
def test_whole_method_matches_dense_brute_force(nc, reg, stokes):
    n = (8, 4)
    nt = 3
    r = rng(20 + nc + reg)
    v = 0.4 * r.standard_normal((nc, 2) + n)
    vt = r.standard_normal((nc, 2) + n)
    X = synth.coords(n)
    mT = np.sin(X[0]) * np.cos(X[1]) + 0.2 * r.standard_normal(n)
    mR = r.standard_normal(n)
    P = O.Problem(n, nt, n_c=nc, beta=0.03, reg=reg, stokes=stokes)
    Dn = Dense(n, nt, nc, 0.03, reg, stokes)
    H = P.hessvec(v, mT, vt).reshape(nc, 2, -1)
    Hd = Dn.hessvec(v, mT, vt)
    assert np.abs(H - Hd).max() < 1e-12 * np.abs(Hd).max()
    g, J = P.gradient(v, mT, mR)
    gd = Dn.gradient(v, mT, mR)
    assert np.abs(g.reshape(nc, 2, -1) - gd).max() < 1e-12 * np.abs(gd).max()
    m1 = Dn.state(v, mT)[-1]
    vv = v.reshape(nc, 2, -1)
    reg_term = 0.03 * np.einsum("lm,lix,xy,miy->", O.cheb_gram(nc), vv, Dn.A, vv)
    Jd = 0.5 * hd(n) * (((mR.reshape(-1) - m1) ** 2).sum() + reg_term)
    assert abs(J - Jd) < 1e-12 * Jd
    assert abs(P.objective(v, mT, mR)[0] - Jd) < 1e-12 * Jd


# ---------------------------------------------------------------------------
# P10-P12 discrete-adjoint (test-only) variant: energy identity, FD of J,
# Hessian symmetry and the inverse-crime Newton limit; trapezoid variant
# converges to it at second order (reading R4).
# ---------------------------------------------------------------------------

def small_problem(nt=8, nc=2, stokes=False, dto=True, reg=1):
    n = (16, 16)
    r = rng(30)
    X = synth.coords(n)
    mT = 0.5 * (np.sin(X[0]) ** 2 + np.sin(X[1]) ** 2) + 0.05 * synth.random_spectral_field(n, r, 4.0)
    v = np.stack([synth.velocity_field(n, r, 4, 0.3, divergence_free=stokes) for _ in range(nc)])
    P = O.Problem(n, nt, n_c=nc, beta=1e-2, reg=reg, stokes=stokes, dto=dto)
    return P, mT, v, r


def test_gn_energy_identity_dto():
    P, mT, v, r = small_problem()
    vt = np.stack([synth.velocity_field(P.n, r, 6, 1.0) for _ in range(2)])
    H = P.hessvec(v, mT, vt)
    data = H - P.reg_apply(vt)
    eps = 1e-5
    mp = P.state(v + eps * vt, mT)[-1]
    mm = P.state(v - eps * vt, mT)[-1]
    dm = (mp - mm) / (2 * eps)
    lhs = P.hd * (vt * data).sum()
    rhs = P.hd * (dm ** 2).sum()
    assert abs(lhs - rhs) < 1e-8 * rhs


def test_gradient_matches_finite_differences_dto():
    P, mT, v, r = small_problem()
    mR = P.state(v * 1.3, mT)[-1] + 0.01 * synth.random_spectral_field(P.n, r, 5.0)
    g, J = P.gradient(v, mT, mR)
    eps = 1e-6
    for s in range(5):
        w = rng(100 + s).standard_normal(P.coef_shape())
        fd = (P.objective(v + eps * w, mT, mR)[0] - P.objective(v - eps * w, mT, mR)[0]) / (2 * eps)
        an = P.hd * (g * w).sum()
        assert abs(fd - an) < 1e-7 * abs(an) + 1e-10


def test_hessian_symmetry_dto_and_inverse_crime_newton_limit():
    P, mT, v, r = small_problem(stokes=False)
    a = rng(40).standard_normal(P.coef_shape())
    b = rng(41).standard_normal(P.coef_shape())
    Ha, Hb = P.hessvec(v, mT, a), P.hessvec(v, mT, b)
    assert abs((b * Ha).sum() - (a * Hb).sum()) < 1e-12 * abs((b * Ha).sum())
    mR = P.state(v, mT)[-1]  # inverse crime: lambda = 0, GN equals Newton
    eps = 1e-5
    gp = P.gradient(v + eps * a, mT, mR)[0]
    gm = P.gradient(v - eps * a, mT, mR)[0]
    assert np.abs((gp - gm) / (2 * eps) - Ha).max() < 1e-7 * np.abs(Ha).max()


def test_trapezoid_converges_to_discrete_adjoint_at_second_order():
    errs = []
    for nt in (8, 16, 32):
        Pd, mT, v, r = small_problem(nt=nt, dto=True)
        Pt, _, _, _ = small_problem(nt=nt, dto=False)
        vt = rng(50).standard_normal(Pd.coef_shape())
        Hd, Ht = Pd.hessvec(v, mT, vt), Pt.hessvec(v, mT, vt)
        errs.append(np.linalg.norm(Hd - Ht) / np.linalg.norm(Hd))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


# ---------------------------------------------------------------------------
# P13 second order in time of the state solve (Sec. 1.2: second order in time)
# ---------------------------------------------------------------------------

def test_state_second_order_in_time():
    c = synth.sinusoid_2d()
    ref = O.Problem(c["n"], 512).state(c["v_true"], c["mT"])[-1]
    errs = [np.abs(O.Problem(c["n"], nt).state(c["v_true"], c["mT"])[-1] - ref).max() for nt in (16, 32, 64)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2) < 0.15), (errs, rates)


# ---------------------------------------------------------------------------
# P14 det F for a divergence-free velocity (App. D Eq. def-grad): det F_1 -> 1
# at second order in h_t
# ---------------------------------------------------------------------------

def test_detF_divergence_free_second_order():
    n = (32, 32)
    X = synth.coords(n)
    vstar = 0.5 * np.stack([np.sin(X[1]) * np.cos(X[0]), -np.sin(X[0]) * np.cos(X[1])])[None]
    errs = [np.abs(O.Problem(n, nt).detF(vstar) - 1).max() for nt in (16, 32, 64, 128)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)
    assert errs[-1] < 3e-6


# ---------------------------------------------------------------------------
# Solve (Alg. 1 with Eq. termination-criterion-ksm and Armijo line search):
# the smooth 32^2 workload converges in a handful of Gauss-Newton steps
# without backtracking, as Tab. 5.3 reports for the smooth problem.
# ---------------------------------------------------------------------------

def test_solve_smooth_problem():
    c = synth.sinusoid_2d()
    P = O.Problem(c["n"], c["n_t"], beta=c["beta"], reg=c["reg"])
    mR = P.state(c["v_true"], c["mT"])[-1]
    v, rep = P.solve(c["mT"], mR, grad_rtol=1e-2)
    assert rep["status"] == 0
    assert rep["g_inf"] <= 1e-2 * rep["g0_inf"]
    assert 2 <= rep["outer"] <= 8
    assert rep["ls_trials"] == rep["outer"]  # alpha = 1 accepted every time
    assert rep["J"] < 0.5 * rep["J0"]


# ---------------------------------------------------------------------------
# Full Newton Hessian (Eq. sec-order-opt-cond, Sec. 3.2.1): equals Gauss-Newton
# where lambda vanishes, and is the derivative of the (trapezoid) gradient up
# to O(h_t^2), while Gauss-Newton keeps an O(1) gap there.
# ---------------------------------------------------------------------------

def newton_setup(nt):
    c = synth.sinusoid_2d()
    P = O.Problem(c["n"], nt, 1, c["beta"], 1, False)
    mR = O.Problem(c["n"], 16).state(c["v_true"], c["mT"])[-1]
    return c, P, mR


def test_newton_equals_gauss_newton_at_the_inverse_crime_point():
    c = synth.stokes_3d(16, n_t=6, n_c=2)
    P = O.Problem(c["n"], 6, 2, c["beta"], 1, True)
    mR = P.state(c["v_true"], c["mT"])[-1]  # lambda = 0 at v_true
    Hn = P.hessvec_newton(c["v_true"], c["mT"], mR, c["vt"])
    Hg = P.hessvec(c["v_true"], c["mT"], c["vt"])
    assert np.abs(Hn - Hg).max() <= 1e-14 * np.abs(Hg).max()


def test_newton_is_the_gradient_derivative_at_second_order():
    errs_n, errs_g = [], []
    for nt in (16, 32, 64):
        c, P, mR = newton_setup(nt)
        v = 0.5 * c["v_true"]
        eps = 1e-5
        fd = (P.gradient(v + eps * c["vt"], c["mT"], mR)[0] - P.gradient(v - eps * c["vt"], c["mT"], mR)[0]) / (2 * eps)
        errs_n.append(np.linalg.norm(P.hessvec_newton(v, c["mT"], mR, c["vt"]) - fd) / np.linalg.norm(fd))
        errs_g.append(np.linalg.norm(P.hessvec(v, c["mT"], c["vt"]) - fd) / np.linalg.norm(fd))
    rates = np.log2(np.array(errs_n[:-1]) / np.array(errs_n[1:]))
    assert np.all(np.abs(rates - 2) < 0.2), (errs_n, rates)
    assert errs_n[-1] < 1e-5
    assert min(errs_g) > 1e3 * errs_n[-1]  # the lambda terms are not negligible here


def test_newton_solve_reaches_the_gauss_newton_minimiser():
    # N-PCG (Sec. 4) and GN-PCG converge to the same stationary point (the
    # gradient is pinned independently against finite differences of the
    # objective); with the exact second derivative, no more outer iterations
    c, P, mR = newton_setup(8)
    vg, rg = P.solve(c["mT"], mR, grad_rtol=1e-6, max_outer=30)
    vn, rn = P.solve(c["mT"], mR, grad_rtol=1e-6, max_outer=30, newton=True)
    assert rg["status"] == 0 and rn["status"] == 0
    assert rn["g_inf"] <= 1e-6 * rn["g0_inf"]
    assert np.linalg.norm(vn - vg) <= 1e-5 * np.linalg.norm(vg)
    assert rn["outer"] <= rg["outer"]
    assert abs(rn["J"] - rg["J"]) <= 1e-9 * rg["J"]


# ---------------------------------------------------------------------------
# Picard / preconditioned gradient descent (Eq. picard, App. C), the step
# memory alpha~ and the C1-C5 stopping set (Sec. 3.3.5, Eq. stopping-criteria)
# ---------------------------------------------------------------------------

def numpy_picard_first_iterate(P, mT, mR):
    # Eq. picard at v = 0 for H1, no Stokes, n_c = 1: the state is m_T at all
    # times and the adjoint is m_R - m_T, so f = (m_R - m_T) grad m_T and
    # v_1 = -(beta A)^{-1} f, with A = -Lap and its k = 0 mode scaled by one
    n = P.n
    ks = [np.fft.fftfreq(k, 1.0 / k) for k in n]
    K = np.meshgrid(*ks, indexing="ij")
    mh = np.fft.fftn(mT)
    f = []
    for i, k in enumerate(n):
        kt = K[i].copy()
        kt[np.abs(kt) == k // 2] = 0  # Nyquist-masked first derivative
        f.append((mR - mT) * np.real(np.fft.ifftn(1j * kt * mh)))
    k2 = sum(k * k for k in K)
    a = P.beta * k2
    a[k2 == 0] = 1.0
    return np.stack([-np.real(np.fft.ifftn(np.fft.fftn(fi) / a)) for fi in f])[None]


def picard_problem():
    c = synth.sinusoid_2d(32)
    P = O.Problem(c["n"], 8, 1, c["beta"], 1, False)
    mR = O.Problem(c["n"], 16).state(c["v_true"], c["mT"])[-1]
    return c, P, mR


def test_picard_first_step_is_the_picard_iterate():
    c, P, mR = picard_problem()
    v1, rep = P.solve(c["mT"], mR, max_outer=1, picard=True, step_memory=False)
    ref = numpy_picard_first_iterate(P, c["mT"], mR)
    alpha = 0.5 ** (rep["ls_trials"] - 1)  # Armijo halvings from alpha = 1
    assert rep["outer"] == 1 and rep["pcg_iters"] == 0
    assert np.abs(v1 - alpha * ref).max() <= 1e-12 * np.abs(ref).max()


def test_picard_step_memory_rule():
    # alpha~ doubles after a full step and is scaled by the accepted alpha otherwise
    c, P, mR = picard_problem()
    amem, trials = 1.0, 0
    for k in range(1, 9):
        _, rep = P.solve(c["mT"], mR, max_outer=k, picard=True)
        t = rep["ls_trials"] - trials
        trials = rep["ls_trials"]
        amem = 2 * amem if t == 1 else amem * 0.5 ** (t - 1)
        assert rep["alpha_mem"] == amem, k


def test_picard_reaches_the_newton_krylov_minimiser():
    c, P, mR = picard_problem()
    vg, rg = P.solve(c["mT"], mR, grad_rtol=1e-8, max_outer=30)
    vp, rp = P.solve(c["mT"], mR, grad_rtol=1e-5, max_outer=2000, picard=True)
    assert rp["status"] == 0 and rp["g_inf"] <= 1e-5 * rp["g0_inf"]
    assert np.linalg.norm(vp - vg) <= 2e-4 * np.linalg.norm(vg)  # linear convergence: ~10x the gradient tolerance
    assert rp["outer"] > 3 * rg["outer"]  # first order: many more outer iterations (Sec. 5.2)


def test_stopping_set_c1_to_c5():
    c, P, mR = picard_problem()
    for kw in (dict(), dict(picard=True), dict(newton=True)):
        v, rep = P.solve(c["mT"], mR, stop_rule=1, tau_J=1e-3, max_outer=100, **kw)
        assert rep["status"] == 0
        tau, J0 = 1e-3, rep["J0"]
        flags = ((rep["J_prev"] - rep["J"] < tau * (1 + J0)) * 1 + (rep["dv_inf"] < tau ** 0.5 * (1 + rep["v_inf"])) * 2
                 + (rep["g_inf"] < tau ** (1 / 3) * (1 + J0)) * 4 + (rep["g_inf"] < 1e3 * np.finfo(float).eps) * 8)
        assert rep["stop_flags"] == flags and (flags & 7) == 7, kw
        # one iterate earlier the set did not hold: capped there, C5 stops the solve
        K = rep["outer"]
        _, r2 = P.solve(c["mT"], mR, stop_rule=1, tau_J=1e-3, max_outer=K - 2, **kw)
        assert r2["status"] == 8 and r2["outer"] == K - 1 and (r2["stop_flags"] & 7) != 7 and r2["stop_flags"] & 16


def test_stopping_set_c4_at_a_stationary_start():
    # m_R = m_T and v_0 = 0: the gradient vanishes identically, C4 stops at k = 0
    c, P, _ = picard_problem()
    v, rep = P.solve(c["mT"], c["mT"], stop_rule=1)
    assert rep["status"] == 0 and rep["outer"] == 0 and rep["stop_flags"] & 8 and rep["g_inf"] == 0.0


# ---------------------------------------------------------------------------
# Presmoothing (Sec. 3.3.5 "Presmoothing"): the periodic Gaussian
# ---------------------------------------------------------------------------

def test_smoothing_single_modes_and_semigroup():
    n = (32, 16)
    P = O.Problem(n, 2)
    X = synth.coords(n)
    sigma = 2 * np.pi / 16
    for k in [(1, 0), (3, 2), (16, 8), (5, 8)]:  # includes both Nyquist indices
        m = np.cos(k[0] * X[0] + k[1] * X[1])
        ref = np.exp(-0.5 * sigma ** 2 * (k[0] ** 2 + k[1] ** 2)) * m
        assert np.abs(P.smooth(m, sigma) - ref).max() < 1e-13
    m = rng(60).standard_normal(n)
    a, b = 0.11, 0.23
    assert np.abs(P.smooth(P.smooth(m, a), b) - P.smooth(m, np.hypot(a, b))).max() < 1e-13
    assert abs(P.smooth(m, 0.4).mean() - m.mean()) < 1e-15
    assert np.abs(P.smooth(m, 0.0) - m).max() < 1e-13


def test_smoothing_a_point_mass_gives_the_periodised_gaussian():
    n = (32, 32)
    P = O.Problem(n, 2)
    h = hd(n)
    sigma = 0.6  # exp(-sigma^2 n^2 / 8) ~ 1e-20: the truncated spectrum is exact
    e = np.zeros(n)
    e[5, 9] = 1.0 / h  # unit mass
    X = synth.coords(n)
    x0 = (2 * np.pi * 5 / 32, 2 * np.pi * 9 / 32)
    G = np.zeros(n)
    for m1 in range(-3, 4):
        for m2 in range(-3, 4):
            r2 = (X[0] - x0[0] + 2 * np.pi * m1) ** 2 + (X[1] - x0[1] + 2 * np.pi * m2) ** 2
            G += np.exp(-r2 / (2 * sigma ** 2)) / (2 * np.pi * sigma ** 2)
    assert np.abs(P.smooth(e, sigma) - G).max() < 1e-12 * G.max()


# ---------------------------------------------------------------------------
# Deformation map (App. D Eq. displacement) and the deformation gradient /
# grid-angle measure (App. D Eq. def-grad, Sec. 3.3.5 "Regularization")
# ---------------------------------------------------------------------------

def trig_eval(field, pts):
    # exact evaluation of the trigonometric interpolant of `field` at arbitrary points
    n = field.shape
    F = np.fft.fftn(field) / field.size
    ks = np.meshgrid(*[np.fft.fftfreq(k, 1.0 / k) for k in n], indexing="ij")
    out = np.zeros(pts[0].size, dtype=complex)
    flat = [p.ravel() for p in pts]
    for idx in zip(*np.nonzero(np.abs(F) > 1e-15)):
        phase = sum(ks[a][idx] * flat[a] for a in range(len(n)))
        out += F[idx] * np.exp(1j * phase)
    return out.real.reshape(pts[0].shape)


def test_displacement_of_a_constant_velocity():
    n = (16, 16)
    P = O.Problem(n, 5)
    v = np.zeros((1, 2) + n)
    v[0, 0], v[0, 1] = 0.3, -0.7
    u = P.displacement(v)
    assert np.abs(u[0] - 0.3).max() < 1e-14 and np.abs(u[1] + 0.7).max() < 1e-14


def test_displacement_map_pulls_back_the_template_at_second_order():
    n = (32, 32)
    r = rng(61)
    mT = synth.random_spectral_field(n, r, 3.0)  # smooth enough that the spatial error stays below 1e-7
    v = synth.velocity_field(n, r, 2, 0.4)[None]
    X = synth.coords(n)
    errs = []
    for nt in (4, 8, 16, 32):
        P = O.Problem(n, nt)
        u = P.displacement(v)
        m1 = P.state(v, mT)[-1]
        pulled = trig_eval(mT, [X[0] - u[0], X[1] - u[1]])
        errs.append(np.abs(pulled - m1).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


def test_deformation_gradient_and_grid_angle_of_a_shear():
    # v = (s sin x2, 0): F_1 = I + grad v exactly (grad v is nilpotent and
    # constant in time, and F does not vary along x1)
    n = (16, 16)
    s = 0.8
    X = synth.coords(n)
    v = np.zeros((1, 2) + n)
    v[0, 0] = s * np.sin(X[1])
    P = O.Problem(n, 7)
    F = P.defgrad(v)
    assert np.abs(F[0, 0] - 1).max() < 1e-13 and np.abs(F[1, 1] - 1).max() < 1e-13
    assert np.abs(F[1, 0]).max() < 1e-13 and np.abs(F[0, 1] - s * np.cos(X[1])).max() < 1e-13
    assert np.abs(P.detF(v) - 1).max() < 1e-13
    c = np.abs(s * np.cos(X[1])) / np.sqrt(1 + (s * np.cos(X[1])) ** 2)
    assert np.abs(P.grid_angle(v) - np.arccos(c)).max() < 1e-12
    assert np.abs(P.grid_angle(np.zeros_like(v)) - np.pi / 2).max() == 0.0


# ---------------------------------------------------------------------------
# Lanczos (Sec. 3.3.5 "Regularization"): extreme Ritz values of H and P^{-1} H
# ---------------------------------------------------------------------------

def dense_hessian(P, v, mT):
    n = int(np.prod(P.coef_shape()))
    H = np.empty((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        H[:, i] = P.hessvec(v, mT, e).ravel()
    return H


def test_lanczos_extremes_match_dense_eigenvalues():
    n = (8, 8)
    r = rng(62)
    P = O.Problem(n, 3, 1, 1e-2, 1, False, dto=True)  # symmetric discrete-adjoint Hessian
    mT = synth.random_spectral_field(n, r, 3.0)
    v = synth.velocity_field(n, r, 2, 0.3)[None]
    H = dense_hessian(P, v, mT)
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    ev = np.linalg.eigvalsh(H)
    q0 = r.standard_normal(P.coef_shape())
    a, b, ritz = P.lanczos(v, mT, q0, 60)
    assert abs(a[0] - (q0.ravel() @ H @ q0.ravel()) / (q0.ravel() @ q0.ravel())) < 1e-12 * ev[-1]
    assert abs(ritz[-1] - ev[-1]) < 1e-10 * ev[-1] and abs(ritz[0] - ev[0]) < 1e-8 * ev[-1]
    # preconditioned: the eigenvalues of P^{-1} H
    m = H.shape[0]
    Pi = np.empty((m, m))
    for i in range(m):
        e = np.zeros(m)
        e[i] = 1.0
        Pi[:, i] = P.precond(e.reshape(P.coef_shape())).ravel()
    evp = np.sort(np.linalg.eigvals(Pi @ H).real)
    _, _, rp = P.lanczos(v, mT, q0, 60, precond=True)
    assert abs(rp[-1] - evp[-1]) < 1e-10 * evp[-1] and abs(rp[0] - evp[0]) < 1e-8 * evp[-1]


def test_lanczos_reproduces_the_printed_beta_1e6_maxima():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "eigen_beta1e6_64.txt")) if not ln.startswith("#")]
    c = synth.blobs_2d(64, n_t=8)
    for reg_name, stokes, value, digits in rows:
        P = O.Problem((64, 64), 8, beta=1e6, reg=1 if reg_name == "H1" else 2, stokes=bool(int(stokes)))
        q0 = rng(63).standard_normal(P.coef_shape())
        _, _, ritz = P.lanczos(c["v_true"], c["mT"], q0, 40)
        assert float(f"{ritz[-1]:.{int(digits) - 1}e}") == float(value), (reg_name, ritz[-1])


# ---------------------------------------------------------------------------
# Beta continuation (Sec. 3.3.5 "Regularization"): the trace follows the rule
# ---------------------------------------------------------------------------

def continuation_problem():
    c = synth.sinusoid_2d(32)
    P = O.Problem(c["n"], 8, 1, 1.0, 1, False)
    mR = O.Problem(c["n"], 16).state(2 * c["v_true"], c["mT"])[-1]
    return c, P, mR


def check_trace(r, eps_F, beta0=1.0, beta_rtol=0.05):
    tb, ok = r["trace_beta"], r["trace_ok"]
    assert tb[0] == beta0
    k = 0
    while k + 1 < len(tb) and ok[k]:  # reduction by one order of magnitude while accepted
        assert np.isclose(tb[k + 1], tb[k] / 10, rtol=1e-15)
        k += 1
    good, bad = tb[k - 1], tb[k]  # then bisection between last accepted and breaching beta
    assert r["beta_breach"] == bad
    for j in range(k + 1, len(tb)):
        assert np.isclose(tb[j], 0.5 * (good + bad), rtol=1e-15)
        if ok[j]:
            good = tb[j]
        else:
            bad = tb[j]
    assert abs(0.5 * (good + bad) - tb[-1]) < beta_rtol * r["beta_breach"]  # stop: change below 5%
    assert r["beta"] == good == min(b for b, o in zip(tb, ok) if o)
    for d, o in zip(r["trace_detF"], ok):
        assert (d >= eps_F) == bool(o)


def test_continuation_follows_the_beta_rule():
    c, P, mR = continuation_problem()
    v, r = O.continuation(P, c["mT"], mR, eps_F=0.8, max_outer=20, pcg_maxit=100)
    assert r["found"] == 1 and r["stop"] == 0
    check_trace(r, 0.8)
    # the returned v is the accepted solution: solving at its beta from it changes nothing
    Pb = O.Problem(c["n"], 8, 1, r["beta"], 1, False)
    assert abs(Pb.detF(v).min() - r["detF_min"]) < 1e-14


def test_continuation_without_a_feasible_beta_and_the_grid_angle_bound():
    c, P, mR = continuation_problem()
    _, r = O.continuation(P, c["mT"], mR, eps_F=0.99, max_outer=20, pcg_maxit=100)
    assert r["found"] == 0 and r["stop"] == 3 and r["solves"] == 1 and r["beta_breach"] == 1.0
    # the grid-angle bound alone (eps_F = 0) decides acceptance
    _, r = O.continuation(P, c["mT"], mR, eps_F=0.0, eps_theta=1.2, max_outer=20, pcg_maxit=100)
    assert r["found"] == 1
    for a, o in zip(r["trace_angle"], r["trace_ok"]):
        assert (a >= 1.2) == bool(o)


def test_continuation_raises_n_t_to_meet_the_cfl_target():
    c, P, mR = continuation_problem()
    v, r = O.continuation(P, c["mT"], mR, eps_F=0.8, cfl_target=0.05, max_outer=20, pcg_maxit=100)
    assert r["n_t"] > 8
    Pn = O.Problem(c["n"], r["n_t"], 1, r["beta"], 1, False)
    assert Pn.cfl(v) <= 0.05


# ---------------------------------------------------------------------------
# CFL number (Sec. 3.3.1: h_t max_j max_i ||v_i(t_j)||_inf / h_x^i over the
# time nodes t_j), against values worked out by hand
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [(16, 32), (8, 16, 32)])
def test_cfl_of_constant_velocities_by_hand(n):
    d, n_t = len(n), 8
    c = np.array([0.3, -0.7, 0.45])[:d]
    v = np.ones((1, d) + n) * c.reshape((1, d) + (1,) * d)
    # h_t |c_i| / (2 pi / n_i), largest over the axes: 0.7 * n_1 / (2 pi n_t)
    expect = max(abs(c[i]) * n[i] / (2 * np.pi) for i in range(d)) / n_t
    assert abs(O.Problem(n, n_t).cfl(v) - expect) <= 1e-15 * expect


def test_cfl_of_a_chebyshev_velocity_by_hand():
    # v(t) = c1 + T_1(2t - 1) c2 + T_2(2t - 1) c3 with constant fields: on the
    # nodes t = 0 and t = 1, T_1 = -1 / +1 and T_2 = 1, so the largest speed of
    # component i is max(|c1 - c2 + c3|, |c1 + c2 + c3|) = |c1 + c3| + |c2|
    # (the middle node t = 1/2 gives |c1 - c3|, smaller here)
    n, n_t = (16, 8), 4
    c1, c2, c3 = np.array([0.2, -0.1]), np.array([0.05, 0.3]), np.array([0.1, 0.02])
    v = np.stack([np.ones((2,) + n) * c.reshape(2, 1, 1) for c in (c1, c2, c3)])
    speed = np.abs(c1 + c3) + np.abs(c2)
    expect = max(speed[i] * n[i] / (2 * np.pi) for i in range(2)) / n_t
    assert abs(O.Problem(n, n_t, n_c=3).cfl(v) - expect) <= 1e-15 * expect
    # a non-constant field: v_1 = a sin(x_2) reaches |a| on the node x_2 = pi/2
    # (n_2 a multiple of 4), v_2 = 0
    X = synth.coords(n)
    a = -0.35
    w = np.stack([a * np.sin(X[1]), np.zeros(n)])[None]
    assert abs(O.Problem(n, n_t).cfl(w) - abs(a) * n[0] / (2 * np.pi) / n_t) <= 1e-15


# ---------------------------------------------------------------------------
# det F_1 on a refined grid (App. D Eq. def-grad): trigonometric interpolation
# of the velocity onto the finer grid, then the same F-equation solve there
# ---------------------------------------------------------------------------

def test_trig_interp_reproduces_trigonometric_polynomials():
    # modes below Nyquist are kept exactly; the Nyquist mode cos(n x / 2),
    # sampled as (-1)^j, is continued as the cosine itself
    n, nf = (8, 16), (32, 64)
    X = synth.coords(n)
    Xf = synth.coords(nf)
    u = 0.3 + np.sin(X[0]) * np.cos(3 * X[1]) + 0.5 * np.cos(2 * X[0] - 5 * X[1]) + 0.25 * np.cos(4 * X[0])
    uf = 0.3 + np.sin(Xf[0]) * np.cos(3 * Xf[1]) + 0.5 * np.cos(2 * Xf[0] - 5 * Xf[1]) + 0.25 * np.cos(4 * Xf[0])
    assert np.abs(O.trig_interp(u, nf) - uf).max() < 1e-14
    # a field with Nyquist content on both axes, in 3D
    n3, nf3 = (4, 8, 8), (8, 16, 32)
    Y = synth.coords(n3)
    Yf = synth.coords(nf3)
    w = np.cos(2 * Y[0]) * np.cos(4 * Y[2]) + np.sin(Y[1] + Y[2])
    wf = np.cos(2 * Yf[0]) * np.cos(4 * Yf[2]) + np.sin(Yf[1] + Yf[2])
    assert np.abs(O.trig_interp(w, nf3) - wf).max() < 1e-14
    # dropping the Nyquist modes keeps only what the masked derivatives see
    assert np.abs(O.trig_interp(w, nf3, "drop") - np.sin(Yf[1] + Yf[2])).max() < 1e-14
    assert np.abs(O.trig_interp(u, nf, "drop") - (uf - 0.25 * np.cos(4 * Xf[0]))).max() < 1e-14


def test_refined_detF_of_a_divergence_free_nyquist_field():
    # v = (cos(n x2 / 2), 0) is a Nyquist mode: divergence-free, with zero masked
    # derivatives, so F_1 = I on the coarse grid; the refined evaluation drops
    # the mode and must give det F_1 = 1 as well
    n = (16, 16)
    X = synth.coords(n)
    v = np.zeros((1, 2) + n)
    v[0, 0] = 0.3 * np.cos(8 * X[1])
    assert np.abs(O.Problem(n, 4).detF(v) - 1).max() < 1e-14
    assert np.abs(O.Problem(n, 4).detF_refined(v, 2) - 1).max() < 1e-14


def test_refined_detF_of_a_shear_is_exact():
    n = (16, 16)
    X = synth.coords(n)
    v = np.zeros((1, 2) + n)
    v[0, 0] = 0.8 * np.sin(X[1])
    for r in (2, 4):
        assert np.abs(O.Problem(n, 5).detF_refined(v, r) - 1).max() < 1e-13


def test_refined_detF_converges_at_second_order():
    # a divergence-free velocity with modes up to |k| = 6 on 16^2: on the coarse
    # grid det F_1 - 1 stalls at a spatial error; four times finer it falls by
    # about 4 per doubling of n_t (Heun is second order) and ends far below
    n = (16, 16)
    v = synth.velocity_field(n, rng(3), 6, 0.4, divergence_free=True)[None]
    coarse, fine = [], []
    for n_t in (16, 32, 64):
        P = O.Problem(n, n_t)
        coarse.append(np.abs(P.detF(v) - 1).max())
        fine.append(np.abs(P.detF_refined(v, 4) - 1).max())
    assert abs(coarse[2] / coarse[0] - 1) < 0.05
    for a, b in zip(fine, fine[1:]):
        assert 3.3 < a / b < 4.7, fine
    assert fine[2] < coarse[2] / 100
