"""Seeded synthetic inputs shaped like the paper's registration problems.

This module only draws inputs: images, velocity coefficient fields and
Hessian directions. It holds none of the registration method's arithmetic
(no transport solve, no regulariser, no projection). The reference image m_R
is *not* produced here: it is the template transported by the true velocity,
and each side (the CUDA library, or the CPU oracle in the tests) computes it
with its own solver.

Fields live on the periodic nodal grid x_j = 2*pi*j/n per axis (Sec. 3.3.1),
row-major, last axis fastest. Velocity coefficient arrays have shape
``(n_c, d, *n)`` (Chebyshev expansion in time, Sec. 3.3.2).

Band-limited random fields are drawn as Hermitian Gaussian Fourier
coefficients (numpy's FFT synthesises them); every mode that touches an
axis's Nyquist index is zero, and so is the k = 0 mode unless asked for.
White-noise fields (independent Gaussian values per grid point) carry the
full spectrum instead, Nyquist modes included.
"""
from __future__ import annotations

import numpy as np


def coords(n):
    """Nodal coordinates, one array per axis, broadcast to the grid."""
    axes = [2 * np.pi * np.arange(k) / k for k in n]
    return np.meshgrid(*axes, indexing="ij")


def _kgrid_r(n):
    """Integer wavenumbers on numpy's rfftn layout (last axis halved)."""
    ks = []
    for a, k in enumerate(n):
        if a == len(n) - 1:
            ks.append(np.arange(k // 2 + 1))
        else:
            ks.append(np.fft.fftfreq(k, 1.0 / k))
    return np.meshgrid(*ks, indexing="ij")


def random_spectral_field(n, rng, kmax, slope=0.0, keep_mean=False):
    """Real field with Gaussian coefficients of amplitude |k|^(-slope) on 0<|k|_2<=kmax."""
    n = tuple(int(k) for k in n)
    K = _kgrid_r(n)
    kk = np.sqrt(sum(k.astype(np.float64) ** 2 for k in K))
    shape = kk.shape
    coef = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    amp = np.zeros(shape)
    mask = (kk <= kmax) & ((kk > 0) | keep_mean)
    amp[mask] = np.where(kk[mask] > 0, kk[mask], 1.0) ** (-slope)
    nyq = np.zeros(shape, dtype=bool)
    for a, k in enumerate(n):
        nyq |= np.abs(K[a]) == k // 2
    amp[nyq] = 0.0
    return np.fft.irfftn(coef * amp, s=n, axes=tuple(range(len(n))))


def white_noise(n, rng, scale=1.0):
    """Independent standard normal values per grid point times scale: every
    Fourier mode, the Nyquist modes of each axis included, is present."""
    return scale * rng.standard_normal(tuple(int(k) for k in n))


def white_noise_velocity(n, rng, n_c, max_speed):
    """n_c white-noise coefficient fields of d components each, scaled so that
    the largest point speed sum_l |v_l(x)|_2 is max_speed (a bound on the
    speed at every time, since every Chebyshev polynomial is bounded by one)."""
    n = tuple(int(k) for k in n)
    v = rng.standard_normal((n_c, len(n)) + n)
    speed = np.sqrt((v ** 2).sum(axis=1)).sum(axis=0).max()
    return v * (max_speed / speed)


def _curl_spectral(n, potentials):
    """Divergence-free field from a stream function (2D) or vector potential (3D).

    Spectral curl of band-limited potentials; all Nyquist modes are zero, so
    the discrete divergence of the result vanishes to rounding.
    """
    d = len(n)
    kvec = [np.fft.fftfreq(k, 1.0 / k) for k in n]
    K = np.meshgrid(*kvec, indexing="ij")
    if d == 2:
        P = np.fft.fftn(potentials[0])
        v = [np.real(np.fft.ifftn(1j * K[1] * P)), np.real(np.fft.ifftn(-1j * K[0] * P))]
    else:
        A = [np.fft.fftn(p) for p in potentials]
        v = [np.real(np.fft.ifftn(1j * (K[(i + 1) % 3] * A[(i + 2) % 3] - K[(i + 2) % 3] * A[(i + 1) % 3])))
             for i in range(3)]
    return np.stack(v)


def velocity_field(n, rng, kmax, max_speed, slope=1.5, divergence_free=False):
    """Random smooth velocity (d fields): coefficient amplitude |k|^-slope (power |k|^-2*slope),
    cut at |k| <= kmax, scaled so that max_x |v(x)|_2 = max_speed."""
    n = tuple(int(k) for k in n)
    d = len(n)
    if divergence_free:
        npot = 1 if d == 2 else 3
        # the curl multiplies by |k|: lower the slope of the potential by one
        pots = [random_spectral_field(n, rng, kmax, slope + 1.0) for _ in range(npot)]
        v = _curl_spectral(n, pots)
    else:
        v = np.stack([random_spectral_field(n, rng, kmax, slope) for _ in range(d)])
    speed = np.sqrt((v ** 2).sum(axis=0)).max()
    return v * (max_speed / speed)


def blobs(n, rng, count=8, sigma=(0.2, 0.5), amp=(0.2, 1.0), kcut=32):
    """Sum of periodic Gaussian blobs with a sharp spectral cut at |k|_2 <= kcut."""
    n = tuple(int(k) for k in n)
    X = coords(n)
    img = np.zeros(n)
    for _ in range(count):
        c = rng.uniform(0, 2 * np.pi, size=len(n))
        s = rng.uniform(*sigma)
        a = rng.uniform(*amp)
        r2 = np.zeros(n)
        for i, x in enumerate(X):
            dx = np.abs(x - c[i])
            dx = np.minimum(dx, 2 * np.pi - dx)  # minimum-image distance
            r2 += dx ** 2
        img += a * np.exp(-r2 / (2 * s * s))
    spec = np.fft.rfftn(img)
    K = _kgrid_r(n)
    kk = np.sqrt(sum(k.astype(np.float64) ** 2 for k in K))
    spec[kk > kcut] = 0.0
    for a, k in enumerate(n):
        spec[np.abs(K[a]) == k // 2] = 0.0
    return np.fft.irfftn(spec, s=n, axes=tuple(range(len(n))))


# ----------------------------------------------------------------------
# Workloads. Each returns a dict with the problem parameters, the template
# m_T, the true velocity coefficients v_true (n_c, d, *n) and a seeded
# Hessian direction vt of the same shape.
# ----------------------------------------------------------------------

def sinusoid_2d(n=32, seed=1001):
    """32^2, H1, beta=1e-2, n_c=1, n_t=16: m_T = (sin^2 x1 + sin^2 x2)/2 and the
    divergence-free v* = 0.5 (sin x2 cos x1, -sin x1 cos x2) plus a seeded
    perturbation on modes |k| <= 4 of max-norm 0.05."""
    rng = np.random.default_rng(seed)
    X = coords((n, n))
    mT = 0.5 * (np.sin(X[0]) ** 2 + np.sin(X[1]) ** 2)
    vstar = 0.5 * np.stack([np.sin(X[1]) * np.cos(X[0]), -np.sin(X[0]) * np.cos(X[1])])
    dv = np.stack([random_spectral_field((n, n), rng, 4.0) for _ in range(2)])
    dv *= 0.05 / np.abs(dv).max()
    vt = velocity_field((n, n), rng, 4.0, 1.0)
    return dict(name="sinusoid-32^2-H1", n=(n, n), n_t=16, n_c=1, beta=1e-2, reg=1, stokes=False,
                mT=mT, v_true=(vstar + dv)[None], vt=vt[None])


def blobs_2d(n=128, seed=1002, n_t=32):
    """128^2, H2, beta=1e-3, n_c=1, n_t=32: eight Gaussian blobs cut at |k|<=32;
    velocity spectrum ~|k|^-3, |k|<=16, max speed 0.3."""
    rng = np.random.default_rng(seed)
    mT = blobs((n, n), rng, kcut=min(32, n // 2 - 1))
    v = velocity_field((n, n), rng, min(16, n // 2 - 1), 0.3)
    vt = velocity_field((n, n), rng, min(16, n // 2 - 1), 1.0)
    return dict(name=f"blobs-{n}^2-H2", n=(n, n), n_t=n_t, n_c=1, beta=1e-3, reg=2, stokes=False,
                mT=mT, v_true=v[None], vt=vt[None])


def stokes_3d(n=64, seed=1003, n_t=32, n_c=3):
    """64^3, Stokes (H1 + Leray), beta=1e-2, n_c=3, n_t=32:
    m_T = prod sin^2 x_i + 0.1 * eta (unit-max, |k|<=8); divergence-free
    coefficient fields whose speeds add up to at most 0.3, so |v(x,t)| <= 0.3
    for every t because every Chebyshev polynomial is bounded by one on [0,1]."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    X = coords(shape)
    eta = random_spectral_field(shape, rng, 8.0)
    eta /= np.abs(eta).max()
    mT = np.sin(X[0]) ** 2 * np.sin(X[1]) ** 2 * np.sin(X[2]) ** 2 + 0.1 * eta
    weights = [0.6, 0.25, 0.15][:n_c] if n_c <= 3 else [1.0 / n_c] * n_c
    v = np.stack([velocity_field(shape, rng, min(16, n // 2 - 1), 0.3 * w, divergence_free=True)
                  for w in weights])
    vt = np.stack([velocity_field(shape, rng, min(16, n // 2 - 1), 1.0, divergence_free=True)
                   for _ in range(n_c)])
    return dict(name=f"stokes-{n}^3-H1-nc{n_c}", n=shape, n_t=n_t, n_c=n_c, beta=1e-2, reg=1, stokes=True,
                mT=mT, v_true=v, vt=vt)


def random_3d(n=256, seed=1004, n_t=64, kimg=48, kvel=8):
    """256^3, H2, beta=1e-3, n_c=1, n_t=64: unit-variance random template with
    |k|<=48; velocity |k|<=8 with max speed 0.5; direction of unit max speed."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    mT = random_spectral_field(shape, rng, float(min(kimg, n // 2 - 1)))
    mT /= mT.std()
    v = velocity_field(shape, rng, min(kvel, n // 2 - 1), 0.5)
    vt = velocity_field(shape, rng, min(kvel, n // 2 - 1), 1.0)
    return dict(name=f"random-{n}^3-H2", n=shape, n_t=n_t, n_c=1, beta=1e-3, reg=2, stokes=False,
                mT=mT, v_true=v[None], vt=vt[None])


def batch_2d(count=256, seed=5000, sizes=(64, 128, 256), ratio=(4, 2, 1), n_t=16):
    """Batch of independent 2D pairs: sizes at ratio 4:2:1 in seeded shuffled
    order, beta in {1e-2, 1e-3}, H1, n_c=1; blobs as in the 128^2 workload."""
    rng = np.random.default_rng(seed)
    tot = sum(ratio)
    counts = [int(round(count * r / tot)) for r in ratio]
    counts[0] += count - sum(counts)
    sz = np.concatenate([np.full(c, s) for c, s in zip(counts, sizes)])
    rng.shuffle(sz)
    out = []
    for s in sz:
        s = int(s)
        mT = blobs((s, s), rng, kcut=min(32, s // 2 - 1))
        v = velocity_field((s, s), rng, min(16, s // 2 - 1), 0.3)
        beta = 1e-2 if rng.random() < 0.5 else 1e-3
        out.append(dict(n=(s, s), n_t=n_t, n_c=1, beta=beta, reg=1, stokes=False, mT=mT, v_true=v[None]))
    return out
