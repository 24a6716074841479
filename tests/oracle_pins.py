"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each pin takes the oracle module as an argument and returns the measured error
(or a bool for exact facts), so the same pins run against the real oracle and,
in the mutation tests, against copies with a planted mistake.

What pins what:
  kb_ft_vs_quadrature     deapodisation closed form vs numerical integration of
                          the window (both branches, normalisation)
  nudft_on_grid_vs_fftn   sign, centring and axis order of the exact operator vs
                          numpy's FFT on integer-grid frequencies
  full_cartesian_gram     A^H A = Nvox I for fully sampled Cartesian k-space
                          (adjoint sign and conjugations)
  gridding_vs_nudft       gridding within the Kaiser-Bessel error floor of the
                          exact sum (every gridding step: deapod, padding, FFT,
                          taps, V contraction, S)
  subspace_permutation    V indexing [T][K] (not transposed) with a permutation V
  adjoint_identity        <A x, y> = <x, A^H y> for the gridding pair
"""
from __future__ import annotations

import numpy as np
from scipy import integrate

from paper_2408_02367_gb300 import synth


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def kb_ft_vs_quadrature(O, W=6, sigma=2.0):
    """max |closed form - quadrature| / phi_hat(0) over xi on both sides of the branch point."""
    beta = O.beatty_beta(W, sigma)
    xis = np.array([0.0, 0.05, 0.13, 0.25, 0.4, 0.5, beta / (np.pi * W) * 0.999,
                    beta / (np.pi * W) * 1.3, 1.1])
    ref = []
    for xi in xis:
        f = lambda u: float(O.kb_window(u, W, beta)) * np.cos(2.0 * np.pi * xi * u)
        v, _ = integrate.quad(f, -W / 2.0, W / 2.0, limit=200, epsabs=1e-14, epsrel=1e-13)
        ref.append(v)
    ref = np.array(ref)
    got = O.kb_ft(xis, W, beta)
    return float(np.max(np.abs(got - ref)) / abs(ref[0]))


def _toy_inputs(n, K, C, T, J, seed):
    x = synth.random_complex((K,) + tuple(n), seed)
    S = synth.random_complex((C,) + tuple(n), seed + 1)
    V = synth.random_complex((T, K), seed + 2)
    rng = np.random.default_rng(seed + 3)
    omega = rng.uniform(-np.pi, np.pi, size=(J, 3)).astype(np.float32)
    frame = np.sort(rng.integers(0, T, size=J)).astype(np.int32)
    return x, S, V, omega, frame


def nudft_on_grid_vs_fftn(O, n=(6, 5, 4)):
    """Integer-grid frequencies omega_d = 2 pi m_d / N_d: the NUDFT with K=1, V=1, S=1
    is the DFT of the centred image, numpy.fft.fftn(ifftshift(x))[m mod N]."""
    x = synth.random_complex((1,) + tuple(n), 11)
    m = np.stack(np.meshgrid(*[np.arange(-(d // 2), d - d // 2) for d in n], indexing="ij"), -1).reshape(-1, 3)
    omega = 2.0 * np.pi * m / np.array(n)          # float64: the integer frequencies exactly
    S = np.ones((1,) + tuple(n), np.complex64)
    V = np.ones((1, 1), np.complex64)
    frame = np.zeros(len(m), np.int32)
    y = O.nudft_forward(x, S, V, omega, frame, [0])[0]
    X = np.fft.fftn(np.fft.ifftshift(x[0].astype(np.complex128)))
    ref = X[tuple((m % np.array(n)).T)]
    return rel(y, ref)


def full_cartesian_gram(O, n=(4, 6, 5)):
    """With every integer frequency sampled once (S=1, V=1, K=1), A^H A x = Nvox x."""
    x = synth.random_complex((1,) + tuple(n), 12)
    m = np.stack(np.meshgrid(*[np.arange(-(d // 2), d - d // 2) for d in n], indexing="ij"), -1).reshape(-1, 3)
    omega = (2.0 * np.pi * m / np.array(n))
    S = np.ones((1,) + tuple(n), np.complex64)
    V = np.ones((1, 1), np.complex64)
    frame = np.zeros(len(m), np.int32)
    y = O.nudft_forward(x, S, V, omega, frame, [0])
    back = O.nudft_adjoint(y, S, V, omega, frame, [0], n)
    return rel(back, float(np.prod(n)) * x.astype(np.complex128))


def gridding_vs_nudft(O, W, sigma, n=(14, 12, 10), K=3, C=2, T=4, J=300, seed=21, adjoint=False):
    """Relative L2 distance of the gridding operator from the exact sum."""
    x, S, V, omega, frame = _toy_inputs(n, K, C, T, J, seed)
    x = synth.ellipsoid_phantom(n, K, seed=seed)
    geo = O.Geometry(n, W, sigma)
    coils = [1, 0]
    if not adjoint:
        return rel(O.gridding_forward(geo, x, S, V, omega, frame, coils),
                   O.nudft_forward(x, S, V, omega, frame, coils))
    y = synth.random_complex((len(coils), J), seed + 9)
    return rel(O.gridding_adjoint(geo, y, S, V, omega, frame, coils),
               O.nudft_adjoint(y, S, V, omega, frame, coils, n))


def subspace_permutation(O, W=6, sigma=2.0, n=(10, 12, 8)):
    """V = a (non-symmetric) permutation matrix, K = T: frame t sees only channel p(t).
    The gridding output of frame t must equal a single-channel NUDFT of x_{p(t)}."""
    T = K = 4
    perm = np.array([2, 0, 3, 1])
    V = np.zeros((T, K), np.complex64)
    V[np.arange(T), perm] = 1.0
    x, S, _V, omega, frame = _toy_inputs(n, K, 1, T, 200, 31)
    geo = O.Geometry(n, W, sigma)
    y = O.gridding_forward(geo, x, S, V, omega, frame, [0])[0]
    ref = np.zeros_like(y)
    one = np.ones((1, 1), np.complex64)
    for t in range(T):
        sel = frame == t
        ref[sel] = O.nudft_forward(x[perm[t]:perm[t] + 1], S, one, omega[sel],
                                   np.zeros(sel.sum(), np.int32), [0])[0]
    return rel(y, ref)


def adjoint_identity(O, W=4, sigma=1.25, n=(12, 10, 14), K=3, C=3, T=5, J=400, seed=41):
    """| <A x, y> - <x, A^H y> | / |<A x, y>| for the gridding pair (exact up to rounding)."""
    x, S, V, omega, frame = _toy_inputs(n, K, C, T, J, seed)
    geo = O.Geometry(n, W, sigma)
    coils = [2, 0]
    y = synth.random_complex((len(coils), J), seed + 5)
    Ax = O.gridding_forward(geo, x, S, V, omega, frame, coils)
    AHy = O.gridding_adjoint(geo, y, S, V, omega, frame, coils)
    lhs = np.vdot(y, Ax)
    rhs = np.vdot(AHy, x.astype(np.complex128))
    return float(abs(lhs - rhs) / abs(lhs))
