"""FP64 CPU oracle of the subspace multicoil NUFFT operator A_c and its adjoint.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this module.  The product path (the CUDA
library and its Python binding) never imports, calls or links it, and this module
imports nothing from the product package.

What it computes (StoDIP, Sec. 2, Eq. 1; Sec. 2.1, Eq. 3):
  The acquisition operator A maps a time-compressed image series (TSMI)
  x in C^{N x K} to multicoil k-space.  Sec. 2 says A "includes coil
  sensitivities, NUFFT and temporal SVD"; Eq. 3 splits A per coil, A = {A_c}.
  Written out, for a sample j of frame t_j at k-space location omega_j:

      A_c(x)[j] = sum_n exp(-i omega_j . n) * S_c[n] * sum_k V[t_j, k] * x_k[n]

  with centred voxel indices n_d = i_d - floor(N_d / 2).  Its adjoint summed
  over a coil minibatch (the gradient of sum_{c in batch} L_c, Eq. 3) is

      (A_B^H y)_k[n] = sum_b conj(S_{c_b}[n]) sum_j conj(V[t_j, k]) exp(+i omega_j . n) y_b[j].

  `nudft_forward` / `nudft_adjoint` are that definition evaluated directly.

  The paper evaluates the NUFFT with a gridding library (Sec. 2.2, Sec. 3) and
  specifies no kernel.  The reading adopted here is Kaiser-Bessel gridding
  (Jackson et al. 1991; beta from Beatty, Nishimura & Pauly 2005):
    A1 u_k = S_c * x_k / psi_hat, zero-padded into the oversampled grid at n mod M
    A2 U = unnormalised forward DFT of the grid
    A3 y[j] = sum_k V[t_j,k] sum_{W^3 taps} phi(g1-m1) phi(g2-m2) phi(g3-m3) U_k[m mod M]
  and the exact adjoint of those three steps (A5 spread with conj(V), A6
  unnormalised inverse DFT, A7 crop, divide by psi_hat, multiply conj(S_c), sum
  over the minibatch).  `gridding_forward` / `gridding_adjoint` follow these
  steps in this order with numpy FFTs and no fusion or reordering.

Decisions that floating point makes on an integer (the grid coordinate g, the
first tap of the window) are taken in float32 exactly as the CUDA path takes
them, so both sides pick the same taps; see `grid_coords` and `window_start`.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * np.pi


# ----------------------------------------------------------------------------
# Kernel, grid and deapodisation (reading of the unspecified gridding kernel)
# ----------------------------------------------------------------------------

def beatty_beta(W: int, sigma: float) -> float:
    """Kaiser-Bessel shape beta for width W and oversampling sigma.

    Beatty, Nishimura & Pauly 2005, Eq. 5: beta = pi*sqrt((W/sigma)^2 (sigma-1/2)^2 - 0.8).
    """
    return math.pi * math.sqrt((W / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8)


def is_smooth235(m: int) -> bool:
    for p in (2, 3, 5):
        while m % p == 0:
            m //= p
    return m == 1


def grid_size(n: int, sigma: float, W: int) -> int:
    """Oversampled grid length: smallest even 2,3,5-smooth integer >= max(ceil(sigma*n), 2W)."""
    m = max(int(math.ceil(sigma * n)), 2 * W)
    while m % 2 or not is_smooth235(m):
        m += 1
    return m


def kb_window(u, W: int, beta: float):
    """phi(u) = I0(beta*sqrt(1-(2u/W)^2)) / I0(beta) for |u| <= W/2, else 0 (u in grid units)."""
    u = np.asarray(u, dtype=np.float64)
    t = 1.0 - (2.0 * u / W) ** 2
    out = np.i0(beta * np.sqrt(np.maximum(t, 0.0))) / np.i0(beta)
    return np.where(np.abs(u) <= W / 2.0, out, 0.0)


def kb_ft(xi, W: int, beta: float):
    """Continuous Fourier transform of kb_window, phi_hat(xi) = int phi(u) e^{-2 pi i xi u} du.

    Closed form: W sinh(z)/(z I0(beta)) with z = sqrt(beta^2 - (pi W xi)^2); for
    imaginary z it becomes W sin(|z|)/(|z| I0(beta)); at z = 0 it is W/I0(beta).
    """
    xi = np.asarray(xi, dtype=np.float64)
    z2 = beta ** 2 - (np.pi * W * xi) ** 2
    z = np.sqrt(np.abs(z2))
    with np.errstate(invalid="ignore", divide="ignore"):
        pos = np.sinh(z) / z
        neg = np.sin(z) / z
    val = np.where(z2 > 0, pos, neg)
    val = np.where(z == 0, 1.0, val)
    return W * val / np.i0(beta)


def centred_index(nd: int) -> np.ndarray:
    """Centred voxel index n_d = i_d - floor(N_d/2) for storage offsets i_d = 0..N_d-1."""
    return np.arange(nd) - nd // 2


def deapod_1d(nd: int, md: int, W: int, beta: float) -> np.ndarray:
    """psi_hat_d(n_d) = phi_hat(n_d / M_d) for the centred indices of one axis."""
    return kb_ft(centred_index(nd) / md, W, beta)


# ----------------------------------------------------------------------------
# Grid coordinates and window start (integer decisions, float32 like the kernel)
# ----------------------------------------------------------------------------

def grid_coords(omega32: np.ndarray, M) -> np.ndarray:
    """g_d = (omega_d * M_d / (2 pi)) mod M_d, rounded to float32.

    Steps (all IEEE, no fused multiply-add): s = M_d / (2 pi) in float64;
    g = float64(omega) * s; g += M_d if g < 0; g -= M_d if g >= M_d; round to
    float32; a float32 value equal to M_d becomes 0.  Returns g32 [J][3].
    """
    om = np.asarray(omega32, dtype=np.float32).astype(np.float64)
    out = np.empty(om.shape, dtype=np.float32)
    for d in range(3):
        m = float(M[d])
        s = m / TWO_PI
        g = om[:, d] * s
        g = np.where(g < 0.0, g + m, g)
        g = np.where(g >= m, g - m, g)
        g32 = g.astype(np.float32)
        g32 = np.where(g32 >= np.float32(m), np.float32(0.0), g32)
        out[:, d] = g32
    return out


def window_start(g32: np.ndarray, W: int) -> np.ndarray:
    """First tap m0 = ceil(g - W/2), evaluated in float32 (the kernel's precision)."""
    g32 = np.asarray(g32, dtype=np.float32)
    return np.ceil(g32 - np.float32(W / 2.0)).astype(np.int64)


def tap_weights(g32: np.ndarray, W: int, beta: float):
    """Per-axis window start m0 [J][3] and weights phi(g - (m0 + a)) [J][3][W] in float64."""
    m0 = window_start(g32, W)
    a = np.arange(W)
    u = g32.astype(np.float64)[:, :, None] - (m0[:, :, None] + a[None, None, :])
    return m0, kb_window_clamped(u, W, beta)


def kb_window_clamped(u, W: int, beta: float):
    """kb_window without the support test: the taps chosen by window_start lie in
    |u| <= W/2 up to float32 rounding, so the square-root argument is clamped at 0."""
    t = 1.0 - (2.0 * np.asarray(u, dtype=np.float64) / W) ** 2
    return np.i0(beta * np.sqrt(np.maximum(t, 0.0))) / np.i0(beta)


# ----------------------------------------------------------------------------
# Problem description
# ----------------------------------------------------------------------------

class Geometry:
    """Image size, grid size, kernel parameters of one operator."""

    def __init__(self, n, W: int, sigma: float):
        self.n = tuple(int(v) for v in n)
        self.W = int(W)
        self.sigma = float(sigma)
        self.beta = beatty_beta(self.W, self.sigma)
        self.M = tuple(grid_size(v, self.sigma, self.W) for v in self.n)
        self.psi = [deapod_1d(self.n[d], self.M[d], self.W, self.beta) for d in range(3)]

    def psi_hat(self) -> np.ndarray:
        """Separable deapodisation psi_hat(n) = prod_d psi_hat_d(n_d), shape [N1][N2][N3]."""
        p1, p2, p3 = self.psi
        return p1[:, None, None] * p2[None, :, None] * p3[None, None, :]


def _as_c128(a):
    return np.asarray(a).astype(np.complex128)


# ----------------------------------------------------------------------------
# Exact operator (NUDFT), Eq. 1 / Eq. 3 written out
# ----------------------------------------------------------------------------

def _phase_factors(omega, n, sign):
    """Per-axis factors exp(sign * i * omega_d * n_d), each [J][N_d]."""
    om = np.asarray(omega, dtype=np.float64)
    return [np.exp(sign * 1j * om[:, d:d + 1] * centred_index(n[d])[None, :]) for d in range(3)]


def nudft_forward(x, S, V, omega, frame, coils, chunk: int = 512):
    """y[b, j] = sum_n exp(-i omega_j.n) S_{c_b}[n] sum_k V[t_j,k] x_k[n]  (Eq. 1, Eq. 3).

    x [K][N1][N2][N3], S [C][...], V [T][K], omega [J][3], frame [J], coils [B].
    Returns y [B][J] complex128.
    """
    x = _as_c128(x)
    S = _as_c128(S)
    V = _as_c128(V)
    K = x.shape[0]
    n = x.shape[1:]
    J = omega.shape[0]
    y = np.zeros((len(coils), J), dtype=np.complex128)
    for b, c in enumerate(coils):
        z = S[c][None] * x                                        # [K][N1][N2][N3]
        for j0 in range(0, J, chunk):
            j1 = min(J, j0 + chunk)
            e1, e2, e3 = _phase_factors(omega[j0:j1], n, -1.0)
            t = np.einsum("jc,kabc->jkab", e3, z, optimize=True)
            t = np.einsum("jb,jkab->jka", e2, t, optimize=True)
            yk = np.einsum("ja,jka->jk", e1, t, optimize=True)      # [chunk][K]
            y[b, j0:j1] = np.sum(V[frame[j0:j1]] * yk, axis=1)
    return y


def nudft_adjoint(y, S, V, omega, frame, coils, n, chunk: int = 512):
    """out_k[n] = sum_b conj(S_{c_b}[n]) sum_j conj(V[t_j,k]) exp(+i omega_j.n) y_b[j].

    Returns out [K][N1][N2][N3] complex128 (summed over the minibatch).
    """
    y = _as_c128(y)
    S = _as_c128(S)
    V = _as_c128(V)
    K = V.shape[1]
    J = omega.shape[0]
    out = np.zeros((K,) + tuple(n), dtype=np.complex128)
    for b, c in enumerate(coils):
        h = np.zeros((K,) + tuple(n), dtype=np.complex128)
        for j0 in range(0, J, chunk):
            j1 = min(J, j0 + chunk)
            e1, e2, e3 = _phase_factors(omega[j0:j1], n, +1.0)
            w = np.conj(V[frame[j0:j1]]) * y[b, j0:j1, None]      # [chunk][K]
            t = np.einsum("ja,jk->jka", e1, w, optimize=True)
            t = np.einsum("jb,jka->jkab", e2, t, optimize=True)
            h += np.einsum("jc,jkab->kabc", e3, t, optimize=True)
        out += np.conj(S[c])[None] * h
    return out


# ----------------------------------------------------------------------------
# Gridding NUFFT (the reading the CUDA path implements), steps A1..A7
# ----------------------------------------------------------------------------

def _wrap_positions(nd: int, md: int) -> np.ndarray:
    """Grid position n_d mod M_d of each centred voxel index of one axis."""
    return np.mod(centred_index(nd), md)


def _tap_indices(m0, W, M):
    """Flattened grid indices [J][W^3] of the W^3 taps (axis-3 fastest), wrapped mod M."""
    a = np.arange(W)
    i1 = np.mod(m0[:, 0:1] + a[None, :], M[0])
    i2 = np.mod(m0[:, 1:2] + a[None, :], M[1])
    i3 = np.mod(m0[:, 2:3] + a[None, :], M[2])
    flat = (i1[:, :, None, None] * M[1] + i2[:, None, :, None]) * M[2] + i3[:, None, None, :]
    return flat.reshape(len(m0), -1)


def _tap_products(w):
    """Separable tap weights phi1*phi2*phi3 [J][W^3] (axis-3 fastest)."""
    return (w[:, 0, :, None, None] * w[:, 1, None, :, None] * w[:, 2, None, None, :]).reshape(len(w), -1)


def fwd_prologue(geo: Geometry, x_k, S_c):
    """A1: u = S_c * x_k / psi_hat placed at n mod M in a zero grid [M1][M2][M3]."""
    u = _as_c128(S_c) * _as_c128(x_k) / geo.psi_hat()
    grid = np.zeros(geo.M, dtype=np.complex128)
    p = [_wrap_positions(geo.n[d], geo.M[d]) for d in range(3)]
    grid[np.ix_(p[0], p[1], p[2])] = u
    return grid


def fwd_fft(grid):
    """A2: unnormalised forward DFT, U[m] = sum_p grid[p] exp(-2 pi i m.p / M)."""
    return np.fft.fftn(grid)


def fwd_interp(geo: Geometry, U, V, g32, frame, chunk: int = 65536):
    """A3: y[j] = sum_k V[t_j,k] sum_taps phi*phi*phi * U_k[m mod M].  U is [K][M1][M2][M3]."""
    K = U.shape[0]
    J = g32.shape[0]
    Uf = U.reshape(K, -1)
    y = np.zeros(J, dtype=np.complex128)
    for j0 in range(0, J, chunk):
        j1 = min(J, j0 + chunk)
        m0, w = tap_weights(g32[j0:j1], geo.W, geo.beta)
        idx = _tap_indices(m0, geo.W, geo.M)
        wt = _tap_products(w)
        acc = np.zeros((j1 - j0, K), dtype=np.complex128)
        for k in range(K):
            acc[:, k] = np.sum(wt * Uf[k][idx], axis=1)
        y[j0:j1] = np.sum(_as_c128(V)[frame[j0:j1]] * acc, axis=1)
    return y


def adj_spread(geo: Geometry, r, V, g32, frame, chunk: int = 65536):
    """A5: H_k[m mod M] += phi*phi*phi * conj(V[t_j,k]) * r[j].  Returns H [K][M1][M2][M3]."""
    V = _as_c128(V)
    K = V.shape[1]
    G = int(np.prod(geo.M))
    H = np.zeros((K, G), dtype=np.complex128)
    r = _as_c128(r)
    for j0 in range(0, len(r), chunk):
        j1 = min(len(r), j0 + chunk)
        m0, w = tap_weights(g32[j0:j1], geo.W, geo.beta)
        idx = _tap_indices(m0, geo.W, geo.M).ravel()
        wt = _tap_products(w)
        for k in range(K):
            c = np.conj(V[frame[j0:j1], k]) * r[j0:j1]              # [chunk]
            v = (wt * c[:, None]).ravel()
            H[k] += np.bincount(idx, weights=v.real, minlength=G)
            H[k] += 1j * np.bincount(idx, weights=v.imag, minlength=G)
    return H.reshape((K,) + geo.M)


def adj_ifft(H):
    """A6: unnormalised inverse DFT, h[p] = sum_m H[m] exp(+2 pi i m.p / M)."""
    return np.fft.ifftn(H) * H.size


def adj_epilogue(geo: Geometry, h, S_c):
    """A7: crop the voxels n mod M, divide by psi_hat, multiply by conj(S_c)."""
    p = [_wrap_positions(geo.n[d], geo.M[d]) for d in range(3)]
    crop = h[np.ix_(p[0], p[1], p[2])]
    return np.conj(_as_c128(S_c)) * crop / geo.psi_hat()


def gridding_forward(geo: Geometry, x, S, V, omega, frame, coils):
    """Gridding approximation of nudft_forward: A1 -> A2 -> A3 per coil.  Returns y [B][J]."""
    K = x.shape[0]
    g32 = grid_coords(omega, geo.M)
    y = np.zeros((len(coils), omega.shape[0]), dtype=np.complex128)
    for b, c in enumerate(coils):
        U = np.stack([fwd_fft(fwd_prologue(geo, x[k], S[c])) for k in range(K)])
        y[b] = fwd_interp(geo, U, V, g32, frame)
    return y


def gridding_adjoint(geo: Geometry, y, S, V, omega, frame, coils):
    """Exact adjoint of gridding_forward summed over the minibatch: A5 -> A6 -> A7."""
    K = V.shape[1]
    g32 = grid_coords(omega, geo.M)
    out = np.zeros((K,) + geo.n, dtype=np.complex128)
    for b, c in enumerate(coils):
        H = adj_spread(geo, y[b], V, g32, frame)
        for k in range(K):
            out[k] += adj_epilogue(geo, adj_ifft(H[k]), S[c])
    return out


# ----------------------------------------------------------------------------
# Loss of Alg. 1 (DCF = 1) and its gradient
# ----------------------------------------------------------------------------

def dip_loss(forward, x, y_meas):
    """L = sum_b || y_b - A_{c_b}(x) ||^2 (Eq. 3 summed over the minibatch, DCF = 1)."""
    r = forward(x) - y_meas
    return float(np.sum(np.abs(r) ** 2))


def dip_grad(forward, adjoint, x, y_meas):
    """Gradient of dip_loss in PyTorch's convention dL/dRe + i dL/dIm = A^H (2 r)."""
    r = forward(x) - y_meas
    return adjoint(2.0 * r)
