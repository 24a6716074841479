"""FP64 oracle of the reconstruction building blocks (test infrastructure only;
never imported by the product path).

- `dcf_pipe_menon`: density compensation for Eq. 2 (Sec. 2) by the iteration
  of Pipe & Menon 1999, w <- w / (Phi Phi^H w), with Phi the gridding
  interpolator of `nufft` (no subspace, no coil map).  The paper names a DCF
  without saying how it is computed; this is the reading adopted.
- `dc_loss_dcf` / `dc_grad_dcf`: the Eq. 2/3 loss sum_b sum_j DCF_j |r_bj|^2
  and its gradient A^H (2 DCF r) in PyTorch's convention.
- `svd_mrf_init`, `cg_normal`: the initialisers of Sec. 2.2 ("SVD-MRF with a
  scaling factor", "low rank optimisation with conjugate gradient"), written as
  the plain algorithms on the oracle operator.
"""
from __future__ import annotations

import numpy as np

from . import nufft as O


def gram_samples(geo: O.Geometry, w, omega):
    """Phi Phi^H w: spread the samples onto the grid, interpolate back (K = 1, V = 1)."""
    J = omega.shape[0]
    g32 = O.grid_coords(omega, geo.M)
    V = np.ones((1, 1))
    frame = np.zeros(J, np.int64)
    H = O.adj_spread(geo, np.asarray(w, np.complex128), V, g32, frame)
    return O.fwd_interp(geo, H, V, g32, frame)


def dcf_pipe_menon(geo: O.Geometry, omega, iters: int = 10):
    """w_0 = 1, w_{i+1} = w_i / Re(Phi Phi^H w_i)."""
    w = np.ones(omega.shape[0])
    for _ in range(iters):
        w = w / np.real(gram_samples(geo, w, omega))
    return w


def dc_loss_dcf(forward, x, y_meas, dcf):
    r = forward(x) - y_meas
    return float(np.sum(np.asarray(dcf)[None, :] * np.abs(r) ** 2))


def dc_grad_dcf(forward, adjoint, x, y_meas, dcf):
    r = forward(x) - y_meas
    return adjoint(2.0 * np.asarray(dcf)[None, :] * r)


def _all_coils(C):
    return np.arange(C)


def svd_mrf_init(geo: O.Geometry, y_all, S, V, omega, frame, dcf=None):
    """x0 = alpha A^H(DCF y), alpha = Re<A x1, DCF y> / <A x1, DCF A x1>."""
    C = S.shape[0]
    w = np.ones(omega.shape[0]) if dcf is None else np.asarray(dcf, np.float64)
    coils = _all_coils(C)
    x1 = O.gridding_adjoint(geo, w[None, :] * y_all, S, V, omega, frame, coils)
    ax = O.gridding_forward(geo, x1, S, V, omega, frame, coils)
    alpha = np.real(np.sum(np.conj(ax) * w[None, :] * y_all)) / np.sum(w[None, :] * np.abs(ax) ** 2)
    return alpha * x1


def cg_normal(geo: O.Geometry, y_all, S, V, omega, frame, dcf=None, iters: int = 10, lam: float = 0.0):
    """Conjugate gradients on (A^H DCF A + lam I) x = A^H DCF y over all coils, from x = 0."""
    C = S.shape[0]
    w = np.ones(omega.shape[0]) if dcf is None else np.asarray(dcf, np.float64)
    coils = _all_coils(C)

    def N(v):
        return O.gridding_adjoint(geo, w[None, :] * O.gridding_forward(geo, v, S, V, omega, frame, coils), S, V,
                                  omega, frame, coils) + lam * v

    b = O.gridding_adjoint(geo, w[None, :] * y_all, S, V, omega, frame, coils)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rs = np.real(np.vdot(r, r))
    hist = [float(np.sqrt(rs))]
    for _ in range(iters):
        Np = N(p)
        alpha = rs / np.real(np.vdot(p, Np))
        x = x + alpha * p
        r = r - alpha * Np
        rs_new = np.real(np.vdot(r, r))
        p = r + (rs_new / rs) * p
        rs = rs_new
        hist.append(float(np.sqrt(rs)))
    return x, hist


# ----------------------------------------------------------------------------
# Spatial total variation, Algorithm 1 line 6 (reading: isotropic, eps-smoothed,
# per channel, forward differences with a zero difference at the last index)
# ----------------------------------------------------------------------------

def _forward_diffs(x):
    """D_d x for d = 1, 2, 3 over the last three axes of x [K][N1][N2][N3]."""
    out = []
    for ax in (1, 2, 3):
        d = np.zeros_like(x)
        sl_hi = [slice(None)] * 4
        sl_lo = [slice(None)] * 4
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        d[tuple(sl_lo)] = x[tuple(sl_hi)] - x[tuple(sl_lo)]
        out.append(d)
    return out


def tv_value(x, eps):
    """sum_k sum_n sqrt(|D1 x|^2 + |D2 x|^2 + |D3 x|^2 + eps^2)."""
    x = np.asarray(x, np.complex128)
    d1, d2, d3 = _forward_diffs(x)
    return float(np.sum(np.sqrt(np.abs(d1) ** 2 + np.abs(d2) ** 2 + np.abs(d3) ** 2 + eps ** 2)))


def tv_grad(x, eps):
    """dTV/dRe + i dTV/dIm = sum_d [ D_d x(m - e_d) / s(m - e_d) - D_d x(m) / s(m) ]."""
    x = np.asarray(x, np.complex128)
    ds = _forward_diffs(x)
    s = np.sqrt(sum(np.abs(d) ** 2 for d in ds) + eps ** 2)
    g = -sum(ds) / s
    for ax, d in zip((1, 2, 3), ds):
        q = d / s
        sl_dst = [slice(None)] * 4
        sl_src = [slice(None)] * 4
        sl_dst[ax] = slice(1, None)
        sl_src[ax] = slice(0, -1)
        g[tuple(sl_dst)] += q[tuple(sl_src)]
    return g
