"""Reconstruction building blocks on top of the operator (StoDIP Sec. 2, Eq. 2;
Sec. 2.2, "Initialisation of x^(0)").

- `dcf_operator` / `dcf_pipe_menon`: the density compensation of Eq. 2.  The
  paper uses a DCF as preconditioner without saying how it is obtained; the
  reading here is the iterative estimate of Pipe & Menon 1999,
  w <- w / (Phi Phi^H w), with Phi the gridding interpolator of the operator
  (K = 1, V = 1), i.e. `sdp_gram_samples`.
- `svd_mrf_init`: the SVD-MRF initialiser with a scaling factor,
  x0 = alpha sum_c A_c^H (DCF y_c) with alpha minimising
  sum_c || sqrt(DCF) (alpha A_c x0 - y_c) ||^2.
- `cg_normal`: the low-rank conjugate-gradient initialiser, CG on
  (sum_c A_c^H DCF A_c + lam I) x = sum_c A_c^H DCF y_c (lam > 0 gives the
  Tikhonov-regularised variant).

The operator applications run in the library's kernels; the scalar and
vector updates of the iterations are torch glue on the device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import op as _op


def dcf_operator(omega, n, width, oversamp, max_batch=1, device="cuda"):
    """Plan of the bare interpolator: K = 1, V = 1, one frame, one coil map of ones."""
    J = omega.shape[0]
    V = np.ones((1, 1), np.complex64)
    S = np.ones((1,) + tuple(n), np.complex64)
    return _op.make_operator(omega, np.zeros(J, np.int32), n, width, oversamp, V, S, max_batch, device=device)


def dcf_pipe_menon(op_dcf: _op.SubspaceNufft, iters: int = 10) -> torch.Tensor:
    """w_{i+1} = w_i / Re(Phi Phi^H w_i), starting from w_0 = 1; returns float32 [J]."""
    w = torch.ones((1, op_dcf.J), dtype=torch.complex64, device=op_dcf.device)
    for _ in range(iters):
        d = op_dcf.gram_samples(w)
        w = (w.real / d.real).to(torch.complex64)
    return w.real[0].contiguous()


def _coil_batches(C: int, B: int, device):
    return [torch.arange(c0, min(C, c0 + B), dtype=torch.int32, device=device) for c0 in range(0, C, B)]


def normal_apply(op: _op.SubspaceNufft, v: torch.Tensor, dcf=None, lam: float = 0.0) -> torch.Tensor:
    """sum_c A_c^H (DCF A_c v) + lam v over all C coils, in minibatches of max_batch."""
    out = torch.zeros_like(v)
    for ci in _coil_batches(op.C, op.max_batch, op.device):
        y = op.forward(v, ci)
        if dcf is not None:
            y = y * dcf[None, :]
        op.adjoint(y, ci, out=out, accumulate=True)
    if lam:
        out += lam * v
    return out


def adjoint_all(op: _op.SubspaceNufft, y_all: torch.Tensor, dcf=None) -> torch.Tensor:
    """sum_c A_c^H (DCF y_c) for y_all [C][J]."""
    out = torch.zeros((op.K,) + op.n, dtype=torch.complex64, device=op.device)
    for ci in _coil_batches(op.C, op.max_batch, op.device):
        y = y_all[ci.long()]
        if dcf is not None:
            y = y * dcf[None, :]
        op.adjoint(y.contiguous(), ci, out=out, accumulate=True)
    return out


def svd_mrf_init(op: _op.SubspaceNufft, y_all: torch.Tensor, dcf=None) -> torch.Tensor:
    """x0 = alpha A^H(DCF y) with alpha = Re<A x1, DCF y> / <A x1, DCF A x1>, x1 = A^H(DCF y)."""
    x1 = adjoint_all(op, y_all, dcf)
    num = torch.zeros((), dtype=torch.float64, device=op.device)
    den = torch.zeros((), dtype=torch.float64, device=op.device)
    for ci in _coil_batches(op.C, op.max_batch, op.device):
        ax = op.forward(x1, ci).to(torch.complex128)
        yc = y_all[ci.long()].to(torch.complex128)
        w = dcf.double()[None, :] if dcf is not None else 1.0
        num += torch.real(torch.sum(torch.conj(ax) * w * yc))
        den += torch.sum(w * torch.abs(ax) ** 2)
    return ((num / den).to(torch.float32) * x1).contiguous()


def cg_normal(op: _op.SubspaceNufft, y_all: torch.Tensor, dcf=None, x0=None, iters: int = 10, lam: float = 0.0):
    """Conjugate gradients on (sum_c A_c^H DCF A_c + lam I) x = sum_c A_c^H DCF y_c.

    Returns (x, residual norms ||r_i|| for i = 0..iters)."""
    b = adjoint_all(op, y_all, dcf)
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    r = b - normal_apply(op, x, dcf, lam) if x0 is not None else b.clone()
    p = r.clone()
    rs = torch.real(torch.vdot(r.flatten().to(torch.complex128), r.flatten().to(torch.complex128)))
    hist = [float(rs.sqrt())]
    for _ in range(iters):
        Np = normal_apply(op, p, dcf, lam)
        pNp = torch.real(torch.vdot(p.flatten().to(torch.complex128), Np.flatten().to(torch.complex128)))
        alpha = (rs / pNp).to(torch.float32)
        x = x + alpha * p
        r = r - alpha * Np
        rs_new = torch.real(torch.vdot(r.flatten().to(torch.complex128), r.flatten().to(torch.complex128)))
        p = r + (rs_new / rs).to(torch.float32) * p
        rs = rs_new
        hist.append(float(rs.sqrt()))
    return x, hist
