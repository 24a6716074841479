"""Stochastic DIP training harness around the operator (StoDIP Algorithm 1).

The generator is a plain 3D convolutional U-Net run by PyTorch/cuDNN (the
paper's networks are library convolutions, not part of this library's
kernels).  What the harness adds around the library's data-consistency loss:

- `UNet3D`: 4 levels, base 32 channels doubling per level (32, 64, 128, 256),
  two 3x3x3 convolutions with LeakyReLU per level, average-pool down,
  2x2x2 transposed-convolution up (deterministic under cuDNN's deterministic
  mode, unlike interpolation's backward) with skip concatenation, a 1x1x1
  output convolution; 2K real
  input channels (the noise z ~ U(0, 0.1)) and 2K real outputs, read as the K
  complex TSMI channels (Sec. 3: the complex TSMI as 2K real channels).
- `DipRunner`: Algorithm 1's loop.  Each epoch draws a random permutation of
  the C coils and walks it in minibatches of B (the last one may be smaller);
  each iteration computes x = G(z), the loss sum_{c in batch} ||A_c x - y_c||^2
  (+ lambda TV(x) when lambda > 0, Algorithm 1 line 6), backpropagates through
  the library's adjoint and the U-Net, and takes an Adam step (Sec. 3: Adam).
- `state_dict` / `load_state_dict`: the network, the optimiser, the RNG of the
  coil draws and the position in the coil permutation, so a run resumes
  exactly where it stopped.
"""
from __future__ import annotations

import torch
import torch.nn as nn
import torch.nn.functional as F

from . import op as _op


def _block(cin: int, cout: int) -> nn.Sequential:
    return nn.Sequential(nn.Conv3d(cin, cout, 3, padding=1), nn.LeakyReLU(0.2, inplace=True),
                         nn.Conv3d(cout, cout, 3, padding=1), nn.LeakyReLU(0.2, inplace=True))


class UNet3D(nn.Module):
    """3D U-Net with len(ch) levels; spatial sizes must be divisible by 2^(levels-1)."""

    def __init__(self, cin: int, cout: int, ch=(32, 64, 128, 256)):
        super().__init__()
        self.enc = nn.ModuleList()
        c = cin
        for w in ch:
            self.enc.append(_block(c, w))
            c = w
        self.up = nn.ModuleList([nn.ConvTranspose3d(ch[i + 1], ch[i + 1], 2, stride=2) for i in range(len(ch) - 1)])
        self.dec = nn.ModuleList([_block(ch[i + 1] + ch[i], ch[i]) for i in range(len(ch) - 1)])
        self.out = nn.Conv3d(ch[0], cout, 1)

    def forward(self, z):
        skips = []
        h = z
        for i, blk in enumerate(self.enc):
            h = blk(h)
            if i < len(self.enc) - 1:
                skips.append(h)
                h = F.avg_pool3d(h, 2)
        for i in range(len(self.dec) - 1, -1, -1):
            h = self.up[i](h)
            h = self.dec[i](torch.cat([h, skips[i]], dim=1))
        return self.out(h)


def to_complex(g: torch.Tensor) -> torch.Tensor:
    """[1][2K][N1][N2][N3] real -> [K][N1][N2][N3] complex64 (channel 2k real, 2k+1 imaginary part of x_k)."""
    K = g.shape[1] // 2
    r = g[0].reshape(K, 2, *g.shape[2:])
    return torch.complex(r[:, 0], r[:, 1]).contiguous()


class DipRunner:
    """Algorithm 1 on one GPU: op (SubspaceNufft with max_batch >= B), y_meas [C][J] complex64."""

    def __init__(self, op: _op.SubspaceNufft, y_meas: torch.Tensor, net: nn.Module, z: torch.Tensor, B: int,
                 lr: float = 1e-3, lam_tv: float = 0.0, eps_tv: float = 1e-6, dcf=None, seed: int = 0):
        if B < 1 or B > op.max_batch:
            raise ValueError(f"minibatch {B} outside 1..{op.max_batch}")
        self.op, self.y, self.net, self.z, self.B = op, y_meas, net, z, int(B)
        self.lam_tv, self.eps_tv, self.dcf = float(lam_tv), float(eps_tv), dcf
        self.opt = torch.optim.Adam(net.parameters(), lr=lr)
        self.gen = torch.Generator().manual_seed(seed)
        self.epoch = 0
        self.pos = 0
        self.perm = torch.randperm(op.C, generator=self.gen)
        self.iteration = 0

    def next_coils(self) -> torch.Tensor:
        """The next minibatch of the current epoch's coil permutation (a new permutation per epoch)."""
        if self.pos >= self.op.C:
            self.epoch += 1
            self.pos = 0
            self.perm = torch.randperm(self.op.C, generator=self.gen)
        c = self.perm[self.pos:self.pos + self.B]
        self.pos += len(c)
        return c.to(torch.int32)

    def step(self) -> torch.Tensor:
        """One iteration; returns the loss as a device scalar (no host synchronisation)."""
        coils = self.next_coils().to(self.op.device)
        x = to_complex(self.net(self.z))
        loss = _op.dc_loss(self.op, x, coils, self.y, dcf=self.dcf)
        if self.lam_tv > 0:
            loss = loss + _op.tv_loss(self.op, x, self.lam_tv, self.eps_tv)
        self.opt.zero_grad(set_to_none=True)
        loss.backward()
        self.opt.step()
        self.iteration += 1
        return loss.detach()

    def state_dict(self) -> dict:
        return {"net": self.net.state_dict(), "opt": self.opt.state_dict(), "gen": self.gen.get_state(),
                "epoch": self.epoch, "pos": self.pos, "perm": self.perm.clone(), "iteration": self.iteration}

    def load_state_dict(self, s: dict) -> None:
        self.net.load_state_dict(s["net"])
        self.opt.load_state_dict(s["opt"])
        self.gen.set_state(s["gen"])
        self.epoch, self.pos, self.iteration = int(s["epoch"]), int(s["pos"]), int(s["iteration"])
        self.perm = s["perm"].clone()
