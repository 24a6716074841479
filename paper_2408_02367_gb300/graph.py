"""CUDA-graph captured data-consistency step of StoDIP (Algorithm 1, lines 4, 5, 7).

One captured step computes, for the coil minibatch held in a device buffer,
    L = sum_b || A_{c_b}(x) - y_meas[c_b] ||^2   and   x.grad = dL/dx
with every kernel of the forward operator, the residual/loss and the adjoint
recorded once and replayed by a single graph launch.  New coil indices (and a
new x) are written into the graph's static buffers before each replay; the
library reads the indices on the device, so nothing else changes between
replays.
"""
from __future__ import annotations

import torch

from . import op as _op


class DipStepGraph:
    """Captured `dc_loss(op, x, coil_idx, y_meas).backward()` for minibatches of B coils."""

    def __init__(self, op: _op.SubspaceNufft, y_meas: torch.Tensor, x_init: torch.Tensor, B: int, warmup: int = 3):
        self.op = op
        dev = op.device
        self.x = x_init.detach().clone().contiguous().requires_grad_(True)
        self.coil = torch.zeros((B,), dtype=torch.int32, device=dev)
        self.y_meas = y_meas
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.x.grad = None
                loss = _op.dc_loss(op, self.x, self.coil, y_meas)
                loss.backward()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        self.x.grad = None
        n0 = _op.launch_count()
        with torch.cuda.graph(self.graph):
            self.loss = _op.dc_loss(op, self.x, self.coil, y_meas)
            self.loss.backward()
        self.launches_per_step = _op.launch_count() - n0
        self.grad = self.x.grad

    def step(self, coil_idx: torch.Tensor, x: torch.Tensor | None = None):
        """Replay for coils `coil_idx` (device int32 [B]); returns (loss, grad) static tensors."""
        self.coil.copy_(coil_idx, non_blocking=True)
        if x is not None:
            with torch.no_grad():
                self.x.copy_(x, non_blocking=True)
        self.graph.replay()
        return self.loss, self.grad
