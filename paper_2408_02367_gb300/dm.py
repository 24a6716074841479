"""Dictionary matching of the reconstructed TSMI (StoDIP Sec. 2 after Eq. 1):
idx_v = argmax_p |d_p^H x_v| / ||d_p||, PD_v = d_idx^H x_v / ||d_idx||^2, and
(T1, T2) of the matched atom.  A thin binding of include/stodip_dm.h: every
step runs in the library's kernels (a tcgen05 GEMM with a fused chunk-argmax
epilogue, then a float32 refine pass); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes

import torch

from .op import SdpError, _check, _dev_ptr, _require, _stream_ptr, lib


class DictionaryMatcher:
    """atoms: complex64 [P][K] (device); params: optional float32 [P][2] (T1, T2) (device);
    max_vox: the largest number of voxels a `match` call takes."""

    def __init__(self, atoms: torch.Tensor, max_vox: int, params: torch.Tensor | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("DictionaryMatcher needs a CUDA device (no CPU fallback)")
        self.device = atoms.device
        if self.device.type != "cuda":
            raise ValueError("atoms must be a CUDA tensor")
        if atoms.dim() != 2:
            raise ValueError("atoms must be [P][K]")
        self.P, self.K = int(atoms.shape[0]), int(atoms.shape[1])
        _require(atoms, "atoms", torch.complex64, self.device)
        if params is not None:
            _require(params, "params", torch.float32, self.device, (self.P, 2))
        self.max_vox = int(max_vox)
        self.has_params = params is not None
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().sdp_dm_create(ctypes.byref(self._h), _dev_ptr(atoms),
                                       _dev_ptr(params) if params is not None else None, self.P, self.K,
                                       self.max_vox, _stream_ptr(self.device)), "sdp_dm_create")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().sdp_dm_destroy(h)
            except Exception:
                pass
            self._h = ctypes.c_void_p()

    def match(self, x: torch.Tensor, out=None, qmap: bool = False):
        """x: complex64 [K][...] TSMI.  Returns (idx int32, PD complex64[, (T1, T2) float32 [..., 2]])
        shaped like x's voxel axes."""
        _require(x, "x", torch.complex64, self.device)
        if x.shape[0] != self.K:
            raise ValueError(f"x must have {self.K} channels, got {x.shape[0]}")
        vshape = tuple(x.shape[1:])
        nvox = int(x[0].numel())
        if qmap and not self.has_params:
            raise ValueError("qmap needs the parameter table given at construction")
        if out is None:
            idx = torch.empty(vshape, dtype=torch.int32, device=self.device)
            pd = torch.empty(vshape, dtype=torch.complex64, device=self.device)
            qm = torch.empty(vshape + (2,), dtype=torch.float32, device=self.device) if qmap else None
        else:
            idx, pd, qm = out
        _check(lib().sdp_dm_match(self._h, _dev_ptr(x), nvox, _dev_ptr(idx), _dev_ptr(pd),
                                  _dev_ptr(qm) if qm is not None else None, _stream_ptr(self.device)),
               "sdp_dm_match")
        return (idx, pd, qm) if qmap else (idx, pd)

    def set_wait_test(self, withhold_tile: int = -1, timeout_ns: int = 0):
        """Test hook of the GEMM kernel's bounded waits (sdp_dm_set_wait_test): later matches use
        `timeout_ns` per wait (0: one second) and, for withhold_tile >= 0, the first CTA never copies that
        atom tile, so its wait runs out and the match reports SDP_ERR_TIMEOUT through status()."""
        _check(lib().sdp_dm_set_wait_test(self._h, int(withhold_tile), int(timeout_ns)), "sdp_dm_set_wait_test")

    def status(self) -> int:
        return int(lib().sdp_dm_status(self._h, _stream_ptr(self.device)))

    def info(self) -> dict:
        buf = (ctypes.c_int64 * 8)()
        _check(lib().sdp_dm_info(self._h, buf, 8), "sdp_dm_info")
        keys = ["P", "K", "ksteps", "atom_tiles", "max_vox", "device_bytes", "gemm_ctas", "flops_per_voxel"]
        return dict(zip(keys, [int(v) for v in buf]))


__all__ = ["DictionaryMatcher", "SdpError"]
