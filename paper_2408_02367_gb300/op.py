"""Python binding of libstodip_op.so: argument marshalling only.

Every step of the operator runs in the library's CUDA kernels; this module
checks tensor shapes/dtypes/devices, passes raw device pointers and the current
CUDA stream through ctypes, and wraps the forward/adjoint pair as a
torch.autograd.Function whose backward is the library's adjoint (StoDIP
Algorithm 1: loss.backward() through A_c).  Function names mirror the C ABI of
include/stodip_op.h.

If the compiled library is missing this module raises on first use: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstodip_op.so")

SDP_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "timeout",
                5: "bounds", 6: "unsupported"}
STAGES = ["fwd_prologue_fft3", "fwd_fft2", "fwd_fft1", "interp", "spread", "adj_ifft1", "adj_ifft2",
          "adj_ifft3_epilogue", "residual_loss", "tv"]


class SdpError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: status {code} ({_lib_strerror(code)})")
        self.code = code


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64 * 3),
        ("oversamp", ctypes.c_double),
        ("width", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("T", ctypes.c_int32),
        ("C", ctypes.c_int32),
        ("J", ctypes.c_int64),
        ("max_batch", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("frame_offsets", ctypes.POINTER(ctypes.c_int64)),
        ("traj", ctypes.c_void_p),
        ("V", ctypes.c_void_p),
        ("coil_maps", ctypes.c_void_p),
    ]


class Tuning(ctypes.Structure):
    """sdp_tuning: kernel shapes of a plan (include/stodip_op.h)."""
    _fields_ = [
        ("spread_bins", ctypes.c_int32 * 3),
        ("spread_chunk", ctypes.c_int32),
        ("fft_engine", ctypes.c_int32),
        ("fft_lines", ctypes.c_int32),
        ("fft_cols", ctypes.c_int32),
        ("interp_threads", ctypes.c_int32),
        ("spread_coils", ctypes.c_int32),
        ("interp_run", ctypes.c_int32),
        ("interp_coils", ctypes.c_int32),
        ("fft_staged", ctypes.c_int32),
        ("interp_tiled", ctypes.c_int32),
    ]

    @staticmethod
    def of(d):
        """From a dict {spread_bins: (8, 4, 8), spread_chunk: 512, fft_engine: 0, fft_lines: 0, fft_cols: 0,
        interp_threads: 0, spread_coils: 0, interp_run: 0, interp_coils: 0, fft_staged: 0, interp_tiled: 0};
        missing keys take those defaults."""
        t = Tuning()
        t.spread_bins = (ctypes.c_int32 * 3)(*[int(v) for v in d.get("spread_bins", (8, 4, 8))])
        t.spread_chunk = int(d.get("spread_chunk", 512))
        t.fft_engine = int(d.get("fft_engine", 0))
        t.fft_lines = int(d.get("fft_lines", 0))
        t.fft_cols = int(d.get("fft_cols", 0))
        t.interp_threads = int(d.get("interp_threads", 0))
        t.spread_coils = int(d.get("spread_coils", 0))
        t.interp_run = int(d.get("interp_run", 0))
        t.interp_coils = int(d.get("interp_coils", 0))
        t.fft_staged = int(d.get("fft_staged", 0))
        t.interp_tiled = int(d.get("interp_tiled", 0))
        return t

    def as_dict(self):
        return {"spread_bins": tuple(int(v) for v in self.spread_bins), "spread_chunk": int(self.spread_chunk),
                "fft_engine": int(self.fft_engine), "fft_lines": int(self.fft_lines), "fft_cols": int(self.fft_cols),
                "interp_threads": int(self.interp_threads), "spread_coils": int(self.spread_coils),
                "interp_run": int(self.interp_run), "interp_coils": int(self.interp_coils),
                "fft_staged": int(self.fft_staged), "interp_tiled": int(self.interp_tiled)}


class Work(ctypes.Structure):
    _fields_ = [
        ("plan", ctypes.c_void_p),
        ("in_", ctypes.c_void_p),
        ("coil_idx", ctypes.c_void_p),
        ("B", ctypes.c_int32),
        ("accumulate", ctypes.c_int32),
        ("out", ctypes.c_void_p),
    ]


_LIB = None

EXPORTS = {
    "sdp_plan_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(PlanDesc), ctypes.c_void_p]),
    "sdp_plan_destroy": (None, [ctypes.c_void_p]),
    "sdp_plan_create_tuned": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(PlanDesc),
                                             ctypes.POINTER(Tuning), ctypes.c_void_p]),
    "sdp_plan_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Tuning)]),
    "sdp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    "sdp_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "sdp_forward_channels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_void_p]),
    "sdp_adjoint_channels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_void_p]),
    "sdp_adjoint_scaled": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "sdp_residual_loss_weighted": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                  ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p]),
    "sdp_tv_value": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "sdp_tv_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "sdp_gram_samples": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "sdp_residual_loss": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "sdp_residual_loss_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                 ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    "sdp_forward_batched": (ctypes.c_int, [ctypes.POINTER(Work), ctypes.c_int32, ctypes.c_void_p]),
    "sdp_adjoint_batched": (ctypes.c_int, [ctypes.POINTER(Work), ctypes.c_int32, ctypes.c_void_p]),
    "sdp_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sdp_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    "sdp_plan_beta": (ctypes.c_double, [ctypes.c_void_p]),
    "sdp_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "sdp_workspace_bytes_for": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int32]),
    "sdp_plan_set_wait_test": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "sdp_launch_count": (ctypes.c_int64, []),
    "sdp_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "sdp_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    "sdp_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sdp_grid_size": (ctypes.c_int64, [ctypes.c_int64, ctypes.c_double, ctypes.c_int32]),
    "sdp_kb_beta": (ctypes.c_double, [ctypes.c_int32, ctypes.c_double]),
    # dictionary matching (include/stodip_dm.h)
    "sdp_dm_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p]),
    "sdp_dm_destroy": (None, [ctypes.c_void_p]),
    "sdp_dm_match": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sdp_dm_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sdp_dm_set_wait_test": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "sdp_dm_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
}


def lib():
    """Load libstodip_op.so (built by paper_2408_02367_gb300.build) and declare its exports."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                               f"g.build()\"` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _lib_strerror(code):
    try:
        return lib().sdp_strerror(int(code)).decode()
    except Exception:
        return STATUS_NAMES.get(code, "unknown")


def _check(code, what):
    if code != SDP_OK:
        raise SdpError(code, what)


def _stream_ptr(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _require(t, name, dtype, device, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class SubspaceNufft:
    """Plan of the per-coil subspace NUFFT operator A_c and its adjoint on one GPU.

    traj      float32 [J][3] radians (device), frame_offsets int64 [T+1] (host/CPU),
    V         complex64 [T][K] (device), coil_maps complex64 [C][N1][N2][N3] (device).
    """

    def __init__(self, traj, frame_offsets, n, width, oversamp, V, coil_maps, max_batch=1, tuning=None,
                 borrow_maps=False):
        if not torch.cuda.is_available():
            raise RuntimeError("SubspaceNufft needs a CUDA device (no CPU fallback)")
        self.device = traj.device
        if self.device.type != "cuda":
            raise ValueError("traj must be a CUDA tensor")
        L = lib()
        self.n = tuple(int(v) for v in n)
        T, K = V.shape
        C = coil_maps.shape[0]
        J = traj.shape[0]
        _require(traj, "traj", torch.float32, self.device, (J, 3))
        _require(V, "V", torch.complex64, self.device, (T, K))
        _require(coil_maps, "coil_maps", torch.complex64, self.device, (C,) + self.n)
        off = np.ascontiguousarray(np.asarray(frame_offsets, dtype=np.int64))
        if off.shape != (T + 1,):
            raise ValueError("frame_offsets must have T+1 entries")
        self._off = off
        d = PlanDesc()
        d.n = (ctypes.c_int64 * 3)(*self.n)
        d.oversamp = float(oversamp)
        d.width = int(width)
        d.K, d.T, d.C, d.J = int(K), int(T), int(C), int(J)
        d.max_batch = int(max_batch)
        # SDP_FLAG_BORROW_MAPS: the plan reads the caller's coil_maps; this object keeps the tensor alive
        d.flags = 1 if borrow_maps else 0
        self._borrowed_maps = coil_maps if borrow_maps else None
        d.frame_offsets = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.traj = traj.data_ptr()
        d.V = V.data_ptr()
        d.coil_maps = coil_maps.data_ptr()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if tuning is None:
                _check(L.sdp_plan_create(ctypes.byref(h), ctypes.byref(d), _stream_ptr(self.device)),
                       "sdp_plan_create")
            else:
                t = Tuning.of(tuning)
                _check(L.sdp_plan_create_tuned(ctypes.byref(h), ctypes.byref(d), ctypes.byref(t),
                                               _stream_ptr(self.device)), "sdp_plan_create_tuned")
        self._h = h
        self.K, self.T, self.C, self.J = int(K), int(T), int(C), int(J)
        self.max_batch = int(max_batch)
        self.width = int(width)
        self.oversamp = float(oversamp)
        t = Tuning()
        _check(L.sdp_plan_tuning(self._h, ctypes.byref(t)), "sdp_plan_tuning")
        self.tuning = t.as_dict()

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sdp_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- facts --
    def info(self):
        arr = (ctypes.c_int64 * 16)()
        _check(lib().sdp_plan_info(self._h, arr, 16), "sdp_plan_info")
        keys = ["M1", "M2", "M3", "J", "K", "max_batch", "bs1", "bs2", "bs3", "nbins", "nsub", "ninc",
                "workspace_bytes", "total_bytes", "W", "C"]
        return dict(zip(keys, [int(v) for v in arr]))

    @property
    def grid(self):
        i = self.info()
        return (i["M1"], i["M2"], i["M3"])

    def workspace_bytes_for(self, max_batch):
        """Workspace a plan of this geometry would hold for minibatches of up to max_batch coils."""
        return int(lib().sdp_workspace_bytes_for(self._h, int(max_batch)))

    def set_wait_test(self, withhold_row, timeout_ns=0):
        """Test hook of the tiled interpolation's bounded copy waits (include/stodip_op.h,
        sdp_plan_set_wait_test): withhold_row >= 0 makes the first CTA skip that tile row's
        copy so its wait runs out; -1 turns it off."""
        _check(lib().sdp_plan_set_wait_test(self._h, int(withhold_row), int(timeout_ns)), "sdp_plan_set_wait_test")

    def launches_per_step(self, B):
        """Kernel launches of one dc_loss forward + backward on B coils (all K channels):
        4 forward, 1 residual/loss, one spread per group of 8 channels and 3 inverse passes."""
        return 4 + 1 + ((self.K + 7) // 8) + 3

    @property
    def beta(self):
        return float(lib().sdp_plan_beta(self._h))

    def status(self):
        """Synchronise the current stream and return (and clear) the device status word."""
        return int(lib().sdp_status(self._h, _stream_ptr(self.device)))

    # -- argument checks --
    def _coils(self, coil_idx):
        _require(coil_idx, "coil_idx", torch.int32, self.device)
        if coil_idx.dim() != 1 or not (1 <= coil_idx.numel() <= self.max_batch):
            raise ValueError(f"coil_idx must be 1-D with 1..{self.max_batch} entries")
        return coil_idx.numel()

    # -- operator --
    def forward(self, x, coil_idx, out=None, k0=0, nk=None, accumulate=False):
        """y[b] = A_{coil_idx[b]}(x) (channels k0..k0+nk of x when given), y [B][J] complex64."""
        B = self._coils(coil_idx)
        _require(x, "x", torch.complex64, self.device, (self.K,) + self.n)
        if out is None:
            if accumulate:
                raise ValueError("accumulate needs out")
            out = torch.empty((B, self.J), dtype=torch.complex64, device=self.device)
        _require(out, "y", torch.complex64, self.device, (B, self.J))
        st = _stream_ptr(self.device)
        if nk is None and k0 == 0 and not accumulate:
            rc = lib().sdp_forward(self._h, _dev_ptr(x), _dev_ptr(coil_idx), B, _dev_ptr(out), st)
        else:
            nk = self.K - k0 if nk is None else nk
            rc = lib().sdp_forward_channels(self._h, _dev_ptr(x), _dev_ptr(coil_idx), B, int(k0), int(nk),
                                            _dev_ptr(out), int(bool(accumulate)), st)
        _check(rc, "sdp_forward")
        return out

    def adjoint(self, y, coil_idx, out=None, accumulate=False, k0=0, nk=None):
        """out_k (+)= sum_b A_{coil_idx[b]}^H y[b], out [K][N1][N2][N3] complex64."""
        B = self._coils(coil_idx)
        _require(y, "y", torch.complex64, self.device, (B, self.J))
        if out is None:
            out = (torch.zeros if (accumulate or nk is not None) else torch.empty)(
                (self.K,) + self.n, dtype=torch.complex64, device=self.device)
        _require(out, "out", torch.complex64, self.device, (self.K,) + self.n)
        st = _stream_ptr(self.device)
        if nk is None and k0 == 0:
            rc = lib().sdp_adjoint(self._h, _dev_ptr(y), _dev_ptr(coil_idx), B, _dev_ptr(out),
                                   int(bool(accumulate)), st)
        else:
            nk = self.K - k0 if nk is None else nk
            rc = lib().sdp_adjoint_channels(self._h, _dev_ptr(y), _dev_ptr(coil_idx), B, int(k0), int(nk),
                                            _dev_ptr(out), int(bool(accumulate)), st)
        _check(rc, "sdp_adjoint")
        return out

    def adjoint_scaled(self, y, coil_idx, scale, out=None, accumulate=False):
        """out_k (+)= (*scale) sum_b A^H y[b] with `scale` a 0-dim float32 device tensor."""
        B = self._coils(coil_idx)
        _require(y, "y", torch.complex64, self.device, (B, self.J))
        _require(scale, "scale", torch.float32, self.device, ())
        if out is None:
            out = torch.empty((self.K,) + self.n, dtype=torch.complex64, device=self.device)
        _require(out, "out", torch.complex64, self.device, (self.K,) + self.n)
        _check(lib().sdp_adjoint_scaled(self._h, _dev_ptr(y), _dev_ptr(coil_idx), B, _dev_ptr(scale),
                                        _dev_ptr(out), int(bool(accumulate)), _stream_ptr(self.device)),
               "sdp_adjoint_scaled")
        return out

    def residual_loss(self, yhat, y_meas, meas_idx, r2=None, loss=None, dcf=None):
        """r2 = 2 dcf (yhat - y_meas[meas_idx]) and loss = sum dcf |yhat - y_meas[meas_idx]|^2 (device scalar);
        dcf: float32 [J] device weights or None (1)."""
        B = self._coils(meas_idx)
        _require(yhat, "yhat", torch.complex64, self.device, (B, self.J))
        if y_meas.dim() != 2 or y_meas.shape[1] != self.J:
            raise ValueError("y_meas must be [rows][J]")
        _require(y_meas, "y_meas", torch.complex64, self.device)
        if dcf is not None:
            _require(dcf, "dcf", torch.float32, self.device, (self.J,))
        if r2 is None:
            r2 = torch.empty_like(yhat)
        if loss is None:
            loss = torch.empty((), dtype=torch.float32, device=self.device)
        _require(r2, "r2", torch.complex64, self.device, (B, self.J))
        _require(loss, "loss", torch.float32, self.device, ())
        st = _stream_ptr(self.device)
        if dcf is None:
            rc = lib().sdp_residual_loss(self._h, _dev_ptr(yhat), _dev_ptr(y_meas), int(y_meas.shape[0]),
                                         _dev_ptr(meas_idx), B, _dev_ptr(r2), _dev_ptr(loss), st)
        else:
            rc = lib().sdp_residual_loss_weighted(self._h, _dev_ptr(yhat), _dev_ptr(y_meas), int(y_meas.shape[0]),
                                                  _dev_ptr(meas_idx), B, _dev_ptr(dcf), _dev_ptr(r2),
                                                  _dev_ptr(loss), st)
        _check(rc, "sdp_residual_loss")
        return r2, loss

    def gram_samples(self, y, out=None):
        """out[b] = Phi_V Phi_V^H y[b]: the spread step followed by the interpolation step."""
        if y.dim() != 2 or y.shape[1] != self.J or not (1 <= y.shape[0] <= self.max_batch):
            raise ValueError(f"y must be [B][J] with 1 <= B <= {self.max_batch}")
        _require(y, "y", torch.complex64, self.device)
        if out is None:
            out = torch.empty_like(y)
        _require(out, "out", torch.complex64, self.device, tuple(y.shape))
        _check(lib().sdp_gram_samples(self._h, _dev_ptr(y), int(y.shape[0]), _dev_ptr(out),
                                      _stream_ptr(self.device)), "sdp_gram_samples")
        return out

    def tv_value(self, x, lam=1.0, eps=1e-6, out=None):
        """lam TV(x) as a device float32 scalar (isotropic, eps-smoothed, per channel)."""
        _require(x, "x", torch.complex64, self.device, (self.K,) + self.n)
        if out is None:
            out = torch.empty((), dtype=torch.float32, device=self.device)
        _check(lib().sdp_tv_value(self._h, _dev_ptr(x), float(eps), float(lam), _dev_ptr(out),
                                  _stream_ptr(self.device)), "sdp_tv_value")
        return out

    def tv_grad(self, x, lam=1.0, eps=1e-6, scale=None, out=None, accumulate=False):
        """(accumulate ? out : 0) + lam (*scale) grad TV(x)."""
        _require(x, "x", torch.complex64, self.device, (self.K,) + self.n)
        if out is None:
            out = torch.empty_like(x)
        _require(out, "out", torch.complex64, self.device, (self.K,) + self.n)
        if scale is not None:
            _require(scale, "scale", torch.float32, self.device, ())
        _check(lib().sdp_tv_grad(self._h, _dev_ptr(x), float(eps), float(lam),
                                 _dev_ptr(scale) if scale is not None else None, _dev_ptr(out),
                                 int(bool(accumulate)), _stream_ptr(self.device)), "sdp_tv_grad")
        return out

    # -- profiling --
    def profile(self, enable=True):
        _check(lib().sdp_profile_enable(self._h, int(bool(enable))), "sdp_profile_enable")

    def profile_read(self):
        ms = (ctypes.c_double * len(STAGES))()
        nl = (ctypes.c_int64 * len(STAGES))()
        n = lib().sdp_profile_read(self._h, ms, nl, len(STAGES))
        if n < 0:
            raise SdpError(-n, "sdp_profile_read")
        return {STAGES[i]: (float(ms[i]), int(nl[i])) for i in range(n)}


def _batched(items, adjoint):
    if not items:
        return []
    dev = items[0][0].device
    arr = (Work * len(items))()
    outs = []
    for i, (op, inp, coil_idx, out, acc) in enumerate(items):
        B = op._coils(coil_idx)
        if adjoint:
            _require(inp, "y", torch.complex64, op.device, (B, op.J))
            if out is None:
                out = torch.empty((op.K,) + op.n, dtype=torch.complex64, device=op.device)
            _require(out, "out", torch.complex64, op.device, (op.K,) + op.n)
        else:
            _require(inp, "x", torch.complex64, op.device, (op.K,) + op.n)
            if out is None:
                out = torch.empty((B, op.J), dtype=torch.complex64, device=op.device)
            _require(out, "y", torch.complex64, op.device, (B, op.J))
        arr[i] = Work(op._h.value, inp.data_ptr(), coil_idx.data_ptr(), B, int(bool(acc)), out.data_ptr())
        outs.append(out)
    fn = lib().sdp_adjoint_batched if adjoint else lib().sdp_forward_batched
    _check(fn(arr, len(items), _stream_ptr(dev)), "sdp_adjoint_batched" if adjoint else "sdp_forward_batched")
    return outs


def forward_batched(items):
    """items: [(op, x, coil_idx, y_out_or_None)] -> list of y.  Plans differing
    between items run concurrently on the library's worker streams."""
    return _batched([(op, x, c, o, False) for (op, x, c, o) in items], adjoint=False)


def adjoint_batched(items):
    """items: [(op, y, coil_idx, out_or_None, accumulate)] -> list of out."""
    return _batched(list(items), adjoint=True)


def launch_count() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().sdp_launch_count())


class _ApplyA(torch.autograd.Function):
    """y = A_B(x) with backward grad_x = A_B^H grad_y (PyTorch's conjugate-Wirtinger
    convention makes the vector-Jacobian product of a linear complex map its adjoint)."""

    @staticmethod
    def forward(ctx, x, coil_idx, op):
        ctx.op = op
        ctx.save_for_backward(coil_idx)
        return op.forward(x.contiguous(), coil_idx)

    @staticmethod
    def backward(ctx, gy):
        (coil_idx,) = ctx.saved_tensors
        gx = ctx.op.adjoint(gy.contiguous(), coil_idx) if ctx.needs_input_grad[0] else None
        return gx, None, None


def apply_A(op: SubspaceNufft, x, coil_idx):
    """Differentiable A_B(x) for a coil minibatch coil_idx (Algorithm 1, lines 4 and 7)."""
    return _ApplyA.apply(x, coil_idx, op)


class _DataConsistency(torch.autograd.Function):
    """L = sum_b ||A_{c_b}(x) - y_meas[row_b]||^2 (Eq. 3, DCF = 1) with the whole
    forward (operator + residual + loss) and backward (scaled adjoint of 2r) in
    the library's kernels."""

    @staticmethod
    def forward(ctx, x, coil_idx, meas_idx, y_meas, op, dcf):
        yhat = op.forward(x.contiguous(), coil_idx)
        r2, loss = op.residual_loss(yhat, y_meas, meas_idx, r2=yhat, dcf=dcf)   # r2 overwrites yhat in place
        ctx.op = op
        ctx.save_for_backward(coil_idx, r2)
        return loss

    @staticmethod
    def backward(ctx, gL):
        coil_idx, r2 = ctx.saved_tensors
        gx = None
        if ctx.needs_input_grad[0]:
            gx = ctx.op.adjoint_scaled(r2, coil_idx, gL.to(torch.float32).contiguous())
        return gx, None, None, None, None, None


def dc_loss(op: SubspaceNufft, x, coil_idx, y_meas, meas_idx=None, dcf=None):
    """Differentiable data-consistency loss of a coil minibatch (Algorithm 1, lines 4-5; Eq. 2/3).

    y_meas [rows][J]: measured k-space; row meas_idx[b] is compared with coil
    coil_idx[b] (default meas_idx = coil_idx, i.e. y_meas holds all C coils).
    dcf: optional float32 [J] density compensation (Eq. 2), None for DCF = 1.
    """
    return _DataConsistency.apply(x, coil_idx, coil_idx if meas_idx is None else meas_idx, y_meas, op, dcf)


class _TotalVariation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op, lam, eps):
        xc = x.contiguous()
        ctx.op, ctx.lam, ctx.eps = op, lam, eps
        ctx.save_for_backward(xc)
        return op.tv_value(xc, lam, eps)

    @staticmethod
    def backward(ctx, gL):
        (x,) = ctx.saved_tensors
        gx = None
        if ctx.needs_input_grad[0]:
            gx = ctx.op.tv_grad(x, ctx.lam, ctx.eps, scale=gL.to(torch.float32).contiguous())
        return gx, None, None, None


def tv_loss(op: SubspaceNufft, x, lam: float, eps: float = 1e-6):
    """Differentiable lam TV(x) (Algorithm 1 line 6), value and gradient in the library's kernels."""
    return _TotalVariation.apply(x, op, float(lam), float(eps))


def make_operator(omega, frame, n, width, oversamp, V, S, max_batch, device="cuda", tuning=None, borrow_maps=False):
    """Plan from numpy inputs (omega float32 [J][3], frame int [J] non-decreasing); S may also be a
    complex64 device tensor, which the plan then borrows when borrow_maps is set."""
    T = V.shape[0]
    off = np.searchsorted(np.asarray(frame), np.arange(T + 1), side="left").astype(np.int64)
    off[-1] = len(frame)
    dev = torch.device(device)
    St = S if isinstance(S, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(S, np.complex64)).to(dev)
    return SubspaceNufft(torch.from_numpy(np.ascontiguousarray(omega, np.float32)).to(dev), off, n, width,
                         oversamp, torch.from_numpy(np.ascontiguousarray(V, np.complex64)).to(dev),
                         St, max_batch=max_batch, tuning=tuning, borrow_maps=borrow_maps)
