"""Autotuner of the operator's kernel shapes.

A plan's kernel shapes (include/stodip_op.h, sdp_tuning) do not change what
the operator computes, only how fast it runs on a given trajectory and volume:

- spread bin depth: 8 x 4 x 8 bins (a lane per 8-point axis-3 column) or
  8 x 4 x 4 bins (half the accumulator registers, so more resident warps, but
  about 1.3x the (sample, bin) incidences of a W = 4 window);
- spread chunk length: incidences per spread CTA (load balance on the dense
  k-space centre against the cost of summing partial tiles);
- FFT engine: the two-pass register FFTs or the Stockham kernels;
- FFT lines per CTA of the fused axis-3 prologue and epilogue (16, 8 or 4);
- FFT columns per CTA of the strided axis-1/axis-2 passes (16, 32 or 8);
- threads per CTA of the persistent interpolation kernel (1024 or 256);
- coils per spread warp (two coils share the staging of each incidence where
  their register columns fit, or one);
- consecutive samples per interpolation warp run, and coils per sweep of the
  interpolation over the samples (all, or two at a time);
- the forward prologue with its inputs staged by bulk copies, or loaded directly.

`autotune` builds a plan for every candidate on the caller's geometry, checks
that every candidate's forward and adjoint agree with the first one (they
compute the same operator; only the order of floating-point sums differs),
times one operator step (forward of a coil minibatch, then its adjoint) with
CUDA events and the L2 cache flushed before each repetition, and returns the
fastest tuning with the whole table.  With `cache=` a JSON file keyed by the
geometry, a hash of the trajectory and the GPU name keeps earlier results.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import op as _op

DEFAULT = {"spread_bins": (8, 4, 8), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 0, "fft_cols": 0,
           "interp_threads": 0, "spread_coils": 0, "interp_run": 0, "interp_coils": 0}


def candidates(full: bool = False):
    """The tunings tried: both bin depths x three chunk lengths with the two-pass
    FFTs, both bin depths with 8 and 4 FFT lines per CTA, 32 and 8 strided FFT
    columns per CTA, 256-thread interpolation CTAs, one coil per spread warp,
    and the Stockham engine on the default spread; `full` adds more chunks."""
    chunks = (128, 256, 512, 1024, 2048) if full else (256, 512, 1024)
    out = []
    for bins in ((8, 4, 8), (8, 4, 4)):
        for c in chunks:
            out.append({"spread_bins": bins, "spread_chunk": c, "fft_engine": 0, "fft_lines": 0})
    for bins in ((8, 4, 8), (8, 4, 4)):
        for lines in (8, 4):
            out.append({"spread_bins": bins, "spread_chunk": 512, "fft_engine": 0, "fft_lines": lines})
    for cols in (32, 8):
        out.append({"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8, "fft_cols": cols})
    out.append({"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8, "interp_threads": 256})
    out.append({"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8, "spread_coils": 1})
    for run in (1, 2):
        out.append({"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8,
                    "interp_threads": 1024, "interp_run": run, "interp_coils": 2})
    for threads, run in ((1024, 2), (256, 1)):
        out.append({"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8,
                    "interp_threads": threads, "interp_run": run, "interp_coils": 2, "fft_staged": 1})
    out.append({"spread_bins": (8, 4, 8), "spread_chunk": 512, "fft_engine": 1, "fft_lines": 0})
    return out


def _key(omega, frame, n, width, oversamp, V, S, max_batch, B, device):
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(omega, np.float32).tobytes())
    h.update(np.ascontiguousarray(frame, np.int64).tobytes())
    name = torch.cuda.get_device_name(torch.device(device))
    return (f"{name}|n={tuple(int(v) for v in n)}|W={int(width)}|sigma={float(oversamp)}|K={V.shape[1]}|"
            f"T={V.shape[0]}|C={S.shape[0]}|maxB={int(max_batch)}|B={int(B)}|traj={h.hexdigest()[:16]}")


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def autotune(omega, frame, n, width, oversamp, V, S, max_batch, B=None, cands=None, reps: int = 5,
             cache: str | None = None, device="cuda", agree: float = 1e-5):
    """Fastest tuning for this geometry.  Returns (tuning dict, table of
    {"tuning", "ms", "rel_vs_first"} for every candidate, sorted by time)."""
    B = int(max_batch if B is None else B)
    dev = torch.device(device)
    key = _key(omega, frame, n, width, oversamp, V, S, max_batch, B, device)
    if cache and os.path.exists(cache):
        with open(cache) as f:
            stored = json.load(f)
        if key in stored:
            e = stored[key]
            best = dict(e["best"], spread_bins=tuple(e["best"]["spread_bins"]))
            return best, e["table"]
    cands = candidates() if cands is None else cands
    K = V.shape[1]
    gen = torch.Generator(device="cpu").manual_seed(12345)
    x = torch.complex(torch.randn((K,) + tuple(n), generator=gen), torch.randn((K,) + tuple(n), generator=gen))
    x = x.to(torch.complex64).to(dev)
    ci = torch.arange(B, dtype=torch.int32, device=dev) % S.shape[0]
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)     # 256 MB, larger than L2
    table = []
    ref = None
    for t in cands:
        A = _op.make_operator(omega, frame, n, width, oversamp, V, S, max_batch, device=device, tuning=t)
        y = A.forward(x, ci)
        a = A.adjoint(y, ci)
        if ref is None:
            ref = (y.clone(), a.clone())
            rel = 0.0
        else:
            rel = max(_rel(y, ref[0]), _rel(a, ref[1]))
            if not rel <= agree:
                raise RuntimeError(f"tuning {t} disagrees with {cands[0]}: rel {rel:.2e}")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for i, (e0, e1) in enumerate(evs):
            flush.fill_(float(i))
            e0.record()
            A.forward(x, ci, out=y)
            A.adjoint(y, ci, out=a)
            e1.record()
        torch.cuda.synchronize()
        ms = sorted(e0.elapsed_time(e1) for e0, e1 in evs)[reps // 2]
        table.append({"tuning": dict(A.tuning, spread_bins=list(A.tuning["spread_bins"])), "ms": ms,
                      "rel_vs_first": rel})
        del A
    table.sort(key=lambda r: r["ms"])
    best = dict(table[0]["tuning"], spread_bins=tuple(table[0]["tuning"]["spread_bins"]))
    if cache:
        stored = {}
        if os.path.exists(cache):
            with open(cache) as f:
                stored = json.load(f)
        stored[key] = {"best": dict(best, spread_bins=list(best["spread_bins"])), "table": table}
        with open(cache, "w") as f:
            json.dump(stored, f, indent=1)
    return best, table
