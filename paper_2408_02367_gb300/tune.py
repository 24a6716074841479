"""Autotuner of the operator's kernel shapes.

A plan's kernel shapes (include/stodip_op.h, sdp_tuning) do not change what
the operator computes, only how fast it runs on a given trajectory and volume:

- spread bin shape: 8 x 4 x 8 bins (a lane per 8-point axis-3 column),
  8 x 4 x 4 bins (half the accumulator registers, so more resident warps, but
  about 1.3x the (sample, bin) incidences of a W = 4 window), or 4 x 4 x 8 and
  4 x 4 x 4 bins (two incidences per warp step, one per half-warp: more of each
  multiply-add counts, against more incidences per sample);
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
- the forward prologue and the adjoint epilogue with their inputs staged by bulk
  copies, or loaded directly (each on its own);
- the interpolation from shared-memory tiles, or the row kernel's gathers.

`autotune` tunes the spread's knobs first and the rest on the fastest spread
(they are nearly independent).  It builds a plan for every candidate on the
caller's geometry, checks
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
           "interp_threads": 0, "spread_coils": 0, "interp_run": 0, "interp_coils": 0, "fft_staged": 0,
           "interp_tiled": 0}


SPREAD_BINS = ((8, 4, 8), (8, 4, 4), (4, 4, 8), (4, 4, 4))


def candidates(full: bool = False):
    """First round: the spread's knobs with the default FFT and interpolation
    shapes: every bin shape x three chunk lengths (`full`: five), and one coil
    per spread warp for the 4-deep bins."""
    chunks = (128, 256, 512, 1024, 2048) if full else (256, 512, 1024)
    out = []
    for bins in SPREAD_BINS:
        for c in chunks:
            out.append({"spread_bins": bins, "spread_chunk": c, "fft_engine": 0, "fft_lines": 0})
    for bins in SPREAD_BINS:
        if bins[2] == 4:
            out.append({"spread_bins": bins, "spread_chunk": 512, "fft_engine": 0, "fft_lines": 0, "spread_coils": 1})
    return out


REFINE = [{"fft_lines": 8}, {"fft_lines": 4}, {"fft_lines": 8, "fft_cols": 32}, {"fft_lines": 8, "fft_cols": 8},
          {"fft_lines": 8, "interp_threads": 256},
          {"fft_lines": 8, "interp_threads": 1024, "interp_run": 1, "interp_coils": 2},
          {"fft_lines": 8, "interp_threads": 1024, "interp_run": 2, "interp_coils": 2},
          {"fft_lines": 8, "fft_staged": 3},
          {"fft_lines": 8, "interp_threads": 1024, "interp_run": 2, "interp_coils": 2, "fft_staged": 3},
          {"fft_lines": 8, "interp_threads": 256, "interp_run": 1, "interp_coils": 2, "fft_staged": 3},
          {"fft_lines": 8, "interp_tiled": 1}, {"fft_lines": 8, "interp_tiled": 1, "fft_staged": 1},
          {"fft_lines": 8, "interp_tiled": 1, "fft_staged": 2}, {"fft_lines": 8, "interp_tiled": 1, "fft_staged": 3},
          {"fft_lines": 8, "fft_cols": 32, "interp_tiled": 1, "fft_staged": 3},
          {"fft_lines": 8, "fft_cols": 8, "interp_tiled": 1, "fft_staged": 3},
          {"fft_engine": 1, "fft_lines": 0}]


def refinements(spread, variants=REFINE):
    """Second round, on the spread knobs of the first round's fastest tuning: FFT
    lines (8, 4) and columns (32, 8) per CTA, interpolation CTA size, run length
    and coil blocks, the tiled interpolation, the staged prologue, and the
    Stockham engine."""
    base = {k: spread[k] for k in ("spread_bins", "spread_chunk", "spread_coils")}
    return [dict(base, fft_engine=0, **v) if "fft_engine" not in v else dict(base, **v) for v in variants]


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
             cache: str | None = None, device="cuda", agree: float = 1e-5, refine=None):
    """Fastest tuning for this geometry.  Returns (tuning dict, table of
    {"tuning", "ms", "rel_vs_first"} for every candidate, sorted by time).
    Without `cands`, two rounds: the spread's knobs (`candidates()`), then the
    FFT and interpolation knobs on the fastest spread (`refinements`).  With
    `cands`, one round unless `refine` lists second-round variants."""
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
    if cands is None:
        cands, refine = candidates(), REFINE if refine is None else refine
    K = V.shape[1]
    gen = torch.Generator(device="cpu").manual_seed(12345)
    x = torch.complex(torch.randn((K,) + tuple(n), generator=gen), torch.randn((K,) + tuple(n), generator=gen))
    x = x.to(torch.complex64).to(dev)
    ci = torch.arange(B, dtype=torch.int32, device=dev) % S.shape[0]
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)     # 256 MB, larger than L2
    table = []
    ref = []

    def run(t):
        A = _op.make_operator(omega, frame, n, width, oversamp, V, S, max_batch, device=device, tuning=t)
        y = A.forward(x, ci)
        a = A.adjoint(y, ci)
        if not ref:
            ref.append((y.clone(), a.clone(), t))
            rel = 0.0
        else:
            rel = max(_rel(y, ref[0][0]), _rel(a, ref[0][1]))
            if not rel <= agree:
                raise RuntimeError(f"tuning {t} disagrees with {ref[0][2]}: rel {rel:.2e}")
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

    for t in cands:
        run(t)
    if refine:
        first = min(table, key=lambda r: r["ms"])["tuning"]
        for t in refinements(dict(first, spread_bins=tuple(first["spread_bins"])), refine):
            run(t)
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
