#!/usr/bin/env python
"""Benchmark of one StoDIP data-consistency step on the subspace multicoil NUFFT operator.

One step = Algorithm 1, lines 4, 5 and 7 (DCF = 1, no TV term) on a coil
minibatch drawn uniformly without replacement:
    yhat = A_B(x_hat);  L = sum_b ||yhat_b - y_{c_b}||^2;  L.backward()
i.e. the forward operator, the residual/loss and the autograd adjoint
A_B^H(2r), all in libstodip_op.so kernels, with x_hat a fixed complex TSMI
that requires grad (the generator G_theta is not part of the operator).

Workload (default): 128^3 image, K=5 subspace channels, C=8 coils, T=480
frames of one 1024-sample golden-angle 3D spiral arm (J=491,520 samples per
coil), Kaiser-Bessel W=4 on a 1.25x oversampled grid (160^3), B=2 coils per
step.  Synthetic seeded inputs (phantom, coil maps, trajectory, V).

Beside the headline step the line carries the whole-brain rows (200x200x160,
C=32, J=2,048,000: the captured DIP step at coil minibatches 1, 2, 4 and 8, and
a work list of those four minibatches through the batched calls) and the
six-volume batch (64^3 .. 200x200x160, one DIP step of every volume in one
captured batch, plus the full-coil variant against a 150 GB device-memory
bound).

Prints ONE JSON line (rank 0).  `--impl reference` instead times whole steps of
the FP64 CPU oracle on the same workload, on every host core.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2408_02367_gb300 import synth  # noqa: E402

METRIC = "DIP step ms (A_c fwd + autograd A_c^H) and NU samples/s at 1e-4 rel err vs plain"
UNIT = "NU samples/s"
L2_BYTES = 129 * 1024 * 1024
FLUSH_BYTES = 256 * 1024 * 1024


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_desc(w, B):
    return (f"{w.name}: {w.n[0]}x{w.n[1]}x{w.n[2]} image, K={w.K} subspace channels, C={w.C} coils, "
            f"T={w.T} frames x {w.arms} golden-angle 3D spiral arm(s) x {w.arm_len} samples "
            f"(J={w.J} per coil), Kaiser-Bessel W={w.width}, sigma={w.oversamp}, coil minibatch B={B}")


# ----------------------------------------------------------------------------
# distributed helpers (replicas: each rank runs its own coil minibatches)
# ----------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(base: int, rank: int) -> int:
    """Coil-draw seed of one replica: independent minibatch streams per rank."""
    return base + 1000 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest per-rank value (the slowest replica sets the job time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id=None, interval_ms=100):
        self.gpu_id = gpu_id
        self.interval_ms = interval_ms
        self.lines = []
        self.proc = None
        self.err = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", str(self.interval_ms)]
        if self.gpu_id:
            cmd.insert(1, f"--id={self.gpu_id}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:   # nvidia-smi missing
            self.err = str(e)
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "error": self.err}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, pw, reasons = [], [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# algorithmic bytes per launch of each kernel (the HBM roofline model)
# ----------------------------------------------------------------------------

def stage_bytes(w, B, M, ninc):
    """Bytes each kernel must move per launch (read + write, complex64 = 8 B).

    The oversampled grid of every (coil, channel) is written once and read once
    per pass; x, S, y and the sample tables are read once."""
    N1, N2, N3 = w.n
    M1, M2, M3 = M
    K, J = w.K, w.J
    nvox = N1 * N2 * N3
    G = M1 * M2 * M3
    c = 8
    return {
        "fwd_prologue_fft3": c * (K * nvox + B * nvox + B * K * N1 * N2 * M3),
        "fwd_fft2": c * B * K * (N1 * N2 * M3 + N1 * M2 * M3),
        "fwd_fft1": c * B * K * (N1 * M2 * M3 + G),
        "interp": c * B * K * G + 20 * J + c * B * J,
        "residual_loss": 3 * c * B * J,
        "spread": c * B * J + 20 * J + 4 * ninc + c * B * K * G,
        "adj_ifft1": c * B * K * (G + N1 * M2 * M3),
        "adj_ifft2": c * B * K * (N1 * M2 * M3 + N1 * N2 * M3),
        "adj_ifft3_epilogue": c * (B * K * N1 * N2 * M3 + B * nvox + K * nvox),
    }


# DRAM bytes (read + write) of one launch of each kernel on the vol128_w4
# workload (B=2, K=5), from one `ncu --set full` capture of a DIP step
# (profiles/kernels_vol128_w4.md), keyed with a hash of the kernel's source file
# at capture time and the kernel variant (spread bin shape, tiled interpolation,
# staged prologue or epilogue, strided columns per CTA): a kernel whose source has
# changed since reports null.
NCU_TRAFFIC = {
    ("spread", (4, 4, 4)): ("spread_impl.cuh", "bf009aeec1d9f154", (55.761152 + 279.115520) * 1e6),
    ("interp", 1): ("interp_tiles.cu", "2650bb20b6abb58c", (370.516992 + 10.980864) * 1e6),
    ("fwd_prologue_fft3", 1): ("fft2_staged.cu", "6d826d9b6950716f", (117.908992 + 152.950528) * 1e6),
    ("adj_ifft3_epilogue", 1): ("fft2_staged.cu", "6d826d9b6950716f", (246.183424 + 61.779200) * 1e6),
    ("fwd_fft2", 32): ("fft2_impl.cuh", "2e882cd182edfd57", (209.750528 + 208.728320) * 1e6),
    ("fwd_fft1", 32): ("fft2_impl.cuh", "2e882cd182edfd57", (262.183680 + 274.098176) * 1e6),
    ("adj_ifft1", 32): ("fft2_impl.cuh", "2e882cd182edfd57", (327.721984 + 217.612032) * 1e6),
    ("adj_ifft2", 32): ("fft2_impl.cuh", "2e882cd182edfd57", (262.177024 + 167.035392) * 1e6),
}


def source_hash(fname):
    import hashlib
    path = os.path.join(ROOT, "paper_2408_02367_gb300", "csrc", fname)
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_traffic(stage, workload_name, B, tuning):
    """ncu DRAM bytes per launch of `stage`, if captured for this workload, the kernel the tuning
    selects (spread bin shape, tiled interpolation, staged prologue or epilogue, strided columns
    per CTA) and the current source."""
    cols = int(tuning.get("fft_cols", 0)) or 16
    key = {"spread": ("spread", tuple(tuning["spread_bins"])), "interp": ("interp", int(tuning["interp_tiled"])),
           "fwd_prologue_fft3": ("fwd_prologue_fft3", int(tuning["fft_staged"]) & 1),
           "adj_ifft3_epilogue": ("adj_ifft3_epilogue", int(tuning["fft_staged"]) >> 1 & 1),
           "fwd_fft2": ("fwd_fft2", cols), "fwd_fft1": ("fwd_fft1", cols),
           "adj_ifft1": ("adj_ifft1", cols), "adj_ifft2": ("adj_ifft2", cols)}.get(stage, stage)
    if workload_name != "vol128_w4" or B != 2 or key not in NCU_TRAFFIC:
        return None
    fname, h, nbytes = NCU_TRAFFIC[key]
    return nbytes if source_hash(fname) == h else None


def path_model_bytes(w, B, M):
    """Whole-step model: 8 K Nvox + B (8 Nvox + 16 K G + 8 J) + 12 J per direction."""
    nvox = int(np.prod(w.n))
    G = int(np.prod(M))
    one = 8 * w.K * nvox + B * (8 * nvox + 16 * w.K * G + 8 * w.J) + 12 * w.J
    return 2 * one


# ----------------------------------------------------------------------------
# CPU oracle (baseline / reference arm): whole steps on every host core
# ----------------------------------------------------------------------------
#
# One step of the oracle is the step the GPU times: the forward operator of B
# coils over all K channels, the residual, and the adjoint of 2r over the same
# coils and channels.  The oracle's own step functions (A1-A3, A5-A7, FP64
# numpy) run unchanged; the B*K (coil, channel) pieces of each direction are
# independent, so they run side by side in a pool of spawned processes, one per
# piece, up to the host's core count.  Nothing is sampled or scaled: the value
# is B*J samples over the wall time of whole steps.

_ORACLE = {}


def _oracle_init(n, W, sigma, x, S, V, omega, frame):
    from oracle import nufft as O
    _ORACLE.update(O=O, geo=O.Geometry(n, W, sigma), x=x, S=S, V=V, omega=omega, frame=frame)


def _oracle_fwd(coil, k):
    """Channel k of A_c(x): A1 prologue, A2 FFT, A3 interpolation with V[:, k]."""
    d = _ORACLE
    O, geo = d["O"], d["geo"]
    g32 = O.grid_coords(d["omega"], geo.M)
    U = O.fwd_fft(O.fwd_prologue(geo, d["x"][k], d["S"][coil]))
    return O.fwd_interp(geo, U[None], d["V"][:, k:k + 1], g32, d["frame"])


def _oracle_adj(coil, k, r):
    """Channel k of A_c^H r: A5 spread with conj(V[:, k]), A6 inverse FFT, A7 epilogue."""
    d = _ORACLE
    O, geo = d["O"], d["geo"]
    g32 = O.grid_coords(d["omega"], geo.M)
    H = O.adj_spread(geo, r, d["V"][:, k:k + 1], g32, d["frame"])
    out = O.adj_epilogue(geo, O.adj_ifft(H[0]), d["S"][coil])
    return complex(np.sum(out))      # the image stays in the worker; its sum proves it was formed


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


class OracleSteps:
    """Whole oracle steps of one workload (coils drawn like the GPU arm's) on a spawned process pool."""

    def __init__(self, w, B, coils_of_step=None, max_workers=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.w, self.B = w, B
        x, S, V, omega, frame = synth.make_problem(w)
        self.C = w.C
        self.coils_of_step = coils_of_step
        self.y_meas = synth.complex_noise((w.C, w.J), 1.0).astype(np.complex128)
        self.workers = min(B * w.K, os.cpu_count() or 1) if max_workers is None else max_workers
        self.pool = cf.ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"), initializer=_oracle_init,
                                           initargs=(w.n, w.width, w.oversamp, x, S, V, omega, frame))

    def step(self, coils):
        K = self.w.K
        fut = [[self.pool.submit(_oracle_fwd, int(c), k) for k in range(K)] for c in coils]
        ys = [sum(f.result() for f in row) for row in fut]                       # A_c(x) of every coil
        r2 = [2.0 * (y - self.y_meas[int(c)]) for y, c in zip(ys, coils)]        # dL/dyhat (Eq. 3, DCF = 1)
        loss = float(sum(np.sum(np.abs(0.5 * r) ** 2) for r in r2))
        fut = [self.pool.submit(_oracle_adj, int(c), k, r) for c, r in zip(coils, r2) for k in range(K)]
        chk = sum(f.result() for f in fut)
        return loss, chk

    def time_steps(self, draws):
        ts = []
        for coils in draws:
            t0 = time.perf_counter()
            self.step(coils)
            ts.append(time.perf_counter() - t0)
        return ts

    def close(self):
        self.pool.shutdown(wait=True, cancel_futures=True)


def oracle_line(w, B, ts, workers, what):
    t = float(np.mean(ts))
    return {"value": B * w.J / t, "unit": UNIT, "cores": workers, "kind": "oracle", "host_cpus": os.cpu_count(),
            "cpu_model": cpu_model(), "seconds_per_step": t, "steps_timed": len(ts),
            "sample": (f"{what}: {len(ts)} whole oracle step(s) of {workload_desc(w, B)}: FP64 numpy forward of "
                       f"B={B} coils x K={w.K} channels, residual, adjoint of 2r; the B*K (coil, channel) pieces of "
                       f"each direction run in {workers} spawned processes; nothing scaled")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = synth.WORKLOADS[args.workload]
    B = args.batch or w.batch
    draws = synth.coil_minibatches(w.C, B, args.warmup + args.steps, seed=rank_seed(synth.SEED_COILS_DRAW, rank))
    t_start = time.perf_counter()
    orc = OracleSteps(w, B)
    try:
        orc.time_steps(draws[:args.warmup])
        ts = orc.time_steps(draws[args.warmup:])
    finally:
        orc.close()
    base = oracle_line(w, B, ts, orc.workers, "per step")
    t = base["seconds_per_step"]
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(w, B), "parallelism": f"cpu, {orc.workers} processes"},
            "cpu_baseline": base, "run_seconds": time.perf_counter() - t_start,
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline(w, B, whole_brain=False):
    """The oracle on the host cores: whole steps of the bench workload (the reported value), of the
    32^3 W=6 workload, and with whole_brain one coil x all K of the 200x200x160 workload."""
    draws = synth.coil_minibatches(w.C, B, 3, seed=synth.SEED_COILS_DRAW + 77)
    orc = OracleSteps(w, B)
    try:
        orc.time_steps(draws[:1])                 # starts the workers
        ts = orc.time_steps(draws[1:])
    finally:
        orc.close()
    out = oracle_line(w, B, ts, orc.workers, "bench workload")
    rows = {}
    w1 = synth.WORKLOADS["vol32_w6"]
    orc = OracleSteps(w1, w1.batch)
    try:
        coils = [np.arange(w1.batch)] * 3
        orc.time_steps(coils[:1])
        rows["vol32_w6"] = oracle_line(w1, w1.batch, orc.time_steps(coils[1:]), orc.workers, "32^3 workload")
    finally:
        orc.close()
    if whole_brain:
        w4 = synth.WORKLOADS["vol200_w4"]
        orc = OracleSteps(w4, 1)
        try:
            rows["vol200_w4_one_coil"] = oracle_line(w4, 1, orc.time_steps([np.array([0])]), orc.workers,
                                                     "whole-brain workload, one coil")
        finally:
            orc.close()
    out["other_workloads"] = rows
    return out


# ----------------------------------------------------------------------------
# whole-brain and multi-volume rows (measured beside the headline step)
# ----------------------------------------------------------------------------

def _upload_plan(op, torch, w, omega, frame, V, S, max_batch, dev, tuning):
    """Inputs to the device first, then the plan alone timed (sdp_plan_create: host grid coordinates,
    bin sort and incidence lists, device tables, the coil-map copy)."""
    traj = torch.from_numpy(np.ascontiguousarray(omega, np.float32)).to(dev)
    Vt = torch.from_numpy(np.ascontiguousarray(V, np.complex64)).to(dev)
    St = torch.from_numpy(np.ascontiguousarray(S, np.complex64)).to(dev)
    off = np.searchsorted(np.asarray(frame), np.arange(w.T + 1), side="left").astype(np.int64)
    off[-1] = len(frame)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    A = op.SubspaceNufft(traj, off, w.n, w.width, w.oversamp, Vt, St, max_batch=max_batch, tuning=tuning)
    torch.cuda.synchronize(dev)
    return A, time.perf_counter() - t0


def _measured_kspace(A, torch, x_true, C, dev, maxB):
    """y_c = A_c(x_true) + complex noise at 30 dB SNR for every coil, in minibatches of maxB."""
    xt = torch.from_numpy(x_true).to(dev)
    y = torch.empty((C, A.J), dtype=torch.complex64, device=dev)
    for c0 in range(0, C, maxB):
        c1 = min(C, c0 + maxB)
        A.forward(xt, torch.arange(c0, c1, dtype=torch.int32, device=dev), out=y[c0:c1])
    sig = float(torch.linalg.norm(y).item()) ** 2 / (y.numel() * 1e3)
    y += torch.from_numpy(synth.complex_noise((C, A.J), math.sqrt(sig))).to(dev)
    return y


def _events_ms(torch, fn, n, flush, per_call_args=None):
    """Mean CUDA-event time of n calls, L2 flushed before each (outside the events)."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for i in range(n):
        flush.fill_(float(i))
        evs[i][0].record()
        fn(i)
        evs[i][1].record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / n


def _plain_step(A, torch, x, y_meas, ci, K):
    """The plain form: one coil and one channel per launch, same arithmetic."""
    B = ci.numel()
    y_p = torch.zeros((B, A.J), dtype=torch.complex64, device=x.device)
    for b in range(B):
        for k in range(K):
            A.forward(x, ci[b:b + 1], out=y_p[b:b + 1], k0=k, nk=1, accumulate=True)
    r2, loss = A.residual_loss(y_p, y_meas, ci)
    g = torch.zeros_like(x)
    for b in range(B):
        for k in range(K):
            A.adjoint(r2[b:b + 1].contiguous(), ci[b:b + 1], out=g, accumulate=True, k0=k, nk=1)
    return y_p, loss, g


# whole-brain autotuning at B = 8 (each candidate builds a 16 GB plan): the spread's
# bin shapes first, then the FFT / interpolation knobs on the fastest spread
WHOLE_BRAIN_CANDIDATES = [
    {"spread_bins": bins, "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8, "interp_threads": 1024}
    for bins in ((8, 4, 4), (4, 4, 4), (4, 4, 8), (8, 4, 8))
] + [{"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8, "interp_threads": 1024,
      "spread_coils": 1}]
WHOLE_BRAIN_REFINE = [
    {"fft_lines": 8, "interp_threads": 256},
    {"fft_lines": 8, "interp_threads": 1024, "interp_coils": 2},
    {"fft_lines": 8, "interp_threads": 1024, "interp_coils": 2, "interp_run": 2},
    {"fft_lines": 8, "interp_threads": 256, "interp_coils": 2},
    {"fft_lines": 8, "interp_tiled": 1},
    {"fft_lines": 8, "interp_tiled": 1, "fft_staged": 1},
    {"fft_lines": 8, "interp_tiled": 1, "fft_staged": 2},
    {"fft_lines": 8, "interp_tiled": 1, "fft_staged": 3},
    {"fft_lines": 8, "fft_cols": 8, "interp_tiled": 1, "fft_staged": 2},
    {"fft_lines": 8, "fft_cols": 32, "interp_tiled": 1, "fft_staged": 2},
]


def whole_brain_rows(args, torch, op, dev, tuning, flush, hbm):
    """200x200x160, C=32, J=2,048,000: the graph-captured DIP step at each coil minibatch B in {1,2,4,8}
    (against the plain form at equal accuracy), and the work list of four items (own TSMI each, B=1,2,4,8)
    through one batched forward and one batched adjoint."""
    from paper_2408_02367_gb300 import graph as sdp_graph
    w = synth.WORKLOADS["vol200_w4"]
    Bmax = max(synth.WHOLE_BRAIN_BATCHES)
    # the plan's workspace holds the whole work list's coils (1 + 2 + 4 + 8), so the batched
    # calls run every item in the same launches
    Bplan = sum(synth.WHOLE_BRAIN_BATCHES)
    t0 = time.perf_counter()
    x_true, S, V, omega, frame = synth.make_problem(w)
    synth_s = time.perf_counter() - t0
    tune_table = None
    if not args.no_tune:
        # kernel shapes for this workload, by the autotuner on its own trajectory at B = 8
        from paper_2408_02367_gb300 import tune
        tuning, tune_table = tune.autotune(omega, frame, w.n, w.width, w.oversamp, V, S, max_batch=Bmax, B=Bmax,
                                           cands=WHOLE_BRAIN_CANDIDATES, refine=WHOLE_BRAIN_REFINE, reps=3,
                                           device=dev)
    A, plan_s = _upload_plan(op, torch, w, omega, frame, V, S, Bplan, dev, tuning)
    del S
    info = A.info()
    M = (info["M1"], info["M2"], info["M3"])
    y_meas = _measured_kspace(A, torch, x_true, w.C, dev, Bmax)
    x_hat = torch.from_numpy(synth.ellipsoid_phantom(w.n, w.K, seed=1)).to(dev)
    nsteps = min(args.steps, 20)
    rows = {"workload": workload_desc(w, Bmax).replace(f", coil minibatch B={Bmax}", ""), "grid": list(M),
            "plan_create_s": plan_s, "synth_inputs_s": synth_s, "plan_device_bytes": info["total_bytes"],
            "workspace_bytes": info["workspace_bytes"], "incidences": info["ninc"], "per_batch": {},
            "tuning": dict(A.tuning, spread_bins=list(A.tuning["spread_bins"])), "autotuner": tune_table}
    for B in synth.WHOLE_BRAIN_BATCHES:
        draws = synth.coil_minibatches(w.C, B, nsteps + args.warmup, seed=synth.SEED_COILS_DRAW + 100 + B)
        coil_dev = torch.from_numpy(np.stack(draws)).to(dev)
        g = sdp_graph.DipStepGraph(A, y_meas, x_hat, B)
        for i in range(args.warmup):
            g.step(coil_dev[i])
        graph_ms = _events_ms(torch, lambda i: g.step(coil_dev[args.warmup + i]), nsteps, flush)
        n0 = op.launch_count()
        xg = x_hat.clone().requires_grad_(True)

        def eager(i):
            xg.grad = None
            op.dc_loss(A, xg, coil_dev[args.warmup + i], y_meas).backward()

        A.profile(True)
        A.profile_read()
        eager_ms = _events_ms(torch, eager, nsteps, flush)
        prof = A.profile_read()
        A.profile(False)
        eager_launches = (op.launch_count() - n0) / nsteps
        # accuracy gate against the plain form, then the plain form's time
        ci = coil_dev[0].contiguous()
        loss_b = g.step(ci)[0].clone()
        g_b = g.grad.clone()
        y_b = A.forward(x_hat, ci)
        y_p, loss_p, g_p = _plain_step(A, torch, x_hat, y_meas, ci, w.K)
        torch.cuda.synchronize()
        rel = max(float(torch.linalg.norm(y_p - y_b) / torch.linalg.norm(y_b)),
                  float(torch.linalg.norm(g_p - g_b) / torch.linalg.norm(g_b)),
                  abs(float(loss_p.detach()) - float(loss_b.detach())) / abs(float(loss_b.detach())))
        plain_ms = _events_ms(torch, lambda i: _plain_step(A, torch, x_hat, y_meas, coil_dev[i], w.K), 3, flush)
        model = path_model_bytes(w, B, M)
        stages = {k: v[0] / v[1] for k, v in prof.items() if v[1] > 0}
        sb = stage_bytes(w, B, M, info["ninc"])
        per_kernel = {k: {"ms": stages[k], "alg_bytes": sb[k], "frac_of_hbm": sb[k] / (stages[k] * 1e-3) / (hbm * 1e9)}
                      for k in stages if k in sb}
        rows["per_batch"][str(B)] = {
            "dip_step_ms": {"cuda_graph": graph_ms, "eager": eager_ms},
            "nu_samples_per_s": B * w.J / (graph_ms * 1e-3),
            "path_model": {"bytes_per_step": model, "frac_of_hbm_bound": (model / (hbm * 1e9)) / (graph_ms * 1e-3)},
            "plain_form": {"ms_per_step": plain_ms, "rel_err_vs_plain": rel, "speedup_vs_graph": plain_ms / graph_ms},
            "launches_per_step": {"graph": g.launches_per_step, "eager": eager_launches},
            "kernels": per_kernel}
        del g, xg, coil_dev
        if rel > 1e-4:
            raise SystemExit(f"whole-brain B={B}: batched path differs from the plain form: {rel:.3e}")
    assert A.status() == 0
    # the work list: four items with their own TSMI and coil minibatches of 1, 2, 4 and 8
    xs = [torch.from_numpy(synth.ellipsoid_phantom(w.n, w.K, seed=20 + i)).to(dev)
          for i in range(len(synth.WHOLE_BRAIN_BATCHES))]
    cis = [torch.from_numpy(d[0]).to(dev) for d in
           (synth.coil_minibatches(w.C, B, 1, seed=synth.SEED_COILS_DRAW + 200 + B) for B in synth.WHOLE_BRAIN_BATCHES)]
    ys = [torch.empty((ci.numel(), w.J), dtype=torch.complex64, device=dev) for ci in cis]
    outs = [torch.empty_like(x) for x in xs]

    def worklist(i):
        op.forward_batched([(A, x, ci, y) for x, ci, y in zip(xs, cis, ys)])
        op.adjoint_batched([(A, y, ci, o, False) for y, ci, o in zip(ys, cis, outs)])

    worklist(0)
    n0 = op.launch_count()
    wl_ms = _events_ms(torch, worklist, min(nsteps, 10), flush)
    wl_launches = (op.launch_count() - n0) / min(nsteps, 10)
    nsamp = sum(ci.numel() for ci in cis) * w.J
    model = sum(path_model_bytes(w, ci.numel(), M) for ci in cis)
    rows["work_list"] = {"batches": list(synth.WHOLE_BRAIN_BATCHES), "fwd_adj_ms": wl_ms,
                         "nu_samples_per_s": nsamp / (wl_ms * 1e-3), "launches": wl_launches,
                         "path_model": {"bytes": model, "frac_of_hbm_bound": (model / (hbm * 1e9)) / (wl_ms * 1e-3)}}
    assert A.status() == 0
    A.close()
    del A, y_meas, x_hat, xs, ys, outs
    torch.cuda.empty_cache()
    return rows


def mv_tuning_desc(A):
    return dict(A.tuning, spread_bins=list(A.tuning["spread_bins"]))


def multi_volume_rows(args, torch, op, dev, tuning, flush, hbm):
    """Six independent reconstructions of different matrix sizes (64^3 .. 200x200x160, C in {8,16,32}):
    one DIP step of every volume (coil minibatch C/4 each) as one batched forward, a residual/loss per
    volume and one batched adjoint, captured in a CUDA graph; then the full-coil variant (B = C for
    every volume) against the 150 GB device-memory bound."""
    vols = synth.MULTI_VOLUME
    free0, total = torch.cuda.mem_get_info(dev)
    plans, rows, items = [], [], []
    t0 = time.perf_counter()
    for i, w in enumerate(vols):
        x_true, S, V, omega, frame = synth.make_problem(w)
        A, plan_s = _upload_plan(op, torch, w, omega, frame, V, S, w.C, dev, tuning)
        del S
        y_meas = _measured_kspace(A, torch, x_true, w.C, dev, w.C)
        x_hat = torch.from_numpy(synth.ellipsoid_phantom(w.n, w.K, seed=1)).to(dev).requires_grad_(False)
        draws = synth.coil_minibatches(w.C, w.batch, args.warmup + args.steps, seed=synth.SEED_COILS_DRAW + 300 + i)
        coil_dev = torch.from_numpy(np.stack(draws)).to(dev)
        info = A.info()
        M = (info["M1"], info["M2"], info["M3"])
        plans.append(A)
        items.append(dict(w=w, A=A, y_meas=y_meas, x=x_hat, draws=coil_dev, M=M,
                          ci=torch.empty((w.batch,), dtype=torch.int32, device=dev),
                          yhat=torch.empty((w.batch, w.J), dtype=torch.complex64, device=dev),
                          grad=torch.empty_like(x_hat), loss=torch.empty((), dtype=torch.float32, device=dev)))
        rows.append({"volume": w.name, "image": list(w.n), "grid": list(M), "C": w.C, "B": w.batch, "T": w.T,
                     "J": w.J, "plan_create_s": plan_s, "plan_device_bytes": info["total_bytes"]})
    setup_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)

    def dip_step_all():
        op.forward_batched([(it["A"], it["x"], it["ci"], it["yhat"]) for it in items])
        for it in items:
            it["A"].residual_loss(it["yhat"], it["y_meas"], it["ci"], r2=it["yhat"], loss=it["loss"])
        op.adjoint_batched([(it["A"], it["yhat"], it["ci"], it["grad"], False) for it in items])

    def set_draw(i):
        for it in items:
            it["ci"].copy_(it["draws"][i], non_blocking=True)

    set_draw(0)
    dip_step_all()
    torch.cuda.synchronize()
    # eager (stage times of the batched launches recorded on the first plan), then the same
    # batch on the library's older path for comparison: each plan's nine launches on worker streams
    neager = min(args.steps, 10)
    n0 = op.launch_count()
    plans[0].profile(True)
    plans[0].profile_read()
    eager_ms = _events_ms(torch, lambda i: (set_draw(args.warmup + i), dip_step_all()), neager, flush)
    prof = plans[0].profile_read()
    plans[0].profile(False)
    eager_launches = (op.launch_count() - n0) / neager
    stage_ms = {k: v[0] / neager for k, v in prof.items() if v[1] > 0 and k != "residual_loss"}
    os.environ["SDP_BATCH_STREAMS"] = "1"
    try:
        dip_step_all()
        streams_ms = _events_ms(torch, lambda i: (set_draw(args.warmup + i), dip_step_all()), neager, flush)
    finally:
        del os.environ["SDP_BATCH_STREAMS"]
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(2):
            dip_step_all()
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    n0 = op.launch_count()
    with torch.cuda.graph(gr):
        dip_step_all()
    graph_launches = op.launch_count() - n0
    for i in range(args.warmup):
        set_draw(i)
        gr.replay()
    graph_ms = _events_ms(torch, lambda i: (set_draw(args.warmup + i), gr.replay()), args.steps, flush)
    for p_ in plans:
        assert p_.status() == 0
    nsamp = sum(it["w"].batch * it["w"].J for it in items)
    model = sum(path_model_bytes(it["w"], it["w"].batch, it["M"]) for it in items)
    out = {"volumes": rows, "setup_s": setup_s,
           "dip_step_all_volumes_ms": {"cuda_graph": graph_ms, "eager": eager_ms,
                                       "eager_plan_by_plan_on_worker_streams": streams_ms},
           "batched_stage_ms_per_step": stage_ms,
           "tuning": mv_tuning_desc(items[0]["A"]),
           "nu_samples_per_s": nsamp / (graph_ms * 1e-3),
           "path_model": {"bytes_per_step": model, "frac_of_hbm_bound": (model / (hbm * 1e9)) / (graph_ms * 1e-3)},
           "launches_per_step": {"graph": graph_launches, "eager": eager_launches}}
    del gr
    # full-coil variant: every coil of every volume in one batched forward + adjoint
    full = [dict(it, ci=torch.arange(it["w"].C, dtype=torch.int32, device=dev),
                 yhat=torch.empty((it["w"].C, it["w"].J), dtype=torch.complex64, device=dev)) for it in items]
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info(dev)

    def full_step(i):
        op.forward_batched([(it["A"], it["x"], it["ci"], it["yhat"]) for it in full])
        op.adjoint_batched([(it["A"], it["yhat"], it["ci"], it["grad"], False) for it in full])

    full_step(0)
    full_ms = _events_ms(torch, full_step, 3, flush)
    nfull = sum(it["w"].C * it["w"].J for it in full)
    fmodel = sum(path_model_bytes(it["w"], it["w"].C, it["M"]) for it in full)
    out["full_coil"] = {"fwd_adj_ms": full_ms, "nu_samples_per_s": nfull / (full_ms * 1e-3),
                        "path_model": {"bytes": fmodel, "frac_of_hbm_bound": (fmodel / (hbm * 1e9)) / (full_ms * 1e-3)},
                        "device_used_gb": (total - free2) / 1e9, "bound_gb": 150.0,
                        "within_bound": (total - free2) / 1e9 < 150.0}
    out["device_used_gb"] = {"before": (total - free0) / 1e9, "after_plans": (total - free1) / 1e9,
                             "full_coil_peak": (total - free2) / 1e9}
    for p_ in plans:
        assert p_.status() == 0
        p_.close()
    del plans, items, full
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------------

def run_native(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_02367_gb300 import op

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS[args.workload]
    B = args.batch or w.batch

    x_true, S, V, omega, frame = synth.make_problem(w)
    x_hat = synth.ellipsoid_phantom(w.n, w.K, seed=1)
    # kernel shapes: the framework's autotuner on this trajectory and volume
    tuning, tune_table = None, None
    if args.tuning:
        tuning = json.loads(args.tuning)          # given kernel shapes (reproducible profiling runs)
    elif not args.no_tune:
        from paper_2408_02367_gb300 import tune
        tuning, tune_table = tune.autotune(omega, frame, w.n, w.width, w.oversamp, V, S, max_batch=max(B, 1), B=B,
                                           reps=7, device=dev)
    A = op.make_operator(omega, frame, w.n, w.width, w.oversamp, V, S, max_batch=max(B, 1), device=dev,
                         tuning=tuning)
    info = A.info()
    M = (info["M1"], info["M2"], info["M3"])

    # measured k-space of every coil: A_c(x_true) + complex noise at 30 dB SNR
    xt = torch.from_numpy(x_true).to(dev)
    y_meas = torch.empty((w.C, w.J), dtype=torch.complex64, device=dev)
    for c in range(w.C):
        A.forward(xt, torch.tensor([c], dtype=torch.int32, device=dev), out=y_meas[c:c + 1])
    sig = float(torch.linalg.norm(y_meas).item()) ** 2 / (y_meas.numel() * 1e3)
    y_meas += torch.from_numpy(synth.complex_noise((w.C, w.J), math.sqrt(sig))).to(dev)
    del xt

    nsteps = args.warmup + args.steps
    draws = synth.coil_minibatches(w.C, B, nsteps, seed=rank_seed(synth.SEED_COILS_DRAW, rank))
    coil_dev = torch.from_numpy(np.stack(draws)).to(dev)        # [steps][B], resident
    x = torch.from_numpy(x_hat).to(dev).requires_grad_(True)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def dip_step(ci):
        x.grad = None
        loss = op.dc_loss(A, x, ci, y_meas)
        loss.backward()
        return loss

    # ---- correctness gate vs the plain form (one coil, one channel per launch) ----
    ci0 = coil_dev[0].contiguous()
    loss_b = dip_step(ci0)
    g_b = x.grad.clone()
    y_b = A.forward(x.detach(), ci0)
    y_p = torch.zeros_like(y_b)
    g_p = torch.zeros_like(g_b)

    def plain_step(ci):
        y_p.zero_()
        for b in range(B):
            for k in range(w.K):
                A.forward(x.detach(), ci[b:b + 1], out=y_p[b:b + 1], k0=k, nk=1, accumulate=True)
        r2, lossp = A.residual_loss(y_p, y_meas, ci)
        g_p.zero_()
        for b in range(B):
            for k in range(w.K):
                A.adjoint(r2[b:b + 1].contiguous(), ci[b:b + 1], out=g_p, accumulate=True, k0=k, nk=1)
        return lossp

    loss_p = plain_step(ci0)
    torch.cuda.synchronize()
    rel_y = float(torch.linalg.norm(y_p - y_b) / torch.linalg.norm(y_b))
    rel_g = float(torch.linalg.norm(g_p - g_b) / torch.linalg.norm(g_b))
    rel_l = abs(float(loss_p.detach()) - float(loss_b.detach())) / abs(float(loss_b.detach()))
    assert A.status() == 0
    rel_vs_plain = max(rel_y, rel_g, rel_l)
    if rel_vs_plain > 1e-4:
        raise SystemExit(f"batched path differs from the plain form: {rel_vs_plain:.3e}")

    # ---- eager timed region ----
    def timed(fn, steps, start_index, profile, label="dip_step"):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if profile:
            A.profile(True)
            A.profile_read()
        n0 = op.launch_count()
        # with --profile-range the timed DIP steps run between cudaProfilerStart/Stop
        # (no-ops without a profiler), so `ncu --profile-from-start off` lists exactly
        # their launches, backward included (autograd launches it from its own thread)
        bracket = label == "dip_step" and args.profile_range
        if bracket:
            torch.cuda.profiler.start()
        for i in range(steps):
            flush.fill_(float(i))                # L2 flush, outside the events
            evs[i][0].record()
            fn(coil_dev[start_index + i])
            evs[i][1].record()
        if bracket:
            torch.cuda.profiler.stop()
        torch.cuda.synchronize()
        launches = op.launch_count() - n0
        prof = A.profile_read() if profile else None
        if profile:
            A.profile(False)
        return sum(a.elapsed_time(b) for a, b in evs), launches, prof

    for i in range(args.warmup):
        flush.fill_(0.0)
        dip_step(coil_dev[i])
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    gpu_id = None
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        gpu_id = "GPU-" + str(u)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id).start()
    total_ms, launches, prof = timed(dip_step, args.steps, args.warmup, True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = max_over_ranks(total_ms, dist, dev)
    ms = total_ms / args.steps

    # ---- the same step captured once in a CUDA graph and replayed ----
    from paper_2408_02367_gb300 import graph as sdp_graph
    gstep = sdp_graph.DipStepGraph(A, y_meas, torch.from_numpy(x_hat).to(dev), B)
    for i in range(args.warmup):
        flush.fill_(0.0)
        gstep.step(coil_dev[i])
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        gev[i][0].record()
        gstep.step(coil_dev[args.warmup + i])
        gev[i][1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()      # sampled over both timed regions (eager and graph)
    graph_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in gev), dist, dev) / args.steps
    graph_launches = gstep.launches_per_step * args.steps
    del gstep

    # ---- plain form, same draws, fewer steps ----
    n_plain = min(args.steps, 20)
    plain_ms, plain_launches, _ = timed(plain_step, n_plain, args.warmup, False, label="plain_form")
    plain_ms /= n_plain

    # ---- end to end through the public API with host buffers ----
    xh = torch.from_numpy(x_hat).pin_memory()
    yh = torch.empty((B, w.J), dtype=torch.complex64).pin_memory()
    ch = torch.empty((B,), dtype=torch.int32).pin_memory()
    gh = torch.empty((w.K,) + tuple(w.n), dtype=torch.complex64).pin_memory()
    lh = torch.empty((), dtype=torch.float32).pin_memory()
    ymh = y_meas.cpu()
    meas_rows = torch.arange(B, dtype=torch.int32, device=dev)
    x_e = torch.empty_like(x.detach())
    y_e = torch.empty((B, w.J), dtype=torch.complex64, device=dev)
    c_e = torch.empty((B,), dtype=torch.int32, device=dev)
    n_e2e = min(args.steps, 50)
    e2e_steps = [(draws[args.warmup + i], ymh[torch.from_numpy(draws[args.warmup + i].astype(np.int64))])
                 for i in range(n_e2e)]

    def e2e_step(i):
        # one step at a time: copies in, the step, copies out, wait
        cdraw, ysel = e2e_steps[i]
        ch.copy_(torch.from_numpy(cdraw))
        yh.copy_(ysel)
        c_e.copy_(ch, non_blocking=True)
        y_e.copy_(yh, non_blocking=True)
        x_e.copy_(xh, non_blocking=True)
        x_e.requires_grad_(True)
        x_e.grad = None
        loss = op.dc_loss(A, x_e, c_e, y_e, meas_rows)
        loss.backward()
        gh.copy_(x_e.grad, non_blocking=True)
        lh.copy_(loss.detach(), non_blocking=True)
        torch.cuda.current_stream().synchronize()
        x_e.requires_grad_(False)

    e2e_step(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(n_e2e):
        e2e_step(i)
    e2e_serial_s = (time.perf_counter() - t0) / n_e2e

    # Pipelined: step i's inputs are copied host -> device on one copy stream while step
    # i - 1 computes, and its gradient and loss device -> host on another while step i + 1
    # computes (two slots of device and pinned host buffers, ordered by events).  Every
    # step still moves its own inputs in and its own result out.
    comp = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    xs = [torch.empty_like(x_e) for _ in range(2)]
    ys = [torch.empty_like(y_e) for _ in range(2)]
    cs = [torch.empty_like(c_e) for _ in range(2)]
    yhs = [torch.empty_like(yh).pin_memory() for _ in range(2)]
    chs = [torch.empty_like(ch).pin_memory() for _ in range(2)]
    ghs = [torch.empty_like(gh).pin_memory() for _ in range(2)]
    lhs = [torch.empty_like(lh).pin_memory() for _ in range(2)]
    in_done = [torch.cuda.Event(), torch.cuda.Event()]
    comp_done = [torch.cuda.Event(), torch.cuda.Event()]
    out_done = [torch.cuda.Event(), torch.cuda.Event()]
    grads = [None, None]

    def pipe_in(i):
        q = i % 2
        in_done[q].synchronize()            # step i - 2's copies of these host buffers are done
        cdraw, ysel = e2e_steps[i]
        chs[q].copy_(torch.from_numpy(cdraw))
        yhs[q].copy_(ysel)
        with torch.cuda.stream(s_in):
            s_in.wait_event(comp_done[q])   # step i - 2 no longer reads these device buffers
            cs[q].copy_(chs[q], non_blocking=True)
            ys[q].copy_(yhs[q], non_blocking=True)
            xs[q].copy_(xh, non_blocking=True)
            in_done[q].record(s_in)

    def pipe_step(i):
        q = i % 2
        comp.wait_event(in_done[q])
        xq = xs[q].detach().requires_grad_(True)
        loss = op.dc_loss(A, xq, cs[q], ys[q], meas_rows)
        loss.backward()
        comp_done[q].record(comp)
        out_done[q].synchronize()           # step i - 2's results have reached the host
        grads[q] = (xq.grad, loss.detach())
        with torch.cuda.stream(s_out):
            s_out.wait_event(comp_done[q])
            grads[q][0].record_stream(s_out)
            grads[q][1].record_stream(s_out)
            ghs[q].copy_(grads[q][0], non_blocking=True)
            lhs[q].copy_(grads[q][1], non_blocking=True)
            out_done[q].record(s_out)

    def pipe_run(n):
        pipe_in(0)
        for i in range(n):
            if i + 1 < n:
                pipe_in(i + 1)
            pipe_step(i)
        torch.cuda.synchronize()

    pipe_run(min(n_e2e, 4))
    t0 = time.perf_counter()
    pipe_run(n_e2e)
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_serial_s = max_over_ranks(e2e_serial_s, dist, dev)
    # the pipelined run's last result equals the same step run serially, bit for bit
    e2e_step(n_e2e - 1)
    if not (torch.equal(ghs[(n_e2e - 1) % 2], gh) and torch.equal(lhs[(n_e2e - 1) % 2], lh)):
        raise RuntimeError("pipelined end-to-end step differs from the serial step")
    h2d = xh.numel() * 8 + yh.numel() * 8 + ch.numel() * 4
    d2h = gh.numel() * 8 + 4

    hbm, peak_kind = peaks()

    # ---- whole-brain minibatches and the six-volume batch ----
    scale = {}
    if not args.no_scale_rows:
        scale["whole_brain"] = whole_brain_rows(args, torch, op, dev, tuning, flush, hbm)
        # the six volumes share the whole-brain workload's kernel width and channels: its tuning
        mv_tuning = dict(scale["whole_brain"]["tuning"]) if not args.no_tune else None
        scale["multi_volume"] = multi_volume_rows(args, torch, op, dev, mv_tuning, flush, hbm)

    rows = {}
    if not args.no_operator_rows:
        # ---- rows built on the operator: DCF estimation, SVD-MRF initialiser, CG iteration ----
        from paper_2408_02367_gb300 import recon

        def event_ms(fn, reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fn()
            torch.cuda.synchronize()
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        Ad = recon.dcf_operator(omega, w.n, w.width, w.oversamp, device=dev)
        dcf_iters = 10
        dcf_ms = event_ms(lambda: recon.dcf_pipe_menon(Ad, iters=dcf_iters), 2) / dcf_iters
        dcf = recon.dcf_pipe_menon(Ad, iters=dcf_iters)
        dcf = dcf / dcf.mean()
        del Ad
        init_ms = event_ms(lambda: recon.svd_mrf_init(A, y_meas, dcf), 2)
        cg_iters = 3
        cg_ms = event_ms(lambda: recon.cg_normal(A, y_meas, dcf, iters=cg_iters), 1) / (cg_iters + 1)
        xtv = x.detach()
        tv_grad_buf = torch.empty_like(xtv)
        tv_val_buf = torch.empty((), dtype=torch.float32, device=dev)

        def kernel_ms(fn, reps):
            # device time of the library call alone (its own events), L2 flushed before each call
            fn()
            A.profile_read()
            A.profile(True)
            for i in range(reps):
                flush.fill_(float(i))
                fn()
            A.profile(False)
            torch.cuda.synchronize()
            ms, n = A.profile_read()["tv"]
            return ms / n

        tv_val_ms = kernel_ms(lambda: A.tv_value(xtv, 1e-7, 1e-6, out=tv_val_buf), 20)
        tv_grad_ms = kernel_ms(lambda: A.tv_grad(xtv, 1e-7, 1e-6, out=tv_grad_buf), 20)
        xb = 8.0 * xtv.numel()

        # dictionary matching of the whole TSMI volume against a synthetic MRF dictionary
        from paper_2408_02367_gb300 import dm as dm_mod
        fp, params = synth.mrf_dictionary(480, 128, 96)
        Dm, _ = synth.compress_dictionary(fp, w.K)
        xd_np, _, _ = synth.dm_volume(Dm, w.nvox, noise=0.01, seed=7)
        xd = torch.from_numpy(xd_np.reshape((w.K,) + tuple(w.n))).to(dev)
        del xd_np
        matcher = dm_mod.DictionaryMatcher(torch.from_numpy(Dm).to(dev), max_vox=w.nvox,
                                           params=torch.from_numpy(params).to(dev))
        dm_out = (torch.empty(tuple(w.n), dtype=torch.int32, device=dev),
                  torch.empty(tuple(w.n), dtype=torch.complex64, device=dev),
                  torch.empty(tuple(w.n) + (2,), dtype=torch.float32, device=dev))

        def dm_call():
            matcher.match(xd, out=dm_out, qmap=True)

        dm_call()
        torch.cuda.synchronize()
        dm_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for i, (a_ev, b_ev) in enumerate(dm_ev):
            flush.fill_(float(i))
            a_ev.record()
            dm_call()
            b_ev.record()
        torch.cuda.synchronize()
        dm_ms = sorted(a_ev.elapsed_time(b_ev) for a_ev, b_ev in dm_ev)[len(dm_ev) // 2]
        dm_info = matcher.info()
        dm_status = matcher.status()
        dm_tflops = dm_info["flops_per_voxel"] * w.nvox / (dm_ms * 1e-3) / 1e12
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = float(json.load(f).get("bf16_tflops", 1900.0))
        del matcher, xd, dm_out

        # the full stochastic DIP iteration of Algorithm 1 with the 4-level 3D U-Net generator and Adam
        from paper_2408_02367_gb300 import dip
        torch.backends.cudnn.benchmark = True
        torch.manual_seed(0)
        net = dip.UNet3D(2 * w.K, 2 * w.K).to(dev)
        z = torch.rand((1, 2 * w.K) + tuple(w.n), generator=torch.Generator().manual_seed(1)).mul_(0.1).to(dev)
        runner = dip.DipRunner(A, y_meas, net, z, B=B, lr=1e-3)
        for _ in range(3):
            runner.step()
        torch.cuda.synchronize()
        un_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a_ev, b_ev in un_ev:
            a_ev.record()
            runner.step()
            b_ev.record()
        torch.cuda.synchronize()
        unet_ms = sorted(a_ev.elapsed_time(b_ev) for a_ev, b_ev in un_ev)[len(un_ev) // 2]
        del runner, net, z

        rows = {"dcf_pipe_menon_ms_per_iter": dcf_ms, "svd_mrf_init_ms": init_ms, "cg_ms_per_iter": cg_ms,
                "tv_value_ms": tv_val_ms, "tv_value_gbs": xb / (tv_val_ms * 1e-3) / 1e9,
                "tv_grad_ms": tv_grad_ms, "tv_grad_gbs": 2 * xb / (tv_grad_ms * 1e-3) / 1e9,
                "cg_nu_samples_per_s": w.C * w.J / (cg_ms * 1e-3),
                "dip_unet_step_ms": unet_ms,
                "dip_unet_note": "G(z) by a 4-level 3D U-Net (32..256 channels, cuDNN, TF32 convolutions allowed), "
                                 "DC loss of a coil minibatch through the library, backward, Adam; median of 5",
                "dm_ms": dm_ms, "dm_atoms": int(Dm.shape[0]), "dm_voxels": int(w.nvox),
                "dm_gpairs_per_s": w.nvox * Dm.shape[0] / (dm_ms * 1e-3) / 1e9,
                "dm_tensor_tflops": dm_tflops, "dm_tensor_frac_of_measured_bf16": dm_tflops / bf16_peak,
                "dm_status": dm_status,
                "note": "all C coils per CG iteration in minibatches of B; DCF by Pipe-Menon on the interpolator; "
                        "TV kernels timed alone by the library's stage events, L2 flushed before each call; "
                        "dictionary matching: one match of all voxels (prep + tcgen05 score GEMM + refine), "
                        "median of 5, L2 flushed before each, fp16 tensor flops counted with padding to K=16"}

    # ---- roofline of the dominant kernel ----
    sb = stage_bytes(w, B, M, info["ninc"])
    stages = {k: {"ms_total": v[0], "launches": v[1]} for k, v in prof.items() if v[1] > 0}
    dom = max(stages, key=lambda k: stages[k]["ms_total"])
    avg_ms = stages[dom]["ms_total"] / stages[dom]["launches"]
    per_step = stages[dom]["launches"] / args.steps          # launches of this stage in one step
    bytes_per_launch = sb[dom] / per_step
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    step_share = {k: round(v["ms_total"] / sum(s["ms_total"] for s in stages.values()), 4) for k, v in stages.items()}
    # every stage against the same roofline: algorithmic bytes per launch over its average launch time,
    # beside the ncu DRAM traffic of one launch where a capture of the current kernel exists
    stage_roofline = {}
    for k, v in stages.items():
        if k not in sb:
            continue
        alg = sb[k] / (v["launches"] / args.steps)
        t_ms = v["ms_total"] / v["launches"]
        stage_roofline[k] = {"alg_bytes_per_launch": alg, "avg_launch_ms": t_ms,
                             "achieved_gbs": alg / (t_ms * 1e-3) / 1e9, "frac": alg / (t_ms * 1e-3) / 1e9 / hbm,
                             "traffic": measured_traffic(k, w.name, B, A.tuning)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, B, whole_brain=args.cpu_whole_brain)

    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0
    model = path_model_bytes(w, B, M)
    # headline: the step as a training loop runs it, captured in a CUDA graph
    best_ms = graph_ms
    value = ws * B * w.J / (best_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": best_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc(w, B), "grid": list(M), "l2": "flushed between steps "
                   f"({FLUSH_BYTES >> 20} MiB write outside the timed events)", "timed": "CUDA-graph replay "
                   "of the whole step (eager step reported in dip_step_ms)", "parallelism":
                   "replicas" if ws > 1 else "single GPU", "coil_draws": "uniform without replacement, "
                   "pre-drawn and resident on the device"},
        "dip_step_ms": {"eager": ms, "cuda_graph": graph_ms},
        "plain_form": {"ms_per_step": plain_ms, "launches_per_step": plain_launches / n_plain,
                       "rel_err_vs_plain": rel_vs_plain, "speedup_vs_eager": plain_ms / ms,
                       "speedup_vs_graph": plain_ms / graph_ms},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": peak_kind,
                     "traffic": measured_traffic(dom, w.name, B, A.tuning),
                     "alg_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
                     "launches_per_step": per_step},
        "stage_ms_per_step": {k: v["ms_total"] / args.steps for k, v in stages.items()},
        "stage_share": step_share,
        "stage_roofline": stage_roofline,
        "path_model": {"bytes_per_step": model, "frac_of_hbm_bound": (model / (hbm * 1e9)) / (best_ms * 1e-3)},
        "operator_rows": rows,
        "scale_rows": scale,
        "tuning": {"chosen": dict(A.tuning, spread_bins=list(A.tuning["spread_bins"])),
                   "autotuner": tune_table, "note": "forward + adjoint of one coil minibatch per candidate, "
                   "median of 7 with L2 flushed; every candidate checked against the first to 1e-5"},
        "cpu_baseline": cpu,
        "e2e": {"value": ws * B * w.J / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3, "steps": n_e2e,
                "serial_ms_per_step": e2e_serial_s * 1e3,
                "note": "dc_loss + backward through the public API; every step copies its inputs from pinned host "
                        "memory and its gradient and loss back; the value pipelines the copies of neighbouring "
                        "steps on two copy streams against the compute (serial_ms_per_step: copy, step, copy, "
                        "wait)"},
        "gpu_launches": graph_launches,
        "gpu_launches_eager_region": launches,
        "clocks": clk,
    }
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="vol128_w4", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="default kernel shapes instead of the autotuner's")
    ap.add_argument("--tuning", default="", help="kernel shapes as JSON (sdp_tuning fields) instead of the autotuner's")
    ap.add_argument("--cpu-whole-brain", action="store_true",
                    help="also time one coil x all K of the 200x200x160 workload on the CPU oracle")
    ap.add_argument("--no-scale-rows", action="store_true",
                    help="skip the whole-brain minibatch rows and the six-volume batch")
    ap.add_argument("--no-operator-rows", action="store_true",
                    help="skip the rows built on the operator (DCF, SVD-MRF, CG, TV, dictionary matching, U-Net step)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed DIP steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
