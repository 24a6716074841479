"""The C ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares; host-only entry points answer correctly."""
import ctypes
import os
import re

import pytest

from oracle import nufft as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_02367_gb300 import build, op
    build.build()
    return op.lib()


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sdp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ["sdp_plan_create", "sdp_plan_destroy", "sdp_forward", "sdp_adjoint", "sdp_forward_batched",
                 "sdp_adjoint_batched", "sdp_status", "sdp_workspace_bytes", "sdp_strerror",
                 "sdp_residual_loss", "sdp_adjoint_scaled", "sdp_dm_create", "sdp_dm_match", "sdp_dm_destroy"]:
        assert need in names


def test_every_declared_function_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2408_02367_gb300 import op
    assert set(op.EXPORTS) <= set(declared_functions())


def test_status_strings_and_counters_without_gpu(lib):
    for code in range(7):
        assert lib.sdp_strerror(code)
    assert lib.sdp_launch_count() >= 0
    assert lib.sdp_workspace_bytes(None) == 0
    assert lib.sdp_plan_beta(None) == -1.0


def test_plan_create_rejects_bad_arguments_on_the_host(lib):
    from paper_2408_02367_gb300 import op
    h = ctypes.c_void_p(1234)
    assert lib.sdp_plan_create(ctypes.byref(h), None, None) == 1
    assert h.value is None
    d = op.PlanDesc()
    d.n = (ctypes.c_int64 * 3)(16, 16, 1)       # N3 < 2
    assert lib.sdp_plan_create(ctypes.byref(h), ctypes.byref(d), None) == 1
    assert lib.sdp_forward(None, None, None, 1, None, None) == 1
    assert lib.sdp_forward_batched(None, 0, None) == 0
    assert lib.sdp_residual_loss_noalloc(None, None, 1, None, 1, 1, None, None, None) == 1


def test_plan_create_refuses_oversized_grids_before_any_device_call(lib):
    """A plan whose per-coil grid would need 64-bit offsets (M1 M2 M3 K >= 2^31) or whose grid
    length exceeds 2^14 along an axis is refused with SDP_ERR_UNSUPPORTED on the host, before the
    first CUDA call (so also here, without a GPU) and before anything is read from the trajectory,
    V or the coil maps; a descriptor within the limits gets past the check to that first call."""
    import numpy as np
    from paper_2408_02367_gb300 import op
    assert [lib.sdp_grid_size(v, 1.25, 4) for v in (1024, 640, 20000)] == [1280, 800, 25000]
    off = np.array([0, 4], dtype=np.int64)
    dummy = np.zeros(64, dtype=np.float32)     # never read: stands in for device buffers

    def create(n, K):
        d = op.PlanDesc()
        d.n = (ctypes.c_int64 * 3)(*n)
        d.oversamp, d.width, d.K, d.T, d.C, d.J, d.max_batch, d.flags = 1.25, 4, K, 1, 1, 4, 1, 0
        d.frame_offsets = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.traj = d.V = d.coil_maps = dummy.ctypes.data
        h = ctypes.c_void_p(1234)
        rc = lib.sdp_plan_create(ctypes.byref(h), ctypes.byref(d), None)
        assert h.value is None
        return rc

    # M = 1280 per axis with K = 2 (G K = 4.2e9), 800 with K = 5 (G K = 2.56e9), 25000 along one axis
    for n, K in (((1024, 1024, 1024), 2), ((640, 640, 640), 5), ((20000, 2, 2), 1)):
        assert create(n, K) == 6
    # the descriptors below pass the size check and would go on to copy from the stand-in
    # buffers, so they are only made where there is no device: M = 1280 with K = 1
    # (G = 2.10e9 < 2^31) and M = 640 with K = 5 (G K = 1.3e9)
    import torch
    if not torch.cuda.is_available():
        assert create((1024, 1024, 1024), 1) == 3     # on to cudaGetDevice, which fails here
        assert create((512, 512, 512), 5) == 3


def test_every_autotuner_candidate_passes_the_tuning_checks(lib):
    """Each tuning the autotuner proposes (both rounds, with every first-round spread shape as the
    base of the second; the library's lists and the bench's whole-brain lists) gets past the library's host-side tuning checks: with a descriptor inside
    every limit, plan creation reaches its first CUDA call, which fails here without a device.  (On
    a machine with a device the descriptor's stand-in buffers would be read, so the test skips.)"""
    import numpy as np
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("the stand-in buffers must not reach a device")
    from paper_2408_02367_gb300 import op, tune
    off = np.array([0, 4], dtype=np.int64)
    dummy = np.zeros(64, dtype=np.float32)
    d = op.PlanDesc()
    d.n = (ctypes.c_int64 * 3)(16, 16, 16)
    d.oversamp, d.width, d.K, d.T, d.C, d.J, d.max_batch, d.flags = 1.25, 4, 5, 1, 1, 4, 2, 0
    d.frame_offsets = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.traj = d.V = d.coil_maps = dummy.ctypes.data
    import bench
    first = tune.candidates(full=True)
    tunings = first + [t for base in first for t in tune.refinements(dict(tune.DEFAULT, **base))]
    wb = bench.WHOLE_BRAIN_CANDIDATES
    tunings += wb + [t for base in wb for t in tune.refinements(dict(tune.DEFAULT, **base),
                                                                   bench.WHOLE_BRAIN_REFINE)]
    assert len(tunings) > 100
    for t in tunings:
        h = ctypes.c_void_p(1234)
        tt = op.Tuning.of(t)
        assert lib.sdp_plan_create_tuned(ctypes.byref(h), ctypes.byref(d), ctypes.byref(tt), None) == 3, t
        assert h.value is None


@pytest.mark.parametrize("n,sigma,W", [(32, 2.0, 6), (128, 1.25, 4), (200, 1.25, 4), (160, 1.25, 4),
                                       (14, 2.0, 6), (3, 2.0, 8), (97, 1.5, 5), (24, 1.0, 4)])
def test_grid_size_and_beta_agree_with_the_oracle(lib, n, sigma, W):
    assert lib.sdp_grid_size(n, sigma, W) == O.grid_size(n, sigma, W)
    assert abs(lib.sdp_kb_beta(W, sigma) - O.beatty_beta(W, sigma)) < 1e-12


def test_grid_size_rejects_out_of_range(lib):
    assert lib.sdp_grid_size(0, 2.0, 4) == -1
    assert lib.sdp_grid_size(10, 0.5, 4) == -1
    assert lib.sdp_grid_size(10, 2.0, 9) == -1
    assert lib.sdp_kb_beta(2, 1.0) > 0 or lib.sdp_kb_beta(2, 1.0) == -1.0


def test_dictionary_matcher_rejects_bad_arguments_on_the_host(lib):
    h = ctypes.c_void_p(1234)
    assert lib.sdp_dm_create(None, None, None, 1, 1, 1, None) == 1
    assert lib.sdp_dm_create(ctypes.byref(h), None, None, 10, 5, 100, None) == 1
    assert h.value is None
    assert lib.sdp_dm_create(ctypes.byref(h), ctypes.c_void_p(16), None, 10, 17, 100, None) == 1   # K > 16
    assert lib.sdp_dm_create(ctypes.byref(h), ctypes.c_void_p(16), None, 0, 5, 100, None) == 1     # P < 1
    assert lib.sdp_dm_match(None, None, 0, None, None, None, None) == 1
    assert lib.sdp_dm_status(None, None) == 1
    buf = (ctypes.c_int64 * 8)()
    assert lib.sdp_dm_info(None, buf, 8) == 1
    lib.sdp_dm_destroy(None)


def test_tuned_plan_rejects_bad_tunings_on_the_host(lib):
    from paper_2408_02367_gb300 import op
    h = ctypes.c_void_p(1234)
    t = op.Tuning.of({"spread_bins": (8, 4, 8), "spread_chunk": 16})          # chunk below 32
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    assert h.value is None
    t = op.Tuning.of({"spread_bins": (8, 8, 8)})                               # no kernel for this shape
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 6
    t = op.Tuning.of({"fft_engine": 2})
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    t = op.Tuning.of({"fft_lines": 12})                                       # 0, 8 or 4 only
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    t = op.Tuning.of({"fft_cols": 16})                                        # 0, 32 or 8 only
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    t = op.Tuning.of({"interp_threads": 512})                                 # 0, 256 or 1024 only
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    t = op.Tuning.of({"spread_coils": 3})                                     # 0, 1 or 2 only
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    t = op.Tuning.of({"interp_run": 3})                                       # 0, 1, 2, 4 or 8 only
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    t = op.Tuning.of({"interp_coils": -1})                                    # 0 .. 64
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    t = op.Tuning.of({"fft_staged": 4})                                       # bit mask of 2 bits
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    t = op.Tuning.of({"interp_tiled": 2})                                     # 0 or 1
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    t = op.Tuning.of({"spread_bins": (2, 4, 4)})                               # no kernel for this shape
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 6
    t = op.Tuning.of({})                                                       # valid tuning, no descriptor
    assert lib.sdp_plan_create_tuned(ctypes.byref(h), None, ctypes.byref(t), None) == 1
    assert lib.sdp_plan_tuning(None, ctypes.byref(t)) == 1
