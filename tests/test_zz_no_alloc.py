"""The allocation-free residual/loss entry point against the plan-based one.

sdp_residual_loss_noalloc serves callers that cannot call cudaMalloc (and so
cannot create a plan): its scratch is a fixed array inside the library image.
This checks, through the C ABI, that it returns the same r2 = 2 (yhat - y_meas)
and the same loss as sdp_residual_loss on two calls in a row (the second call
sees the scratch the first one left behind), and that a size above its fixed
maximum is refused before any work is queued.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2408_02367_gb300 import synth

pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-6      # both add a few |r|^2 in float32 (4 here, up to 128 in the plan kernel), then float64


@pytest.fixture(scope="module")
def lib():
    from paper_2408_02367_gb300 import build, op
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return op


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_loss_matches_plan_loss_on_two_calls(lib):
    op = lib
    dev = torch.device("cuda", 0)
    n, T, C, B = (8, 8, 8), 3, 3, 2
    J = 100_003                                   # two rows -> 4 chunks, ragged last chunk
    rng = np.random.default_rng(0)
    omega = rng.uniform(-np.pi, np.pi, size=(J, 3)).astype(np.float32)
    frame = np.sort(rng.integers(0, T, size=J)).astype(np.int32)
    A = op.make_operator(omega, frame, n, 4, 2.0, synth.subspace_basis(T, 2), synth.coil_maps(n, C), B,
                         device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        yhat = torch.from_numpy(synth.random_complex((B, J), 10 + call)).to(dev)
        y_meas = torch.from_numpy(synth.random_complex((C, J), 20 + call)).to(dev)
        rows = torch.tensor([2, 0] if call == 0 else [1, 1], dtype=torch.int32, device=dev)
        r2_ref, loss_ref = A.residual_loss(yhat, y_meas, rows)
        r2 = torch.full((B, J), float("nan"), dtype=torch.complex64, device=dev)
        loss = torch.full((), float("nan"), dtype=torch.float32, device=dev)
        rc = op.lib().sdp_residual_loss_noalloc(_ptr(yhat), _ptr(y_meas), C, _ptr(rows), B, J, _ptr(r2),
                                                _ptr(loss), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(r2, r2_ref)
        lr, l = float(loss_ref), float(loss)
        assert abs(l - lr) / lr < LOSS_RTOL, (call, l, lr)
    assert A.status() == 0


def test_noalloc_rejects_sizes_above_its_scratch(lib):
    op = lib
    dev = torch.device("cuda", 0)
    buf = torch.zeros(4, dtype=torch.complex64, device=dev)
    rows = torch.zeros(2, dtype=torch.int32, device=dev)
    loss = torch.zeros((), dtype=torch.float32, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    too_many = (1 << 28) // 2 + 1                 # B * J = 2^28 + 2 entries
    rc = op.lib().sdp_residual_loss_noalloc(_ptr(buf), _ptr(buf), 1, _ptr(rows), 2, too_many, _ptr(buf),
                                            _ptr(loss), stream)
    assert rc == 1                                # SDP_ERR_INVALID_ARG, nothing launched


@pytest.mark.parametrize("B,J", [(1, (1 << 16) + 1), (3, 1 << 16), (5, 3)])
def test_noalloc_chunk_and_row_boundaries(lib, B, J):
    """A row one past a chunk (ragged last chunk of one entry), rows that end exactly on chunk
    boundaries, and rows shorter than a thread's stride (the row index advances by several rows
    per step): the same residual and loss as the plan-based entry point."""
    op = lib
    dev = torch.device("cuda", 0)
    n, T, C = (8, 8, 8), 2, 4
    rng = np.random.default_rng(B * 7 + J)
    omega = rng.uniform(-np.pi, np.pi, size=(J, 3)).astype(np.float32)
    frame = np.sort(rng.integers(0, T, size=J)).astype(np.int32)
    A = op.make_operator(omega, frame, n, 4, 2.0, synth.subspace_basis(T, 2), synth.coil_maps(n, C), B, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    yhat = torch.from_numpy(synth.random_complex((B, J), 31)).to(dev)
    y_meas = torch.from_numpy(synth.random_complex((C, J), 32)).to(dev)
    rows = torch.from_numpy(rng.integers(0, C, size=B).astype(np.int32)).to(dev)
    r2_ref, loss_ref = A.residual_loss(yhat, y_meas, rows)
    r2 = torch.full((B, J), float("nan"), dtype=torch.complex64, device=dev)
    loss = torch.full((), float("nan"), dtype=torch.float32, device=dev)
    assert op.lib().sdp_residual_loss_noalloc(_ptr(yhat), _ptr(y_meas), C, _ptr(rows), B, J, _ptr(r2),
                                              _ptr(loss), stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(r2, r2_ref)
    assert abs(float(loss) - float(loss_ref)) / float(loss_ref) < LOSS_RTOL
    assert A.status() == 0


def test_noalloc_at_its_maximum_size(lib):
    """B * J = SDP_NOALLOC_MAX_ELEMS exactly: every one of the fixed scratch's 4096 chunk partials is
    used.  A plan for 2^28 samples is out of reach, so the check is against the definition:
    r2 = 2 (yhat - y_meas[row]) bit for bit, and the loss against a float64 sum."""
    op = lib
    dev = torch.device("cuda", 0)
    total = 1 << 28
    B, J = 2, total // 2
    g = torch.Generator(device=dev).manual_seed(5)
    yhat = torch.randn((B, J), dtype=torch.complex64, device=dev, generator=g)
    y_meas = torch.randn((1, J), dtype=torch.complex64, device=dev, generator=g)
    rows = torch.zeros((B,), dtype=torch.int32, device=dev)
    r2 = torch.empty_like(yhat)
    loss = torch.full((), float("nan"), dtype=torch.float32, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    assert op.lib().sdp_residual_loss_noalloc(_ptr(yhat), _ptr(y_meas), 1, _ptr(rows), B, J, _ptr(r2),
                                              _ptr(loss), stream) == 0
    torch.cuda.synchronize()
    d = yhat - y_meas
    assert torch.equal(r2, 2 * d)
    ref = float(torch.sum(torch.view_as_real(d).to(torch.float64) ** 2))
    del d
    assert abs(float(loss) - ref) / ref < LOSS_RTOL
