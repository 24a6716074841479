"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (relative L2 over the whole output):
  W=6, sigma=2     1e-4   (the operator's stated FP32-vs-FP64 bound)
  W=4, sigma=1.25  2e-3   (same)
  every case       FP32_BOUND = 2e-5, derived in the design notes from float32
                   rounding of the taps, the FFT and the subspace contraction
                   (a few ulps times log2(G) stages, measured ~1e-6); it is the
                   bound that catches a dropped tap or a wrong twiddle.
  sigma = 1        the adjoint divides by psi_hat, which falls ~200x per axis
                   from the centre to the edge of the image without
                   oversampling; float32 rounding of the grid (relative to its
                   largest value) is amplified by that ratio at the corners, so
                   that adjoint gets the looser SIGMA1_ADJ_BOUND.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nufft as O
from paper_2408_02367_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_BOUND = 2e-5
SIGMA1_ADJ_BOUND = 2e-2


def stated_tol(W, sigma):
    return 1e-4 if (W >= 6 and sigma >= 2.0) else 2e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2408_02367_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


ELEM_FACTOR = 10.0    # element-wise bound = ELEM_FACTOR x the relative-L2 bound of the case


def elem(a, b):
    """Largest element error relative to the largest reference magnitude, and where it sits."""
    d = np.abs(np.asarray(a) - np.asarray(b)).ravel()
    i = int(np.argmax(d))
    return float(d[i] / np.max(np.abs(np.asarray(b)))), np.unravel_index(i, np.shape(b))


def assert_close(a, b, bound, what=""):
    """Relative L2 below `bound` and every element within ELEM_FACTOR * bound of max |b|: a few
    hundred wrong samples (a bad wrap at the grid edge, one bad bin) cannot hide under the norm."""
    e2 = rel(a, b)
    ee, where = elem(a, b)
    print(f"{what}: rel L2 {e2:.2e}, worst element {ee:.2e} at {tuple(int(v) for v in where)}")
    assert e2 < bound, (what, e2)
    assert ee < ELEM_FACTOR * bound, (what, ee, where)


def make_case(n, W, sigma, K, C, T, arms, arm_len, coils, seed=0, real_V=False):
    x = synth.ellipsoid_phantom(n, K, seed=seed)
    S = synth.coil_maps(n, C)
    V = synth.subspace_basis(T, K, real=real_V)
    omega, frame = synth.spiral_trajectory(T, arms, arm_len)
    return dict(n=tuple(n), W=W, sigma=sigma, x=x, S=S, V=V, omega=omega, frame=frame,
                coils=np.asarray(coils, np.int32))


def gpu_op(c, max_batch=None):
    from paper_2408_02367_gb300 import op
    mb = max_batch or len(c["coils"])
    return op.make_operator(c["omega"], c["frame"], c["n"], c["W"], c["sigma"], c["V"], c["S"], mb)


def t(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = {
    # name: (n, W, sigma, K, C, T, arms, arm_len, coils)
    "vol32_w6_full": ((32, 32, 32), 6, 2.0, 5, 4, 100, 1, 512, [0, 1, 2, 3]),
    "ragged_w4": ((20, 18, 22), 4, 1.25, 3, 3, 7, 2, 300, [2, 0]),
    "odd_w5": ((16, 16, 16), 5, 1.5, 2, 2, 4, 1, 500, [1, 1]),
    "w8_k16": ((12, 14, 10), 8, 2.0, 16, 2, 20, 1, 200, [1]),
    "w2": ((10, 10, 10), 2, 1.25, 2, 2, 3, 1, 300, [0, 1]),
    "sigma1_w4": ((16, 16, 16), 4, 1.0, 3, 2, 5, 1, 400, [1, 0]),
    "w6_anisotropic": ((24, 16, 8), 6, 2.0, 4, 3, 10, 1, 256, [2, 1, 0]),
    # grid lengths served by the two-pass register FFT (axis 3 = fused prologue / epilogue)
    "fft2_160_axis3": ((8, 16, 128), 4, 1.25, 5, 2, 12, 1, 512, [1, 0]),
    "fft2_120_80": ((96, 8, 64), 4, 1.25, 2, 2, 6, 1, 300, [0, 1]),
    "fft2_250_axis1": ((200, 8, 10), 4, 1.25, 3, 2, 5, 1, 300, [1]),
    "fft2_200_250": ((8, 160, 200), 4, 1.25, 2, 2, 4, 1, 300, [0, 1]),
    "fft2_240_256": ((120, 8, 128), 4, 2.0, 1, 1, 3, 1, 200, [0]),
    # channel groups: interpolation runs 32 // W channels per launch (W=6: 5 + 2),
    # the spread 8 per launch (K=10: 8 + 2, 8-byte column stores); three coils at
    # W=4 take interpolation's two-coil gather round and its one-coil tail
    "w6_k7_groups": ((18, 20, 16), 6, 2.0, 7, 2, 9, 1, 300, [1, 0]),
    "w4_k10_groups": ((16, 16, 16), 4, 1.25, 10, 2, 12, 1, 400, [0, 1, 1]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_forward_and_adjoint_match_oracle(name):
    n, W, sigma, K, C, T, arms, arm_len, coils = CASES[name]
    c = make_case(n, W, sigma, K, C, T, arms, arm_len, coils)
    geo = O.Geometry(c["n"], W, sigma)
    A = gpu_op(c)
    assert A.grid == geo.M
    assert abs(A.beta - geo.beta) < 1e-12
    y_ref = O.gridding_forward(geo, c["x"], c["S"], c["V"], c["omega"], c["frame"], c["coils"])
    y = A.forward(t(c["x"]), t(c["coils"])).cpu().numpy()
    r = synth.random_complex(y_ref.shape, 99)
    a_ref = O.gridding_adjoint(geo, r, c["S"], c["V"], c["omega"], c["frame"], c["coils"])
    a = A.adjoint(t(r), t(c["coils"])).cpu().numpy()
    assert A.status() == 0
    assert FP32_BOUND <= stated_tol(W, sigma)
    assert_close(y, y_ref, FP32_BOUND, f"{name} M={geo.M} forward")
    assert_close(a, a_ref, SIGMA1_ADJ_BOUND if sigma == 1.0 else FP32_BOUND, f"{name} adjoint")


def test_generic_fft_engine_matches_oracle(tmp_path):
    """The Stockham fallback (forced by SDP_FFT_GENERIC=1 in a child process) on a
    length the two-pass engine normally serves."""
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, sys\n"
        "sys.path.insert(0, '.')\n"
        "from tests.test_gpu_parity import make_case, gpu_op, t, rel, FP32_BOUND\n"
        "from oracle import nufft as O\n"
        "c = make_case((8, 16, 128), 4, 1.25, 3, 2, 6, 1, 300, [1, 0])\n"
        "geo = O.Geometry(c['n'], 4, 1.25)\n"
        "A = gpu_op(c)\n"
        "y = A.forward(t(c['x']), t(c['coils'])).cpu().numpy()\n"
        "from tests.test_gpu_parity import assert_close\n"
        "assert_close(y, O.gridding_forward(geo, c['x'], c['S'], c['V'], c['omega'], c['frame'], c['coils']),"
        " FP32_BOUND, 'Stockham forward')\n"
        "r = np.ascontiguousarray(y)\n"
        "a = A.adjoint(t(r), t(c['coils'])).cpu().numpy()\n"
        "assert_close(a, O.gridding_adjoint(geo, r, c['S'], c['V'], c['omega'], c['frame'], c['coils']),"
        " FP32_BOUND, 'Stockham adjoint')\n")
    import os
    env = dict(os.environ, SDP_FFT_GENERIC="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("tuning", [
    {"spread_bins": (8, 4, 4), "spread_chunk": 64, "fft_engine": 0},
    {"spread_bins": (8, 4, 8), "spread_chunk": 32, "fft_engine": 1},
    {"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8},
    {"spread_bins": (8, 4, 8), "spread_chunk": 256, "fft_engine": 0, "fft_lines": 4},
    {"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8, "fft_cols": 32},
    {"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 0, "fft_cols": 8},
    {"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8, "interp_threads": 256},
    {"spread_bins": (8, 4, 8), "spread_chunk": 512, "fft_engine": 0, "interp_threads": 1024},
    {"spread_bins": (8, 4, 4), "spread_chunk": 64, "fft_engine": 0, "spread_coils": 1},
    {"spread_bins": (8, 4, 4), "spread_chunk": 64, "fft_engine": 0, "spread_coils": 2},
    {"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "interp_threads": 1024, "interp_run": 2,
     "interp_coils": 2},
    {"spread_bins": (8, 4, 8), "spread_chunk": 512, "fft_engine": 0, "interp_run": 8, "interp_coils": 1},
    {"spread_bins": (4, 4, 4), "spread_chunk": 64, "fft_engine": 0},
    {"spread_bins": (4, 4, 8), "spread_chunk": 32, "fft_engine": 0},
    {"spread_bins": (4, 4, 4), "spread_chunk": 512, "fft_engine": 0, "spread_coils": 1},
    {"spread_bins": (4, 4, 8), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8, "interp_threads": 1024},
    {"spread_bins": (4, 4, 4), "spread_chunk": 512, "fft_engine": 0, "interp_tiled": 1},
    {"spread_bins": (8, 4, 8), "spread_chunk": 64, "fft_engine": 0, "interp_tiled": 1, "fft_staged": 1},
    {"spread_bins": (4, 4, 4), "spread_chunk": 64, "fft_engine": 0, "interp_tiled": 1, "fft_staged": 2},
])
def test_tuned_kernel_shapes_match_oracle(tuning):
    """Every tuning computes the same operator: half-depth spread bins, 4 x 4 bins (two
    incidences per warp step), short spread chunks (many multi-chunk bins), one or two
    coils per spread warp (three coils: a pair and an odd tail) and the Stockham FFT
    engine, forward and adjoint."""
    from paper_2408_02367_gb300 import op
    c = make_case((20, 18, 16), 4, 1.25, 3, 3, 10, 1, 600, [2, 0, 1])
    geo = O.Geometry(c["n"], 4, 1.25)
    A = op.make_operator(c["omega"], c["frame"], c["n"], 4, 1.25, c["V"], c["S"], max_batch=3, tuning=tuning)
    assert A.tuning["spread_bins"] == tuple(tuning["spread_bins"]) and A.tuning["spread_chunk"] == tuning["spread_chunk"]
    assert A.tuning["interp_threads"] == (tuning.get("interp_threads") or 256)      # 256 by default
    y = A.forward(t(c["x"]), t(c["coils"])).cpu().numpy()
    assert_close(y, O.gridding_forward(geo, c["x"], c["S"], c["V"], c["omega"], c["frame"], c["coils"]), FP32_BOUND,
                 f"{tuning} forward")
    r = np.ascontiguousarray(y)
    a = A.adjoint(t(r), t(c["coils"])).cpu().numpy()
    assert_close(a, O.gridding_adjoint(geo, r, c["S"], c["V"], c["omega"], c["frame"], c["coils"]), FP32_BOUND,
                 f"{tuning} adjoint")
    assert A.status() == 0


@pytest.mark.parametrize("bins", [(8, 4, 8), (8, 4, 4), (4, 4, 8), (4, 4, 4)])
def test_spread_bins_on_a_short_axis3_grid(bins):
    """A 4-point image axis at W=6 gets a 12-point axis-3 grid, shorter than an 8-deep bin
    plus a window (B3 + W - 1 = 13): a window can meet a bin in two pieces along axis 3, and
    the spread then runs every position of the column instead of one class's run.  4-deep
    bins still fit (9 <= 12) and take the class runs on a grid of three bins.  The adjoint
    matches the oracle either way."""
    from paper_2408_02367_gb300 import op
    c = make_case((16, 12, 4), 6, 2.0, 5, 2, 6, 1, 300, [1, 0, 1])
    geo = O.Geometry(c["n"], 6, 2.0)
    A = op.make_operator(c["omega"], c["frame"], c["n"], 6, 2.0, c["V"], c["S"], max_batch=3,
                         tuning={"spread_bins": bins, "spread_chunk": 64})
    assert A.grid[2] == 12 and (A.grid[2] < bins[2] + 6 - 1) == (bins[2] == 8)
    r = synth.random_complex((3, A.J), 5)
    a = A.adjoint(t(r), t(c["coils"])).cpu().numpy()
    assert_close(a, O.gridding_adjoint(geo, r, c["S"], c["V"], c["omega"], c["frame"], c["coils"]), FP32_BOUND,
                 f"{bins} short axis 3 adjoint")
    assert A.status() == 0


def test_half_warp_bins_with_channel_groups():
    """4 x 4 x 4 bins with K=10 channels: a group of 8 (one coil per warp) and a group of 2
    (coil pairs), 8-byte column stores, short chunks; three coils."""
    from paper_2408_02367_gb300 import op
    c = make_case((16, 16, 16), 4, 1.25, 10, 2, 12, 1, 400, [0, 1, 1])
    geo = O.Geometry(c["n"], 4, 1.25)
    A = op.make_operator(c["omega"], c["frame"], c["n"], 4, 1.25, c["V"], c["S"], max_batch=3,
                         tuning={"spread_bins": (4, 4, 4), "spread_chunk": 64})
    r = synth.random_complex((3, A.J), 6)
    a = A.adjoint(t(r), t(c["coils"])).cpu().numpy()
    assert_close(a, O.gridding_adjoint(geo, r, c["S"], c["V"], c["omega"], c["frame"], c["coils"]), FP32_BOUND,
                 "4x4x4 bins, K=10 adjoint")
    assert A.status() == 0


@pytest.mark.parametrize("n,W,sigma,K,coils", [((40, 36, 44), 4, 1.25, 5, [2, 0, 1]),
                                               ((24, 20, 16), 2, 2.0, 8, [1, 0]),
                                               ((20, 18, 16), 6, 2.0, 3, [0, 1]),
                                               ((18, 16, 12), 4, 1.25, 10, [1, 0])])
def test_tiled_interpolation_matches_oracle(n, W, sigma, K, coils):
    """The tiled interpolation (8^3 tiles with their window margin in shared memory): W=4 with
    partial edge tiles and three coils, W=2 with 8 channels, and the row kernel where the tiled one
    has no kernel (W=6; K=10 > 8 channels per call), all with interp_tiled=1; plus a channel
    subset (k0 > 0) and accumulate into an existing output."""
    from paper_2408_02367_gb300 import op
    c = make_case(n, W, sigma, K, 3, 12, 1, 500, coils)
    geo = O.Geometry(c["n"], W, sigma)
    A = op.make_operator(c["omega"], c["frame"], c["n"], W, sigma, c["V"], c["S"], max_batch=3,
                         tuning={"interp_tiled": 1})
    assert A.tuning["interp_tiled"] == 1
    y = A.forward(t(c["x"]), t(c["coils"])).cpu().numpy()
    assert_close(y, O.gridding_forward(geo, c["x"], c["S"], c["V"], c["omega"], c["frame"], c["coils"]), FP32_BOUND,
                 f"tiled interpolation n={n} W={W} K={K}")
    if K >= 3:
        # channels 1 .. K-2 added onto a copy of the channel-0 and channel-(K-1) parts
        ci = t(c["coils"])
        xs = t(c["x"])
        yk = A.forward(xs, ci, k0=0, nk=1)
        A.forward(xs, ci, out=yk, accumulate=True, k0=K - 1, nk=1)
        A.forward(xs, ci, out=yk, accumulate=True, k0=1, nk=K - 2)
        assert_close(yk.cpu().numpy(), y, FP32_BOUND, "tiled interpolation, channel subsets")
    assert A.status() == 0


def test_tiled_interpolation_bounded_wait_runs_out_then_recovers():
    """The tiled interpolation's wait for a tile's bulk copies is bounded: with one row of the
    first CTA's first tile withheld (the test hook) and a 20 ms limit, the forward reports
    SDP_ERR_TIMEOUT instead of hanging, the device stays usable, and with the hook off the next
    forward matches the oracle.  Invalid hook arguments are refused on the host."""
    from paper_2408_02367_gb300 import op
    c = make_case((40, 36, 44), 4, 1.25, 5, 3, 12, 1, 500, [2, 0])
    geo = O.Geometry(c["n"], 4, 1.25)
    A = op.make_operator(c["omega"], c["frame"], c["n"], 4, 1.25, c["V"], c["S"], max_batch=2,
                         tuning={"interp_tiled": 1})
    with pytest.raises(op.SdpError):
        A.set_wait_test(144)                       # rows 0 .. 143 of a 12 x 12 tile face
    with pytest.raises(op.SdpError):
        A.set_wait_test(3, timeout_ns=10)          # limit below 1 us
    x, ci = t(c["x"]), t(c["coils"])
    A.set_wait_test(5, timeout_ns=20_000_000)
    A.forward(x, ci)
    assert A.status() == 4                         # SDP_ERR_TIMEOUT
    assert float((torch.ones(4, device="cuda") * 2).sum()) == 8.0   # the context still works
    A.set_wait_test(-1, timeout_ns=0)
    y = A.forward(x, ci).cpu().numpy()
    assert A.status() == 0
    assert_close(y, O.gridding_forward(geo, c["x"], c["S"], c["V"], c["omega"], c["frame"], c["coils"]), FP32_BOUND,
                 "tiled interpolation after the bounded wait ran out")


def test_interp_threads_choice_by_width():
    """1024-thread interpolation CTAs exist for W <= 4 only; wider kernels default to 256."""
    from paper_2408_02367_gb300 import op
    c = make_case((12, 12, 12), 6, 2.0, 2, 2, 4, 1, 200, [1, 0])
    args = (c["omega"], c["frame"], c["n"], 6, 2.0, c["V"], c["S"], 2)
    with pytest.raises(op.SdpError):
        op.make_operator(*args, tuning={"interp_threads": 1024})
    assert op.make_operator(*args).tuning["interp_threads"] == 256
    A = op.make_operator(*args, tuning={"interp_threads": 256})
    y = A.forward(t(c["x"]), t(c["coils"])).cpu().numpy()
    geo = O.Geometry(c["n"], 6, 2.0)
    assert_close(y, O.gridding_forward(geo, c["x"], c["S"], c["V"], c["omega"], c["frame"], c["coils"]), FP32_BOUND,
                 "W=6 with 256-thread interpolation")


def test_autotuner_candidates_agree_and_cache(tmp_path):
    from paper_2408_02367_gb300 import tune
    c = make_case((24, 20, 16), 4, 1.25, 3, 3, 10, 1, 600, [0, 1])
    cands = tune.candidates()[:2] + tune.candidates()[3:5] + tune.candidates()[-1:]
    cache = str(tmp_path / "tune.json")
    best, table = tune.autotune(c["omega"], c["frame"], c["n"], 4, 1.25, c["V"], c["S"], max_batch=2, cands=cands,
                                reps=3, cache=cache)
    assert len(table) == len(cands)
    assert [r["ms"] for r in table] == sorted(r["ms"] for r in table)
    assert all(r["rel_vs_first"] <= 1e-5 for r in table)
    assert best["spread_bins"] == tuple(table[0]["tuning"]["spread_bins"])
    best2, table2 = tune.autotune(c["omega"], c["frame"], c["n"], 4, 1.25, c["V"], c["S"], max_batch=2,
                                  cands=cands, reps=3, cache=cache)
    assert best2 == best and table2 == table                     # served from the cache


def test_adjoint_identity_on_gpu():
    c = make_case((24, 20, 28), 4, 1.25, 5, 4, 30, 1, 400, [3, 1, 2])
    A = gpu_op(c)
    x = t(synth.random_complex(c["x"].shape, 7))
    y = t(synth.random_complex((3, A.J), 8))
    ci = t(c["coils"])
    Ax = A.forward(x, ci)
    AHy = A.adjoint(y, ci)
    lhs = torch.vdot(y.flatten().to(torch.complex128), Ax.flatten().to(torch.complex128))
    rhs = torch.vdot(AHy.flatten().to(torch.complex128), x.flatten().to(torch.complex128))
    assert abs(complex(lhs - rhs)) / abs(complex(lhs)) < 1e-5


def test_integer_grid_frequencies_hit_window_ties():
    """omega on the image's integer grid: every sample sits on a window tie, and the
    float32 window decision must agree with the oracle's."""
    n = (12, 10, 8)
    m = np.stack(np.meshgrid(*[np.arange(-(d // 2), d - d // 2) for d in n], indexing="ij"), -1).reshape(-1, 3)
    omega = (2.0 * np.pi * m / np.array(n)).astype(np.float32)
    for W, sigma in [(4, 1.25), (6, 2.0), (4, 2.0)]:
        c = make_case(n, W, sigma, 1, 2, 1, 1, 4, [1, 0])
        c["omega"] = omega
        c["frame"] = np.zeros(len(omega), np.int32)
        geo = O.Geometry(n, W, sigma)
        A = gpu_op(c)
        y_ref = O.gridding_forward(geo, c["x"], c["S"], c["V"], omega, c["frame"], c["coils"])
        y = A.forward(t(c["x"]), t(c["coils"])).cpu().numpy()
        assert_close(y, y_ref, FP32_BOUND, f"integer-grid ties W={W} sigma={sigma}")


def test_channel_split_and_plain_form_equal_batched():
    """Plain form: one coil and one channel per call, accumulated; equals the batched call."""
    c = make_case((20, 20, 20), 4, 1.25, 5, 4, 40, 1, 256, [3, 0, 2])
    A = gpu_op(c)
    x = t(c["x"])
    ci = t(c["coils"])
    y = A.forward(x, ci)
    plain = torch.zeros_like(y)
    for b in range(3):
        for k in range(5):
            A.forward(x, ci[b:b + 1], out=plain[b:b + 1], k0=k, nk=1, accumulate=True)
    assert (torch.linalg.norm(plain - y) / torch.linalg.norm(y)).item() < 1e-5
    r = t(synth.random_complex((3, A.J), 3))
    a = A.adjoint(r, ci)
    ap = torch.zeros_like(a)
    for b in range(3):
        for k in range(5):
            A.adjoint(r[b:b + 1].contiguous(), ci[b:b + 1], out=ap, accumulate=True, k0=k, nk=1)
    assert (torch.linalg.norm(ap - a) / torch.linalg.norm(a)).item() < 1e-5
    # accumulate flag of the full adjoint
    a2 = A.adjoint(r, ci, out=a.clone(), accumulate=True)
    assert (torch.linalg.norm(a2 - 2 * a) / torch.linalg.norm(2 * a)).item() < 1e-6


def test_channel_subsets_sum_to_the_full_call():
    """Calls on channel ranges [k0, k0 + nk) with nk > 1 (grids interleaved over nk
    channels, not K) add up to the call on all K channels."""
    c = make_case((18, 16, 20), 4, 1.25, 7, 3, 12, 1, 256, [2, 0])
    A = gpu_op(c)
    x = t(c["x"])
    ci = t(c["coils"])
    y = A.forward(x, ci)
    r = t(synth.random_complex((2, A.J), 4))
    a = A.adjoint(r, ci)
    for split in ((0, 3, 7), (0, 2, 5, 7), (0, 6, 7)):
        ys = torch.zeros_like(y)
        as_ = torch.zeros_like(a)
        for k0, k1 in zip(split[:-1], split[1:]):
            A.forward(x, ci, out=ys, k0=k0, nk=k1 - k0, accumulate=True)
            A.adjoint(r, ci, out=as_, k0=k0, nk=k1 - k0, accumulate=True)
        assert (torch.linalg.norm(ys - y) / torch.linalg.norm(y)).item() < 1e-5, split
        assert (torch.linalg.norm(as_ - a) / torch.linalg.norm(a)).item() < 1e-5, split
    assert A.status() == 0


def test_bad_coil_index_sets_status_without_fault():
    c = make_case((10, 10, 10), 4, 1.25, 2, 2, 2, 1, 100, [0, 1])
    A = gpu_op(c)
    y = A.forward(t(c["x"]), torch.tensor([0, 7], dtype=torch.int32, device="cuda"))
    assert A.status() == 5
    assert A.status() == 0
    assert torch.all(y[1] == 0)


def test_empty_frames_and_single_sample():
    n = (8, 8, 8)
    x = synth.ellipsoid_phantom(n, 2)
    S = synth.coil_maps(n, 1)
    V = synth.subspace_basis(4, 2)
    omega = np.array([[0.3, -2.0, 3.14159]], np.float32)
    frame = np.array([2], np.int32)          # frames 0, 1 and 3 are empty
    from paper_2408_02367_gb300 import op
    A = op.make_operator(omega, frame, n, 4, 2.0, V, S, 1)
    geo = O.Geometry(n, 4, 2.0)
    y_ref = O.gridding_forward(geo, x, S, V, omega, frame, [0])
    y = A.forward(t(x), t(np.array([0], np.int32))).cpu().numpy()
    assert_close(y, y_ref, FP32_BOUND, "single sample")


def test_autograd_gradient_matches_oracle_adjoint():
    from paper_2408_02367_gb300 import op
    c = make_case((24, 24, 24), 6, 2.0, 5, 4, 100, 1, 512, [1, 3])
    geo = O.Geometry(c["n"], 6, 2.0)
    A = gpu_op(c)
    y_meas = O.gridding_forward(geo, synth.ellipsoid_phantom(c["n"], 5, seed=9), c["S"], c["V"], c["omega"],
                                c["frame"], c["coils"])
    xg = t(c["x"]).requires_grad_(True)
    ci = t(c["coils"])
    yhat = op.apply_A(A, xg, ci)
    loss = torch.sum(torch.abs(yhat - t(y_meas.astype(np.complex64))) ** 2)
    loss.backward()
    fwd = lambda v: O.gridding_forward(geo, v, c["S"], c["V"], c["omega"], c["frame"], c["coils"])
    adj = lambda r: O.gridding_adjoint(geo, r, c["S"], c["V"], c["omega"], c["frame"], c["coils"])
    g_ref = O.dip_grad(fwd, adj, c["x"].astype(np.complex128), y_meas)
    assert_close(xg.grad.cpu().numpy(), g_ref, 1e-4, "autograd gradient vs oracle A^H(2r)")
    l_ref = O.dip_loss(fwd, c["x"].astype(np.complex128), y_meas)
    assert abs(loss.item() - l_ref) / l_ref < 1e-4


@pytest.mark.parametrize("n,K,coils", [((8, 16, 128), 5, [1, 0]), ((24, 20, 64), 5, [0, 1, 1]),
                                       ((6, 10, 160), 3, [1]), ((10, 12, 63), 5, [1, 0]),
                                       ((12, 8, 200), 8, [0, 1])])
def test_staged_prologue_equals_direct_prologue(n, K, coils):
    """The fused axis-3 kernels with bulk-copy staged inputs (fft_staged = 3: the forward prologue
    and the adjoint epilogue) compute the same operator as the direct-load kernels (the same
    operations per grid line; the compiler may fuse a multiply-add differently, so agreement is to
    float32 rounding, not bits), on grid lengths 160, 80, 200, 250 and with an odd N3 (where the
    direct kernels run)."""
    from paper_2408_02367_gb300 import op
    c = make_case(n, 4, 1.25, K, 2, 12, 1, 300, coils)     # 12 frames: a rank-K subspace for K <= 8
    geo = O.Geometry(c["n"], 4, 1.25)
    base = {"spread_bins": (8, 4, 4), "spread_chunk": 512, "fft_engine": 0, "fft_lines": 8}
    A0 = op.make_operator(c["omega"], c["frame"], c["n"], 4, 1.25, c["V"], c["S"], max_batch=3, tuning=base)
    A1 = op.make_operator(c["omega"], c["frame"], c["n"], 4, 1.25, c["V"], c["S"], max_batch=3,
                          tuning=dict(base, fft_staged=3))
    assert A1.tuning["fft_staged"] == 3
    x, ci = t(c["x"]), t(c["coils"])
    y0, y1 = A0.forward(x, ci), A1.forward(x, ci)
    assert (torch.linalg.norm(y1 - y0) / torch.linalg.norm(y0)).item() < 1e-6
    assert_close(y1.cpu().numpy(), O.gridding_forward(geo, c["x"], c["S"], c["V"], c["omega"], c["frame"],
                                                      c["coils"]), FP32_BOUND, f"staged prologue {n}")
    # a channel subset (nk < K) and an out-of-range coil index (status, zeros)
    ys = torch.zeros_like(y1)
    A1.forward(x, ci, out=ys, k0=1, nk=K - 1, accumulate=True)
    ys0 = torch.zeros_like(y0)
    A0.forward(x, ci, out=ys0, k0=1, nk=K - 1, accumulate=True)
    assert (torch.linalg.norm(ys - ys0) / torch.linalg.norm(ys0)).item() < 1e-6
    assert A1.status() == 0
    bad = torch.tensor([0, 9], dtype=torch.int32, device="cuda")
    yb = A1.forward(x, bad)
    assert A1.status() == 5 and torch.all(yb[1] == 0)
    # the adjoint's staged axis-3 FFT + epilogue against the direct kernel and the oracle,
    # then accumulated into an existing output
    r = t(synth.random_complex(tuple(y0.shape), 17))
    a0, a1 = A0.adjoint(r, ci), A1.adjoint(r, ci)
    assert (torch.linalg.norm(a1 - a0) / torch.linalg.norm(a0)).item() < 1e-6
    assert_close(a1.cpu().numpy(), O.gridding_adjoint(geo, r.cpu().numpy(), c["S"], c["V"], c["omega"], c["frame"],
                                                      c["coils"]), FP32_BOUND, f"staged epilogue {n}")
    acc = a1.clone()
    A1.adjoint(r, ci, out=acc, accumulate=True)
    assert (torch.linalg.norm(acc - 2 * a1) / torch.linalg.norm(2 * a1)).item() < 1e-6
    assert A1.status() == 0
    # an out-of-range coil index in the adjoint: status 5, its term left out of the coil sum
    r2 = t(synth.random_complex((2, A1.J), 18))
    for A in (A0, A1):
        ab = A.adjoint(r2, bad)
        assert A.status() == 5
        assert torch.equal(ab, A.adjoint(r2[:1].contiguous(), bad[:1].contiguous()))
        assert A.status() == 0
