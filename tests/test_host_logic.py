"""Host-side logic: the synthetic inputs and the benchmark's bookkeeping (CPU only)."""
import math

import numpy as np

from paper_2408_02367_gb300 import synth


def test_golden_means_solve_the_cubic():
    p1, p2 = synth.golden_means_3d()
    lam = 1.0 / p2
    assert abs(lam ** 3 - lam ** 2 - 1.0) < 1e-12
    assert abs(p1 - p2 ** 2) < 1e-12
    assert abs(p1 - 0.4656) < 1e-4 and abs(p2 - 0.6823) < 1e-4


def test_spiral_trajectory_shape_range_and_frames():
    om, fr = synth.spiral_trajectory(7, 2, 300)
    assert om.shape == (7 * 2 * 300, 3) and om.dtype == np.float32
    assert np.all(np.abs(om) <= np.float32(np.pi))
    r = np.linalg.norm(om.astype(np.float64), axis=1)
    assert r.max() <= np.pi + 1e-5
    assert np.all(np.diff(fr) >= 0) and fr[0] == 0 and fr[-1] == 6
    assert np.all(np.bincount(fr) == 600)
    # every arm starts at the centre and is planar (normal orthogonal to all its points)
    arms = om.reshape(14, 300, 3).astype(np.float64)
    assert np.allclose(arms[:, 0], 0.0)
    for a in arms[:3]:
        nrm = np.cross(a[10], a[60])
        nrm /= np.linalg.norm(nrm)
        assert np.max(np.abs(a @ nrm)) < 1e-5


def test_subspace_basis_is_orthonormal():
    for real in (False, True):
        V = synth.subspace_basis(50, 5, real=real).astype(np.complex128)
        assert np.allclose(V.conj().T @ V, np.eye(5), atol=1e-5)


def test_coil_maps_have_unit_root_sum_of_squares():
    S = synth.coil_maps((12, 10, 8), 6).astype(np.complex128)
    rss = np.sqrt(np.sum(np.abs(S) ** 2, axis=0))
    assert np.allclose(rss, 1.0, atol=1e-5)


def test_phantom_is_smooth_and_channel_scaled():
    x = synth.ellipsoid_phantom((24, 24, 24), 5, seed=0)
    assert x.shape == (5, 24, 24, 24) and x.dtype == np.complex64
    e = [float(np.linalg.norm(x[k])) for k in range(5)]
    assert e[0] > 0 and e[4] < e[0]


def test_coil_minibatches_without_replacement_and_seeded():
    a = synth.coil_minibatches(8, 3, 20, seed=4)
    b = synth.coil_minibatches(8, 3, 20, seed=4)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))
    for m in a:
        assert len(set(m.tolist())) == 3 and m.min() >= 0 and m.max() < 8


def test_workload_sizes():
    w = synth.WORKLOADS["vol128_w4"]
    assert w.J == 491520 and w.nvox == 128 ** 3
    w = synth.WORKLOADS["vol200_w4"]
    assert w.J == 2048000


def test_bench_byte_model_and_oracle_scaling():
    import bench
    w = synth.WORKLOADS["vol128_w4"]
    M = (160, 160, 160)
    m = bench.path_model_bytes(w, 2, M)
    # 8 K Nvox + B (8 Nvox + 16 K G + 8 J) + 12 J per direction, two directions
    assert m == 2 * (8 * 5 * 128 ** 3 + 2 * (8 * 128 ** 3 + 16 * 5 * 160 ** 3 + 8 * w.J) + 12 * w.J)
    sb = bench.stage_bytes(w, 2, M, 1000)
    assert set(sb) == {"fwd_prologue_fft3", "fwd_fft2", "fwd_fft1", "interp", "residual_loss", "spread",
                       "adj_ifft1", "adj_ifft2", "adj_ifft3_epilogue"}
    assert sb["fwd_fft1"] == 8 * 2 * 5 * (128 * 160 * 160 + 160 ** 3)


def test_bench_measured_traffic_follows_the_captured_kernel(monkeypatch):
    """The bench reports a stage's ncu DRAM traffic only for the captured workload, batch and
    kernel variant, and only while the kernel's source is the captured one."""
    import bench
    tuned = {"spread_bins": [4, 4, 4], "interp_tiled": 1, "fft_staged": 3, "fft_cols": 32}
    captured = {fname: h for fname, h, _ in bench.NCU_TRAFFIC.values()}
    monkeypatch.setattr(bench, "source_hash", lambda fname: captured[fname])
    stages = ["spread", "interp", "fwd_prologue_fft3", "adj_ifft3_epilogue", "fwd_fft2", "fwd_fft1", "adj_ifft1",
              "adj_ifft2"]
    for st in stages:
        assert bench.measured_traffic(st, "vol128_w4", 2, tuned) > 0
    assert bench.measured_traffic("residual_loss", "vol128_w4", 2, tuned) is None
    for st, change in (("spread", {"spread_bins": [8, 4, 4]}), ("interp", {"interp_tiled": 0}),
                       ("fwd_prologue_fft3", {"fft_staged": 2}), ("adj_ifft3_epilogue", {"fft_staged": 1}),
                       ("fwd_fft2", {"fft_cols": 0}), ("adj_ifft1", {"fft_cols": 8})):
        assert bench.measured_traffic(st, "vol128_w4", 2, dict(tuned, **change)) is None
    assert bench.measured_traffic("spread", "vol200_w4", 2, tuned) is None
    assert bench.measured_traffic("spread", "vol128_w4", 4, tuned) is None
    monkeypatch.setattr(bench, "source_hash", lambda fname: "0" * 16)
    assert all(bench.measured_traffic(st, "vol128_w4", 2, tuned) is None for st in stages)


def test_bench_oracle_pieces_sum_to_the_oracle_step():
    """The CPU baseline splits a step into (coil, channel) pieces of the oracle's own steps; their
    sum over channels is the oracle's gridding forward, and the pool runs whole steps."""
    import bench
    from oracle import nufft as O
    w = synth.Workload("tiny", (8, 10, 6), 3, 3, 4, 1, 64, 4, 2.0, 2)
    x, S, V, omega, frame = synth.make_problem(w)
    bench._oracle_init(w.n, w.width, w.oversamp, x, S, V, omega, frame)
    geo = O.Geometry(w.n, w.width, w.oversamp)
    for c in (0, 2):
        y = sum(bench._oracle_fwd(c, k) for k in range(w.K))
        ref = O.gridding_forward(geo, x, S, V, omega, frame, [c])[0]
        assert np.allclose(y, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        r = synth.random_complex(w.J, 5).astype(np.complex128)
        chk = sum(bench._oracle_adj(c, k, r) for k in range(w.K))
        ref_a = O.gridding_adjoint(geo, r[None], S, V, omega, frame, [c])
        assert abs(chk - ref_a.sum()) <= 1e-10 * np.abs(ref_a).sum()
    orc = bench.OracleSteps(w, 2, max_workers=2)
    try:
        ts = orc.time_steps([np.array([0, 2]), np.array([1, 0])])
    finally:
        orc.close()
    assert len(ts) == 2 and all(t > 0 for t in ts)
    line = bench.oracle_line(w, 2, ts, 2, "test")
    assert line["cores"] == 2 and math.isclose(line["value"], 2 * w.J / np.mean(ts))


def test_multi_volume_and_whole_brain_shapes():
    """The six-volume batch and the whole-brain minibatches: sizes, grids and coil minibatches C/4."""
    grids = {"mv64": (80, 80, 80), "mv96": (120, 120, 120), "mv128": (160, 160, 160),
             "mv128x96": (160, 160, 120), "mv160": (200, 200, 200), "mv200x160": (250, 250, 200)}
    from oracle import nufft as O
    for w in synth.MULTI_VOLUME:
        assert w.batch == w.C // 4 and w.arm_len == 1024 and w.arms == 1 and w.K == 5
        assert O.Geometry(w.n, w.width, w.oversamp).M == grids[w.name]
    assert [w.C for w in synth.MULTI_VOLUME] == [8, 8, 16, 16, 32, 32]
    assert synth.WHOLE_BRAIN_BATCHES == (1, 2, 4, 8)


def test_separable_coil_maps_equal_their_elementwise_definition():
    """coil_maps builds each map as an outer product of 1-D profiles; it must equal the map written
    per voxel (Gaussian bump at a Fibonacci-sphere direction, linear phase ramp, unit RSS)."""
    n, C = (9, 12, 7), 5
    S = synth.coil_maps(n, C)
    c1, c2, c3 = [(np.arange(d) - d // 2) / (d / 2.0) for d in n]
    X, Y, Z = np.meshgrid(c1, c2, c3, indexing="ij")
    ga = np.pi * (3.0 - math.sqrt(5.0))
    ref = np.empty((C,) + n, np.complex128)
    for c in range(C):
        zc = 1.0 - 2.0 * (c + 0.5) / C
        rc = math.sqrt(max(0.0, 1.0 - zc * zc))
        d = np.array([rc * math.cos(ga * c), rc * math.sin(ga * c), zc]) * 1.2
        mag = np.exp(-((X - d[0]) ** 2 + (Y - d[1]) ** 2 + (Z - d[2]) ** 2) / (2.0 * 1.44))
        ref[c] = mag * np.exp(1j * (2.0 * np.pi * c / C + 0.3 * (d[0] * X + d[1] * Y + d[2] * Z)))
    ref /= np.sqrt(np.sum(np.abs(ref) ** 2, axis=0))[None]
    assert np.max(np.abs(S - ref)) < 1e-6
    assert np.allclose(np.sum(np.abs(S.astype(np.complex128)) ** 2, axis=0), 1.0, atol=1e-6)
