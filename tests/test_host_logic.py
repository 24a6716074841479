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
    assert math.isclose(bench.oracle_step_seconds(w, 2, 1.0, 0.5, w.J // 4), 2 * 5 * (1.0 + 2.0))
