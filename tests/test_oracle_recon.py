"""Pins of the oracle's reconstruction building blocks (density compensation,
weighted loss, SVD-MRF initialiser, CG on the normal equations).  CPU only."""
import numpy as np

from oracle import nufft as O
from oracle import recon as R
from paper_2408_02367_gb300 import synth
from tests import oracle_pins as P


def _half_integer_grid_omega(M):
    """Every grid cell sampled once at its centre, g = m + 1/2 exactly in float32 (no window ties)."""
    m = np.stack(np.meshgrid(*[np.arange(d) for d in M], indexing="ij"), -1).reshape(-1, 3) + 0.5
    g = np.where(m >= np.array(M) / 2.0, m - np.array(M), m)       # centred, |omega| < pi
    return (2.0 * np.pi * g / np.array(M)).astype(np.float32)


def test_pipe_menon_on_uniform_sampling_is_uniform():
    n = (6, 6, 6)
    geo = O.Geometry(n, 4, 2.0)                                     # grid 12^3, W = 4
    om = _half_integer_grid_omega(geo.M)
    w = R.dcf_pipe_menon(geo, om, iters=3)
    assert np.max(w) / np.min(w) - 1.0 < 1e-10
    # every sample sees the same 4^3 taps at offsets +-1/2, +-3/2:  Phi Phi^H 1 = s^6
    s = float(np.sum(O.kb_window(np.array([-1.5, -0.5, 0.5, 1.5]), geo.W, geo.beta)))
    assert abs(w[0] * s ** 6 - 1.0) < 1e-10


def test_pipe_menon_on_spirals_grows_with_radius():
    n = (16, 16, 16)
    geo = O.Geometry(n, 4, 2.0)
    om, _ = synth.spiral_trajectory(40, 1, 256)
    w = R.dcf_pipe_menon(geo, om, iters=8)
    r = np.linalg.norm(om.astype(np.float64), axis=1)
    inner = np.median(w[r < 0.5])
    outer = np.median(w[r > 2.5])
    assert outer > 10.0 * inner
    # the iteration drives Phi Phi^H w towards 1
    pw = np.real(R.gram_samples(geo, w, om))
    assert np.median(np.abs(pw - 1.0)) < 0.1


def test_weighted_loss_gradient_matches_central_differences():
    n = (10, 12, 8)
    geo = O.Geometry(n, 4, 1.25)
    x, S, V, om, fr = P._toy_inputs(n, 3, 2, 4, 300, 81)
    coils = [1, 0]
    dcf = np.random.default_rng(3).uniform(0.2, 2.0, size=om.shape[0])
    y = synth.random_complex((2, om.shape[0]), 82).astype(np.complex128)
    fwd = lambda v: O.gridding_forward(geo, v, S, V, om, fr, coils)
    adj = lambda r: O.gridding_adjoint(geo, r, S, V, om, fr, coils)
    x = x.astype(np.complex128)
    g = R.dc_grad_dcf(fwd, adj, x, y, dcf)
    d = synth.random_complex(x.shape, 83).astype(np.complex128)
    h = 1e-3
    fd = (R.dc_loss_dcf(fwd, x + h * d, y, dcf) - R.dc_loss_dcf(fwd, x - h * d, y, dcf)) / (2 * h)
    assert abs(fd - np.real(np.vdot(g, d))) / abs(fd) < 1e-8


def test_svd_mrf_scale_minimises_the_weighted_residual():
    n = (8, 8, 8)
    geo = O.Geometry(n, 4, 2.0)
    x, S, V, om, fr = P._toy_inputs(n, 2, 3, 3, 200, 91)
    dcf = np.random.default_rng(4).uniform(0.5, 1.5, size=om.shape[0])
    coils = np.arange(3)
    y = O.gridding_forward(geo, synth.ellipsoid_phantom(n, 2, seed=5), S, V, om, fr, coils)
    x0 = R.svd_mrf_init(geo, y, S, V, om, fr, dcf)
    fwd = lambda v: O.gridding_forward(geo, v, S, V, om, fr, coils)
    base = R.dc_loss_dcf(fwd, x0, y, dcf)
    for f in (0.97, 1.03):
        assert R.dc_loss_dcf(fwd, f * x0, y, dcf) > base


def test_cg_reaches_the_least_squares_solution_of_a_small_system():
    n = (4, 4, 4)
    geo = O.Geometry(n, 4, 2.0)
    x, S, V, om, fr = P._toy_inputs(n, 1, 2, 2, 400, 101)
    dcf = np.random.default_rng(6).uniform(0.5, 1.5, size=om.shape[0])
    coils = np.arange(2)
    y = synth.random_complex((2, om.shape[0]), 102).astype(np.complex128)
    xcg, hist = R.cg_normal(geo, y, S, V, om, fr, dcf, iters=64)
    # dense least squares: columns A e_i, rows weighted by sqrt(DCF)
    nv = int(np.prod(n))
    cols = []
    for i in range(nv):
        e = np.zeros((1,) + n, np.complex128)
        e.flat[i] = 1.0
        cols.append(O.gridding_forward(geo, e, S, V, om, fr, coils).ravel())
    A = np.stack(cols, axis=1) * np.sqrt(np.tile(dcf, 2))[:, None]
    xls = np.linalg.lstsq(A, y.ravel() * np.sqrt(np.tile(dcf, 2)), rcond=None)[0]
    assert P.rel(xcg.ravel(), xls) < 1e-6
    assert hist[-1] < 1e-6 * hist[0]


def test_tv_closed_forms_constant_and_ramp():
    K, n = 2, (5, 4, 6)
    eps = 1e-3
    c = np.full((K,) + n, 0.7 - 0.2j)
    assert abs(R.tv_value(c, eps) - K * np.prod(n) * eps) < 1e-12
    assert np.max(np.abs(R.tv_grad(c, eps))) == 0.0
    a = 0.3 + 0.4j                                   # |a| = 0.5, ramp along axis 1
    ramp = np.broadcast_to(a * np.arange(n[0])[None, :, None, None], (K,) + n)
    expect = K * n[1] * n[2] * ((n[0] - 1) * np.sqrt(0.25 + eps ** 2) + eps)
    assert abs(R.tv_value(ramp, eps) - expect) < 1e-10


def test_tv_gradient_matches_central_differences():
    x = synth.random_complex((2, 6, 5, 7), 111).astype(np.complex128)
    eps = 0.05
    g = R.tv_grad(x, eps)
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
        h = 1e-6
        fd = (R.tv_value(x + h * d, eps) - R.tv_value(x - h * d, eps)) / (2 * h)
        assert abs(fd - np.real(np.vdot(g, d))) / abs(fd) < 1e-6
