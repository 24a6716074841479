"""The FP64 oracle against facts fixed outside it (closed forms, numpy's FFT,
quadrature, invariants, the Kaiser-Bessel error floor).  CPU only."""
import numpy as np
import pytest

from oracle import nufft as O
from paper_2408_02367_gb300 import synth
from tests import oracle_pins as P


@pytest.mark.parametrize("W,sigma", [(6, 2.0), (4, 1.25), (8, 2.0)])
def test_kb_ft_closed_form_matches_quadrature(W, sigma):
    assert P.kb_ft_vs_quadrature(O, W, sigma) < 1e-10


def test_grid_size_is_minimal_even_smooth():
    cases = {(32, 2.0, 6): 64, (128, 1.25, 4): 160, (200, 1.25, 4): 250, (160, 1.25, 4): 200,
             (96, 1.25, 4): 120, (64, 1.25, 4): 80, (24, 2.0, 6): 48, (14, 2.0, 6): 30, (3, 2.0, 6): 12}
    for (n, s, W), m in cases.items():
        got = O.grid_size(n, s, W)
        # brute force: smallest integer meeting every condition
        brute = next(v for v in range(1, 10000)
                     if v >= np.ceil(s * n) and v >= 2 * W and v % 2 == 0 and O.is_smooth235(v))
        assert got == brute == m, (n, s, W, got, brute, m)


def test_nudft_matches_fftn_on_integer_grid():
    assert P.nudft_on_grid_vs_fftn(O) < 1e-12


def test_nudft_full_cartesian_gram_is_nvox_identity():
    assert P.full_cartesian_gram(O) < 1e-12


# Kaiser-Bessel gridding error floor against the exact sum.  The bound of 1e-6
# applies at W=8, sigma=2 (W=6, sigma=2 sits near 5e-6 for this kernel); the
# float32 grid coordinates of the spec contribute a few 1e-7.
@pytest.mark.parametrize("W,sigma,bound", [(8, 2.0, 1e-6), (7, 2.0, 3e-6), (6, 2.0, 2e-5), (4, 1.25, 2e-2)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_gridding_within_kb_error_floor_of_nudft(W, sigma, bound, adjoint):
    err = P.gridding_vs_nudft(O, W, sigma, adjoint=adjoint)
    print(f"gridding vs NUDFT W={W} sigma={sigma} adjoint={adjoint}: {err:.3e}")
    assert err < bound


def test_gridding_on_integer_grid_frequencies():
    """Frequencies exactly on the image's integer grid hit exact window ties."""
    n = (8, 10, 6)
    geo = O.Geometry(n, 6, 2.0)
    m = np.stack(np.meshgrid(*[np.arange(-(d // 2), d - d // 2) for d in n], indexing="ij"), -1).reshape(-1, 3)
    omega = (2.0 * np.pi * m / np.array(n)).astype(np.float32)
    x = synth.ellipsoid_phantom(n, 1, seed=3)
    S = np.ones((1,) + n, np.complex64)
    V = np.ones((1, 1), np.complex64)
    fr = np.zeros(len(m), np.int32)
    y = O.gridding_forward(geo, x, S, V, omega, fr, [0])[0]
    X = np.fft.fftn(np.fft.ifftshift(x[0].astype(np.complex128)))
    ref = X[tuple((m % np.array(n)).T)]
    assert P.rel(y, ref) < 2e-5


def test_subspace_basis_indexing_with_permutation_V():
    assert P.subspace_permutation(O) < 2e-5


def test_gridding_adjoint_identity():
    assert P.adjoint_identity(O) < 1e-12
    assert P.adjoint_identity(O, W=6, sigma=2.0, n=(8, 9, 10)) < 1e-12


def test_nudft_adjoint_identity_and_linearity():
    n = (6, 7, 5)
    x, S, V, omega, frame = P._toy_inputs(n, 2, 3, 3, 150, 51)
    coils = [0, 2, 2]                     # duplicates allowed: they sum
    y = synth.random_complex((3, 150), 52)
    Ax = O.nudft_forward(x, S, V, omega, frame, coils)
    AHy = O.nudft_adjoint(y, S, V, omega, frame, coils, n)
    lhs, rhs = np.vdot(y, Ax), np.vdot(AHy, x.astype(np.complex128))
    assert abs(lhs - rhs) / abs(lhs) < 1e-12
    x2 = synth.random_complex(x.shape, 53).astype(np.complex128)
    a, b = 0.3 - 1.2j, -0.7 + 0.1j
    lin = O.nudft_forward(a * x.astype(np.complex128) + b * x2, S, V, omega, frame, coils)
    assert P.rel(lin, a * Ax + b * O.nudft_forward(x2, S, V, omega, frame, coils)) < 1e-12


def test_coil_algebra_batch_equals_sum_of_single_coils():
    n = (10, 8, 12)
    geo = O.Geometry(n, 4, 1.25)
    x, S, V, omega, frame = P._toy_inputs(n, 3, 4, 5, 300, 61)
    coils = [3, 1, 2]
    y = synth.random_complex((3, 300), 62)
    batch = O.gridding_adjoint(geo, y, S, V, omega, frame, coils)
    singles = sum(O.gridding_adjoint(geo, y[b:b + 1], S, V, omega, frame, [c]) for b, c in enumerate(coils))
    assert P.rel(batch, singles) < 1e-13
    yb = O.gridding_forward(geo, x, S, V, omega, frame, coils)
    for b, c in enumerate(coils):
        assert P.rel(yb[b], O.gridding_forward(geo, x, S, V, omega, frame, [c])[0]) < 1e-14


def test_phase_and_scale_covariance():
    n = (8, 8, 8)
    geo = O.Geometry(n, 6, 2.0)
    x, S, V, omega, frame = P._toy_inputs(n, 2, 2, 2, 100, 71)
    y = O.gridding_forward(geo, x, S, V, omega, frame, [1])
    z = np.exp(0.7j) * 2.5
    y2 = O.gridding_forward(geo, z * x.astype(np.complex128), S, V, omega, frame, [1])
    assert P.rel(y2, z * y) < 1e-13


def test_loss_gradient_matches_central_differences():
    """Eq. 3 loss with DCF = 1 at a 24^3 volume: Re<grad, d> vs central differences."""
    w = synth.WORKLOADS["vol24_w6"]
    x, S, V, omega, frame = synth.make_problem(w)
    geo = O.Geometry(w.n, w.width, w.oversamp)
    coils = [1, 3]
    x = x.astype(np.complex128)
    fwd = lambda v: O.gridding_forward(geo, v, S, V, omega, frame, coils)
    adj = lambda r: O.gridding_adjoint(geo, r, S, V, omega, frame, coils)
    y_meas = fwd(synth.ellipsoid_phantom(w.n, w.K, seed=9).astype(np.complex128))
    g = O.dip_grad(fwd, adj, x, y_meas)
    rng = np.random.default_rng(5)
    for _ in range(3):
        d = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
        h = 1e-3
        fd = (O.dip_loss(fwd, x + h * d, y_meas) - O.dip_loss(fwd, x - h * d, y_meas)) / (2 * h)
        an = float(np.real(np.vdot(g, d)))
        assert abs(fd - an) / abs(an) < 1e-7, (fd, an)


def test_grid_coordinates_wrap_and_ties():
    M = (64, 20, 250)
    om = np.array([[-np.pi, 0.0, np.pi], [-1e-30, 1e-30, -3.0e-8], [2 * np.pi * 3 / 64, -2 * np.pi / 20, 0.5]],
                  dtype=np.float32)
    g = O.grid_coords(om, M)
    assert np.all(g >= 0) and np.all(g < np.array(M, np.float32))
    assert g[0, 0] == 32.0 and g[0, 1] == 0.0 and g[0, 2] == 125.0
    assert g[1, 0] == 0.0                           # tiny negative rounds onto M, which wraps to 0
    m0 = O.window_start(np.array([[32.0, 3.0, 0.0]], np.float32), 4)
    assert list(m0[0]) == [30, 1, -2]
