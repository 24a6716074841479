"""Seeded synthetic inputs for the subspace multicoil NUFFT operator.

The paper's in-vivo dataset (a whole-brain 3D spiral MRF scan, 8 coils, Sec. 3.1)
is not available, so every input here is synthetic with the shapes and structure
of that acquisition: a smooth complex time-compressed image series (TSMI,
Sec. 2 after Eq. 1), smooth coil sensitivities, golden-angle-rotated 3D spiral
arms (one or more per frame), and an orthonormal temporal subspace basis V.

This module holds no NUFFT arithmetic: it only draws inputs.  Both the FP64
oracle tests and the CUDA path consume these arrays unchanged.

Layouts (C order, complex64 unless stated):
  x      [K][N1][N2][N3]      TSMI, K subspace channels
  S      [C][N1][N2][N3]      coil sensitivities
  omega  [J][3] float32       k-space locations in radians, |omega_d| <= pi,
                              omega[:, d] pairs with image axis d
  frame  [J] int32            frame index t of each sample (frames are contiguous)
  V      [T][K]               temporal subspace basis
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Seeds of the independent input streams.
SEED_PHANTOM = 0
SEED_V = 2
SEED_NOISE = 3
SEED_COILS_DRAW = 4


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape of one synthetic reconstruction problem."""

    name: str
    n: tuple            # image matrix (N1, N2, N3)
    K: int              # subspace rank
    C: int              # coils
    T: int              # frames
    arms: int           # spiral arms per frame
    arm_len: int        # samples per arm
    width: int          # Kaiser-Bessel kernel width W
    oversamp: float     # grid oversampling sigma
    batch: int          # coil minibatch per operator call

    @property
    def samples_per_frame(self) -> int:
        return self.arms * self.arm_len

    @property
    def J(self) -> int:
        return self.T * self.samples_per_frame

    @property
    def nvox(self) -> int:
        return int(np.prod(self.n))


# Workloads named by what they are.  The 128^3 one is the single-GPU throughput
# workload; the 32^3 one is small enough for the FP64 oracle to finish in seconds.
WORKLOADS = {
    "vol32_w6": Workload("vol32_w6", (32, 32, 32), 5, 4, 100, 1, 512, 6, 2.0, 4),
    "vol128_w4": Workload("vol128_w4", (128, 128, 128), 5, 8, 480, 1, 1024, 4, 1.25, 2),
    "vol200_w4": Workload("vol200_w4", (200, 200, 160), 5, 32, 1000, 2, 1024, 4, 1.25, 8),
    "vol24_w6": Workload("vol24_w6", (24, 24, 24), 5, 4, 100, 1, 512, 6, 2.0, 2),
}

# Whole-brain coil minibatches: one 200x200x160, C=32 volume applied to a work list
# of uneven minibatches (each item with its own TSMI).
WHOLE_BRAIN_BATCHES = (1, 2, 4, 8)

# Six independent reconstructions of different matrix sizes in one batch: 1024-sample
# arms, one arm per frame, coil minibatch C/4 per volume, W=4, sigma=1.25, K=5.
MULTI_VOLUME = (
    Workload("mv64", (64, 64, 64), 5, 8, 300, 1, 1024, 4, 1.25, 2),
    Workload("mv96", (96, 96, 96), 5, 8, 400, 1, 1024, 4, 1.25, 2),
    Workload("mv128", (128, 128, 128), 5, 16, 500, 1, 1024, 4, 1.25, 4),
    Workload("mv128x96", (128, 128, 96), 5, 16, 600, 1, 1024, 4, 1.25, 4),
    Workload("mv160", (160, 160, 160), 5, 32, 800, 1, 1024, 4, 1.25, 8),
    Workload("mv200x160", (200, 200, 160), 5, 32, 1000, 1, 1024, 4, 1.25, 8),
)


def golden_means_3d():
    """Multidimensional golden means for 3D direction sampling.

    They are 1/lam and 1/lam^2 for the real root lam of lam^3 = lam^2 + 1
    (Chan et al. 2009, the 3D generalisation of the golden ratio).
    """
    lam = 1.0
    for _ in range(60):  # Newton on f(l) = l^3 - l^2 - 1
        f = lam ** 3 - lam ** 2 - 1.0
        lam -= f / (3 * lam ** 2 - 2 * lam)
    return 1.0 / lam ** 2, 1.0 / lam  # (~0.4656, ~0.6823)


def spiral_trajectory(T: int, arms: int, arm_len: int, dtype=np.float32):
    """Golden-angle-rotated planar Archimedean spiral arms in 3D k-space.

    Arm i = t*arms + a.  Radius r(s) = pi * s / (arm_len - 1) and angle
    theta(s) = 2*pi*(arm_len/64)*s/(arm_len - 1) (arm_len/64 turns per arm).  The
    plane normal of arm i follows the 3D golden means and the arm is turned
    in-plane by the golden angle pi*(3 - sqrt 5)*i.  |k| <= pi everywhere.

    Returns (omega [T*arms*arm_len][3] float32, frame [J] int32).
    """
    phi1, phi2 = golden_means_3d()
    n_arms = T * arms
    i = np.arange(n_arms, dtype=np.float64)
    cz = 2.0 * np.mod(i * phi1, 1.0) - 1.0
    az = 2.0 * np.pi * np.mod(i * phi2, 1.0)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    nrm = np.stack([sz * np.cos(az), sz * np.sin(az), cz], axis=1)
    # orthonormal in-plane basis (e1, e2) perpendicular to the normal
    ref = np.where(np.abs(nrm[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(nrm, ref)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(nrm, e1)
    s = np.arange(arm_len, dtype=np.float64) / max(arm_len - 1, 1)
    r = np.pi * s
    theta = 2.0 * np.pi * (arm_len / 64.0) * s
    psi = np.pi * (3.0 - math.sqrt(5.0)) * i
    ang = theta[None, :] + psi[:, None]                     # [n_arms][arm_len]
    k = (r[None, :, None] * (np.cos(ang)[:, :, None] * e1[:, None, :]
                             + np.sin(ang)[:, :, None] * e2[:, None, :]))
    omega = k.reshape(-1, 3)
    omega = np.clip(omega, -np.pi, np.pi).astype(dtype)
    frame = np.repeat(np.arange(T, dtype=np.int32), arms * arm_len)
    return omega, frame


def _fftn(a, inverse=False):
    """3D FFT over the last three axes on every host core (scipy.fft), else numpy."""
    try:
        import scipy.fft as sf
        return (sf.ifftn if inverse else sf.fftn)(a, axes=(-3, -2, -1), workers=-1)
    except ImportError:
        return (np.fft.ifftn if inverse else np.fft.fftn)(a, axes=(-3, -2, -1))


def _smooth_fft(vol: np.ndarray, sigma_vox: float) -> np.ndarray:
    """Gaussian smoothing (periodic) of the last three axes by FFT multiplication."""
    shp = vol.shape[-3:]
    f = _fftn(vol)
    g = np.ones(shp)
    for d, nd in enumerate(shp):
        fr = np.fft.fftfreq(nd)
        gd = np.exp(-2.0 * (np.pi * sigma_vox * fr) ** 2)
        sh = [1, 1, 1]
        sh[d] = nd
        g = g * gd.reshape(sh)
    return _fftn(f * g, inverse=True)


def _centred_coords(n):
    """Normalised coordinates in [-1, 1) along each axis (FOV/2 units)."""
    return [(np.arange(nd) - nd // 2) / (nd / 2.0) for nd in n]


def ellipsoid_phantom(n, K: int, seed: int = SEED_PHANTOM, n_ell: int = 12, dtype=np.complex64):
    """Sum of random ellipsoids with complex per-channel amplitudes, smoothed.

    Centres ~ U(-0.6, 0.6), semi-axes ~ U(0.1, 0.45) (FOV/2 units), random
    rotation, amplitude of ellipsoid e in channel k ~ CN(0,1)/(k+1); the sum is
    smoothed with a Gaussian of one voxel.  Returns x [K][N1][N2][N3].
    """
    rng = np.random.default_rng(seed)
    coords = _centred_coords(n)
    x = np.zeros((K,) + tuple(n), dtype=np.complex128)
    for _ in range(n_ell):
        ctr = rng.uniform(-0.6, 0.6, size=3)
        ax = rng.uniform(0.1, 0.45, size=3)
        q, _r = np.linalg.qr(rng.standard_normal((3, 3)))
        amp = (rng.standard_normal(K) + 1j * rng.standard_normal(K)) / np.sqrt(2.0)
        amp = amp / (np.arange(K) + 1.0)
        # only the voxels within the ellipsoid's bounding sphere (radius max(ax)) can lie inside it
        sl = []
        for d, u in enumerate(coords):
            idx = np.nonzero(np.abs(u - ctr[d]) <= ax.max() + 1e-12)[0]
            sl.append(slice(idx[0], idx[-1] + 1) if idx.size else slice(0, 0))
        if any(v.stop <= v.start for v in sl):
            continue
        X, Y, Z = np.meshgrid(coords[0][sl[0]], coords[1][sl[1]], coords[2][sl[2]], indexing="ij")
        loc = (np.stack([X, Y, Z], axis=-1) - ctr) @ q
        inside = np.sum((loc / ax) ** 2, axis=-1) <= 1.0
        sub = x[:, sl[0], sl[1], sl[2]]
        sub[:, inside] += amp[:, None]
    x = _smooth_fft(x, 1.0)
    return x.astype(dtype)


def coil_maps(n, C: int, dtype=np.complex64):
    """Smooth Gaussian-bump coil sensitivities normalised to unit root-sum-of-squares.

    Coil c sits at a Fibonacci-sphere direction at radius 1.2 (FOV/2 units); its
    magnitude is a Gaussian with standard deviation 0.6 FOV and its phase is 2*pi*c/C plus a small
    linear ramp.  Returns S [C][N1][N2][N3].
    """
    # Both the Gaussian magnitude and the linear phase ramp factor over the axes, so
    # coil c is the outer product of three 1-D complex profiles (times its constant
    # phase); only the root-sum-of-squares normalisation couples the coils.
    coords = _centred_coords(n)
    ga = np.pi * (3.0 - math.sqrt(5.0))
    prof = []
    for c in range(C):
        zc = 1.0 - 2.0 * (c + 0.5) / C
        rc = math.sqrt(max(0.0, 1.0 - zc * zc))
        d = np.array([rc * math.cos(ga * c), rc * math.sin(ga * c), zc]) * 1.2
        # magnitude exp(-|r - d|^2 / (2 * 1.2^2)) (std 0.6 FOV = 1.2 in FOV/2 units), phase ramp 0.3 d.r
        a = [np.exp(-(u - d[i]) ** 2 / (2.0 * 1.2 ** 2)) * np.exp(1j * 0.3 * d[i] * u)
             for i, u in enumerate(coords)]
        a[0] = a[0] * np.exp(1j * 2.0 * np.pi * c / C)
        prof.append(a)
    ss = np.zeros(tuple(n))
    for a in prof:
        m = [np.abs(v) ** 2 for v in a]
        ss += m[0][:, None, None] * m[1][None, :, None] * m[2][None, None, :]
    inv_rss = 1.0 / np.sqrt(ss)
    S = np.empty((C,) + tuple(n), dtype=dtype)
    for c, a in enumerate(prof):
        S[c] = (a[0][:, None, None] * a[1][None, :, None] * a[2][None, None, :]) * inv_rss
    return S


def subspace_basis(T: int, K: int, seed: int = SEED_V, real: bool = False, dtype=np.complex64):
    """Orthonormal T x K basis: Q of the reduced QR of a seeded Gaussian matrix."""
    rng = np.random.default_rng(seed)
    if real:
        g = rng.standard_normal((T, K))
    else:
        g = rng.standard_normal((T, K)) + 1j * rng.standard_normal((T, K))
    q, _ = np.linalg.qr(g)
    return q.astype(dtype)


def coil_minibatches(C: int, B: int, steps: int, seed: int = SEED_COILS_DRAW):
    """Coil minibatches of size B drawn uniformly without replacement per call."""
    rng = np.random.default_rng(seed)
    return [np.sort(rng.choice(C, size=B, replace=False)).astype(np.int32) for _ in range(steps)]


def complex_noise(shape, sigma: float, seed: int = SEED_NOISE, dtype=np.complex64):
    """Circular complex Gaussian noise with per-component std sigma/sqrt(2)."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * (sigma / math.sqrt(2.0))
    return z.astype(dtype)


def random_complex(shape, seed: int, dtype=np.complex64):
    """Unstructured complex Gaussian array (for adjoint-identity and linearity cases)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)


def make_problem(w: Workload, seed: int = SEED_PHANTOM):
    """All per-trajectory inputs of a workload: (x, S, V, omega, frame)."""
    x = ellipsoid_phantom(w.n, w.K, seed=seed)
    S = coil_maps(w.n, w.C)
    V = subspace_basis(w.T, w.K)
    omega, frame = spiral_trajectory(w.T, w.arms, w.arm_len)
    return x, S, V, omega, frame


# ----------------------------------------------------------------------------
# Synthetic MRF dictionaries for dictionary matching (no Bloch simulation)
# ----------------------------------------------------------------------------

SEED_DM = 6


def mrf_dictionary(T: int, n_t1: int = 64, n_t2: int = 48, dtype=np.complex64):
    """A smooth parametric stand-in for a Bloch-simulated MRF dictionary.

    Fingerprints f_t(T1, T2) = sin(a_t) (1 - 2 exp(-tau_t / T1)) exp(-kappa_t / T2) exp(i phi_t)
    for t = 0..T-1: an inversion-recovery-like T1 weighting, a T2 weighting
    that varies along the train, a smooth flip-angle train a_t and a slow
    phase phi_t.  It is not a Bloch response; it has what matching needs:
    atoms that vary smoothly with (T1, T2), so that neighbours are highly
    correlated, and norms that differ from atom to atom.  T1 on a log grid
    100..4000 ms, T2 on a log grid 10..2000 ms, pairs with T2 < T1 only.

    Returns (fingerprints [P][T], params [P][2] float32 (T1, T2) in ms).
    """
    t = np.arange(T, dtype=np.float64)
    tr = 10.0
    a = np.deg2rad(5.0 + 55.0 * np.sin(np.pi * t / 200.0) ** 2)
    tau = (t + 1.0) * tr
    kappa = 2.0 + 60.0 * np.sin(3.0 * np.pi * t / T) ** 2
    phi = 0.3 * np.sin(2.0 * np.pi * t / T)
    t1 = np.geomspace(100.0, 4000.0, n_t1)
    t2 = np.geomspace(10.0, 2000.0, n_t2)
    pairs = np.array([(a1, a2) for a1 in t1 for a2 in t2 if a2 < a1])
    f = (np.sin(a)[None, :] * (1.0 - 2.0 * np.exp(-tau[None, :] / pairs[:, :1]))
         * np.exp(-kappa[None, :] / pairs[:, 1:]) * np.exp(1j * phi)[None, :])
    return f.astype(dtype), pairs.astype(np.float32)


def compress_dictionary(fingerprints, K: int):
    """Temporal SVD compression (Sec. 2 after Eq. 1): V = the first K right singular
    vectors of the dictionary, atoms d_p = V^H f_p.  Returns (D [P][K], V [T][K])."""
    f = np.asarray(fingerprints, np.complex128)
    _, _, wh = np.linalg.svd(f, full_matrices=False)
    V = wh[:K].conj().T
    D = f @ V.conj()
    return D.astype(np.complex64), V.astype(np.complex64)


def dm_volume(D, nvox: int, noise: float = 0.0, seed: int = SEED_DM, dtype=np.complex64):
    """A TSMI [K][nvox] whose voxels are PD_v d_{p_v} plus complex noise (std
    `noise` times the mean voxel norm), with p_v uniform over the atoms and
    PD_v complex with magnitude in [0.5, 2].  Returns (x, p, PD)."""
    D = np.asarray(D, np.complex128)
    rng = np.random.default_rng(seed)
    p = rng.integers(0, D.shape[0], size=nvox)
    pd = rng.uniform(0.5, 2.0, size=nvox) * np.exp(1j * rng.uniform(-np.pi, np.pi, size=nvox))
    x = (pd[:, None] * D[p]).T
    if noise > 0:
        s = noise * np.mean(np.linalg.norm(x, axis=0)) / math.sqrt(2.0 * D.shape[1])
        x = x + s * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape))
    return np.ascontiguousarray(x.astype(dtype)), p.astype(np.int64), pd
