"""Density compensation, the DCF-weighted loss and the initialisers on the GPU,
against the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nufft as O
from oracle import recon as R
from paper_2408_02367_gb300 import synth

pytestmark = pytest.mark.gpu
FP32_BOUND = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2408_02367_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.fixture(scope="module")
def case():
    from paper_2408_02367_gb300 import op
    n, W, sigma, K, C, T = (20, 18, 16), 4, 1.25, 3, 4, 24
    x = synth.ellipsoid_phantom(n, K)
    S = synth.coil_maps(n, C)
    V = synth.subspace_basis(T, K)
    om, fr = synth.spiral_trajectory(T, 1, 256)
    A = op.make_operator(om, fr, n, W, sigma, V, S, max_batch=2)
    geo = O.Geometry(n, W, sigma)
    y_all = O.gridding_forward(geo, synth.ellipsoid_phantom(n, K, seed=4), S, V, om, fr, np.arange(C))
    y_all = y_all + synth.complex_noise(y_all.shape, 0.01 * np.abs(y_all).mean())
    return dict(n=n, W=W, sigma=sigma, x=x, S=S, V=V, om=om, fr=fr, A=A, geo=geo, y_all=y_all)


def test_gram_samples_and_pipe_menon_dcf(case):
    from paper_2408_02367_gb300 import recon
    Ad = recon.dcf_operator(case["om"], case["n"], case["W"], case["sigma"])
    w = np.random.default_rng(1).uniform(0.5, 2.0, size=case["om"].shape[0])
    g = Ad.gram_samples(_t(w.astype(np.complex64)[None]))[0].cpu().numpy()
    assert rel(g, R.gram_samples(case["geo"], w, case["om"])) < FP32_BOUND
    dg = recon.dcf_pipe_menon(Ad, iters=6).cpu().numpy()
    dr = R.dcf_pipe_menon(case["geo"], case["om"], iters=6)
    e = rel(dg, dr)
    print(f"Pipe-Menon DCF rel {e:.2e}")
    assert e < 1e-4


def test_weighted_loss_and_gradient(case):
    from paper_2408_02367_gb300 import op
    A, geo = case["A"], case["geo"]
    coils = np.array([3, 1], np.int32)
    dcf = np.random.default_rng(2).uniform(0.2, 3.0, size=case["om"].shape[0]).astype(np.float32)
    xg = _t(case["x"]).requires_grad_(True)
    loss = op.dc_loss(A, xg, _t(coils), _t(case["y_all"].astype(np.complex64)), dcf=_t(dcf))
    loss.backward()
    fwd = lambda v: O.gridding_forward(geo, v, case["S"], case["V"], case["om"], case["fr"], coils)
    adj = lambda r: O.gridding_adjoint(geo, r, case["S"], case["V"], case["om"], case["fr"], coils)
    ym = case["y_all"][coils]
    l_ref = R.dc_loss_dcf(fwd, case["x"].astype(np.complex128), ym, dcf)
    g_ref = R.dc_grad_dcf(fwd, adj, case["x"].astype(np.complex128), ym, dcf)
    assert abs(loss.item() - l_ref) / l_ref < 1e-5
    assert rel(xg.grad.cpu().numpy(), g_ref) < FP32_BOUND


def test_svd_mrf_initialiser(case):
    from paper_2408_02367_gb300 import recon
    dcf = np.random.default_rng(3).uniform(0.5, 1.5, size=case["om"].shape[0]).astype(np.float32)
    xg = recon.svd_mrf_init(case["A"], _t(case["y_all"].astype(np.complex64)), _t(dcf)).cpu().numpy()
    xr = R.svd_mrf_init(case["geo"], case["y_all"], case["S"], case["V"], case["om"], case["fr"], dcf)
    assert rel(xg, xr) < 1e-4


def test_cg_on_the_normal_equations(case):
    from paper_2408_02367_gb300 import recon
    dcf = np.random.default_rng(5).uniform(0.5, 1.5, size=case["om"].shape[0]).astype(np.float32)
    for lam in (0.0, 0.5):
        xg, hg = recon.cg_normal(case["A"], _t(case["y_all"].astype(np.complex64)), _t(dcf), iters=5, lam=lam)
        xr, hr = R.cg_normal(case["geo"], case["y_all"], case["S"], case["V"], case["om"], case["fr"], dcf,
                             iters=5, lam=lam)
        e = rel(xg.cpu().numpy(), xr)
        print(f"CG lam={lam}: rel {e:.2e}, residuals {hg[-1] / hg[0]:.3e} vs {hr[-1] / hr[0]:.3e}")
        assert e < 1e-4
        assert abs(hg[-1] / hg[0] - hr[-1] / hr[0]) < 1e-3 * max(1e-3, hr[-1] / hr[0]) + 1e-6


def test_total_variation_value_gradient_and_autograd(case):
    from paper_2408_02367_gb300 import op
    A = case["A"]
    eps, lam = 1e-2, 0.3
    x = case["x"]
    v = A.tv_value(_t(x), lam, eps).item()
    v_ref = lam * R.tv_value(x, eps)
    assert abs(v - v_ref) / v_ref < 1e-5
    g = A.tv_grad(_t(x), lam, eps).cpu().numpy()
    assert rel(g, lam * R.tv_grad(x, eps)) < FP32_BOUND
    # loss = data consistency + lam TV, one backward through both (Algorithm 1 lines 4-7)
    coils = np.array([0, 2], np.int32)
    xg = _t(x).requires_grad_(True)
    loss = op.dc_loss(A, xg, _t(coils), _t(case["y_all"].astype(np.complex64))) + op.tv_loss(A, xg, lam, eps)
    loss.backward()
    fwd = lambda u: O.gridding_forward(case["geo"], u, case["S"], case["V"], case["om"], case["fr"], coils)
    adj = lambda r: O.gridding_adjoint(case["geo"], r, case["S"], case["V"], case["om"], case["fr"], coils)
    ym = case["y_all"][coils]
    g_ref = O.dip_grad(fwd, adj, x.astype(np.complex128), ym) + lam * R.tv_grad(x, eps)
    assert rel(xg.grad.cpu().numpy(), g_ref) < FP32_BOUND


def test_total_variation_ragged_tiles_and_accumulate():
    """A volume that spans several 32 x 8 tiles and 16-plane segments with ragged edges on every axis."""
    from paper_2408_02367_gb300 import op
    n, K = (35, 19, 41), 2
    x = synth.random_complex((K,) + n, 121)
    om, fr = synth.spiral_trajectory(4, 1, 64)
    A = op.make_operator(om, fr, n, 4, 1.25, synth.subspace_basis(4, K), synth.coil_maps(n, 1), max_batch=1)
    eps, lam = 0.05, 0.9
    v = A.tv_value(_t(x), lam, eps).item()
    v_ref = lam * R.tv_value(x, eps)
    assert abs(v - v_ref) / v_ref < 1e-5
    base = synth.random_complex((K,) + n, 122)
    out = _t(base)
    A.tv_grad(_t(x), lam, eps, out=out, accumulate=True)
    assert rel(out.cpu().numpy(), base + lam * R.tv_grad(x, eps)) < FP32_BOUND
