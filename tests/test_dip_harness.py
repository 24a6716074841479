"""The DIP harness: U-Net shapes and the complex view on the CPU; on the GPU, a
few stochastic steps lower the loss, every coil is visited once per epoch, and a
checkpoint resumes the run bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2408_02367_gb300 import synth


def test_unet_shapes_and_complex_view():
    from paper_2408_02367_gb300 import dip
    net = dip.UNet3D(6, 6, ch=(4, 8, 8, 16))
    z = torch.rand(1, 6, 16, 8, 24) * 0.1
    g = net(z)
    assert g.shape == (1, 6, 16, 8, 24)
    x = dip.to_complex(g)
    assert x.shape == (3, 16, 8, 24) and x.dtype == torch.complex64
    assert torch.equal(x[1].real, g[0, 2]) and torch.equal(x[1].imag, g[0, 3])


@pytest.mark.gpu
def test_dip_runner_descends_visits_every_coil_and_resumes():
    from paper_2408_02367_gb300 import build, dip, op
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.backends.cudnn.deterministic = True
    torch.backends.cudnn.benchmark = False
    n, K, C, T = (16, 16, 16), 3, 5, 12
    x_true = synth.ellipsoid_phantom(n, K)
    S = synth.coil_maps(n, C)
    V = synth.subspace_basis(T, K)
    om, fr = synth.spiral_trajectory(T, 1, 300)
    A = op.make_operator(om, fr, n, 4, 1.25, V, S, max_batch=2)
    dev = A.device
    ci_all = [torch.tensor(c, dtype=torch.int32, device=dev) for c in ([0, 1], [2, 3], [4])]
    xt = torch.from_numpy(x_true).to(dev)
    y = torch.cat([A.forward(xt, c) for c in ci_all]).contiguous()

    def fresh():
        torch.manual_seed(3)
        net = dip.UNet3D(2 * K, 2 * K, ch=(8, 16, 16, 32)).to(dev)
        z = torch.rand((1, 2 * K) + n, generator=torch.Generator().manual_seed(4)).mul_(0.1).to(dev)
        return dip.DipRunner(A, y, net, z, B=2, lr=1e-3, lam_tv=1e-4, seed=5)

    def full_loss(run):
        with torch.no_grad():
            x = dip.to_complex(run.net(run.z))
            return sum(float(torch.sum(torch.abs(A.forward(x, c) - y[c.long()]) ** 2)) for c in ci_all)

    r = fresh()
    l0 = full_loss(r)
    seen = []
    losses = []
    for _ in range(3):                                   # one epoch of 5 coils: minibatches 2, 2, 1
        seen += r.perm[r.pos:r.pos + 2].tolist() if r.pos < C else []
        losses.append(float(r.step()))
    assert sorted(seen) == list(range(C)) and r.epoch == 0 and r.pos == C
    for _ in range(27):
        losses.append(float(r.step()))
    assert r.epoch == 9
    l1 = full_loss(r)
    assert l1 < 0.9 * l0, (l0, l1, losses)

    # checkpoint after 30 steps, run 5 more; a fresh runner loaded from the checkpoint repeats them
    ck = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in r.state_dict().items()}
    import copy
    ck["net"] = copy.deepcopy(ck["net"])
    ck["opt"] = copy.deepcopy(ck["opt"])
    after = [float(r.step()) for _ in range(5)]
    r2 = fresh()
    r2.load_state_dict(ck)
    again = [float(r2.step()) for _ in range(5)]
    assert again == after, (after, again)
