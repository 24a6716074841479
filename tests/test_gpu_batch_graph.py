"""Batched multi-volume calls and the CUDA-graph captured DIP step, against the
plain per-item calls (which the parity tests pin to the FP64 oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nufft as O
from paper_2408_02367_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2408_02367_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _volume(n, W, sigma, K, C, T, arm_len, seed, tuning=None):
    from paper_2408_02367_gb300 import op
    x = synth.ellipsoid_phantom(n, K, seed=seed)
    S = synth.coil_maps(n, C)
    V = synth.subspace_basis(T, K, seed=seed + 10)
    omega, frame = synth.spiral_trajectory(T, 1, arm_len)
    A = op.make_operator(omega, frame, n, W, sigma, V, S, max_batch=4, tuning=tuning)
    return A, x


def test_batched_items_equal_single_calls():
    from paper_2408_02367_gb300 import op
    vols = [_volume((16, 16, 16), 4, 1.25, 5, 4, 20, 256, 1),
            _volume((20, 24, 18), 6, 2.0, 3, 3, 10, 300, 2),
            _volume((12, 12, 12), 4, 2.0, 5, 2, 8, 200, 3)]
    coil_sets = [[3, 1], [2], [1, 0, 1], [0]]
    plan_of = [0, 1, 2, 0]            # two items share the first plan
    items = []
    for i, (pi, cs) in enumerate(zip(plan_of, coil_sets)):
        A, x = vols[pi]
        items.append((A, _t(x), _t(np.array(cs, np.int32)), None))
    ys = op.forward_batched(items)
    for (A, x, c, _), y in zip(items, ys):
        assert torch.equal(y, A.forward(x, c))
    adj_items = [(A, y, c, None, False) for (A, _, c, _), y in zip(items, ys)]
    outs = op.adjoint_batched(adj_items)
    for (A, y, c, _, _), o in zip(adj_items, outs):
        assert torch.equal(o, A.adjoint(y, c))
    # accumulate into a shared output of one plan across two items
    A0, _ = vols[0]
    acc = torch.zeros_like(outs[0])
    op.adjoint_batched([(A0, ys[0], items[0][2], acc, True), (A0, ys[3], items[3][2], acc, True)])
    ref = A0.adjoint(ys[0], items[0][2]) + A0.adjoint(ys[3], items[3][2])
    assert (torch.linalg.norm(acc - ref) / torch.linalg.norm(ref)).item() < 1e-6
    for A, _ in vols:
        assert A.status() == 0


def test_batched_rejects_bad_item_before_launching():
    from paper_2408_02367_gb300 import op
    A, x = _volume((10, 10, 10), 4, 2.0, 2, 2, 4, 100, 4)
    xt = _t(x)
    good = torch.tensor([0], dtype=torch.int32, device="cuda")
    n0 = op.launch_count()
    bad = (A, xt, torch.zeros(9, dtype=torch.int32, device="cuda"), None)   # B = 9 > max_batch
    with pytest.raises(ValueError):
        op.forward_batched([(A, xt, good, None), bad])
    assert op.launch_count() == n0


def test_graph_replay_equals_eager_step():
    from paper_2408_02367_gb300 import graph, op
    n, W, sigma, K, C, T = (24, 24, 24), 4, 1.25, 5, 4, 30
    x = synth.ellipsoid_phantom(n, K)
    S = synth.coil_maps(n, C)
    V = synth.subspace_basis(T, K)
    omega, frame = synth.spiral_trajectory(T, 1, 512)
    A = op.make_operator(omega, frame, n, W, sigma, V, S, max_batch=2)
    y_meas = torch.stack([A.forward(_t(synth.ellipsoid_phantom(n, K, seed=7)),
                                    torch.tensor([c], dtype=torch.int32, device="cuda"))[0] for c in range(C)])
    g = graph.DipStepGraph(A, y_meas, _t(x), B=2)
    assert g.launches_per_step == A.launches_per_step(2)
    xe = _t(x).requires_grad_(True)
    for cs in ([1, 3], [0, 2], [3, 3]):
        ci = torch.tensor(cs, dtype=torch.int32, device="cuda")
        loss, grad = g.step(ci)
        xe.grad = None
        le = op.dc_loss(A, xe, ci, y_meas)
        le.backward()
        torch.cuda.synchronize()
        assert torch.equal(loss, le.detach())
        assert torch.equal(grad, xe.grad)
    # a new x through the static input
    x2 = _t(synth.ellipsoid_phantom(n, K, seed=11))
    loss, grad = g.step(torch.tensor([2, 0], dtype=torch.int32, device="cuda"), x=x2)
    x2e = x2.clone().requires_grad_(True)
    le = op.dc_loss(A, x2e, torch.tensor([2, 0], dtype=torch.int32, device="cuda"), y_meas)
    le.backward()
    assert torch.equal(grad, x2e.grad)
    assert A.status() == 0


def test_one_launch_per_stage_for_a_mixed_size_batch():
    """Three volumes of different grid sizes (80^3, 120 x 100 x 80, 80 x 160 x 96 grids), W=4, K=5,
    uneven minibatches, two items sharing a plan: the batched forward is 4 launches and the batched
    adjoint 4 launches, each item's result equals its own single call bit for bit (the same per-unit
    bodies run), and each item matches the FP64 oracle."""
    from paper_2408_02367_gb300 import op
    from tests.test_gpu_parity import FP32_BOUND, assert_close
    specs = [((64, 64, 64), 5, 12, 300, 11), ((96, 80, 64), 4, 10, 400, 12), ((64, 128, 76), 6, 8, 256, 13)]
    vols = []
    for n, C, T, arm, seed in specs:
        x = synth.ellipsoid_phantom(n, 5, seed=seed)
        S = synth.coil_maps(n, C)
        V = synth.subspace_basis(T, 5, seed=seed + 10)
        omega, frame = synth.spiral_trajectory(T, 1, arm)
        A = op.make_operator(omega, frame, n, 4, 1.25, V, S, max_batch=4)
        vols.append(dict(A=A, x=x, S=S, V=V, omega=omega, frame=frame, n=n))
    coil_sets = [[3, 1], [2], [0, 4, 1], [2, 0]]
    plan_of = [0, 1, 2, 0]            # items 0 and 3 share the first plan (2 + 2 coils <= max_batch 4)
    items = [(vols[p]["A"], _t(vols[p]["x"]), _t(np.array(cs, np.int32)), None) for p, cs in zip(plan_of, coil_sets)]
    n0 = op.launch_count()
    ys = op.forward_batched(items)
    assert op.launch_count() - n0 == 4
    for (A, x, c, _), y in zip(items, ys):
        assert torch.equal(y, A.forward(x, c))
    rs = [_t(synth.random_complex(tuple(y.shape), 40 + i)) for i, y in enumerate(ys)]
    adj = [(A, r, c, None, False) for (A, _, c, _), r in zip(items, rs)]
    n0 = op.launch_count()
    outs = op.adjoint_batched(adj)
    assert op.launch_count() - n0 == 4
    for (A, r, c, _, _), o in zip(adj, outs):
        assert torch.equal(o, A.adjoint(r, c))
    for q, (p, cs) in enumerate(zip(plan_of, coil_sets)):
        v = vols[p]
        geo = O.Geometry(v["n"], 4, 1.25)
        y_ref = O.gridding_forward(geo, v["x"], v["S"], v["V"], v["omega"], v["frame"], cs)
        assert_close(ys[q].cpu().numpy(), y_ref, FP32_BOUND, f"batched item {q} forward")
        a_ref = O.gridding_adjoint(geo, rs[q].cpu().numpy(), v["S"], v["V"], v["omega"], v["frame"], cs)
        assert_close(outs[q].cpu().numpy(), a_ref, FP32_BOUND, f"batched item {q} adjoint")
    for v in vols:
        assert v["A"].status() == 0


def test_tiled_interpolation_batched_equals_single_calls():
    """Plans with the tiled interpolation, of different grid sizes, share one launch per
    stage: the batched forward is 4 launches and each item equals its own single call bit
    for bit (the same per-work-item body runs)."""
    from paper_2408_02367_gb300 import op
    tun = {"spread_bins": (4, 4, 4), "spread_chunk": 256, "interp_tiled": 1}
    vols = [_volume((64, 64, 64), 4, 1.25, 5, 4, 12, 300, 21, tuning=tun),          # grids 80^3,
            _volume((96, 80, 64), 4, 1.25, 5, 3, 10, 400, 22, tuning=tun),          # 120 x 100 x 80,
            _volume((64, 128, 76), 4, 1.25, 5, 4, 8, 256, 23, tuning=tun)]         # 80 x 160 x 96
    coil_sets = [[3, 1], [2, 0, 1], [0]]
    items = [(A, _t(x), _t(np.array(cs, np.int32)), None) for (A, x), cs in zip(vols, coil_sets)]
    n0 = op.launch_count()
    ys = op.forward_batched(items)
    assert op.launch_count() - n0 == 4
    for (A, x, c, _), y in zip(items, ys):
        assert torch.equal(y, A.forward(x, c))
        assert A.status() == 0


@pytest.mark.parametrize("bins", [(8, 4, 8), (4, 4, 4), (4, 4, 8)])
def test_batched_items_beyond_a_plans_workspace_run_in_waves(bins):
    """Items of one plan whose minibatches exceed its max_batch together run in waves (one launch
    set each); accumulate adds into a shared output; results equal the single calls (for every
    spread bin width)."""
    from paper_2408_02367_gb300 import op
    A, x = _volume((38, 51, 38), 4, 1.25, 5, 6, 12, 300, 5,
                   tuning={"spread_bins": bins, "spread_chunk": 256})      # grid 48 x 64 x 48
    xt = _t(x)
    cs = [[0, 1, 2], [3, 4], [5], [1, 3, 5, 0]]               # 3 + 2 + 1 + 4 = 10 > max_batch 4
    items = [(A, xt, _t(np.array(c, np.int32)), None) for c in cs]
    n0 = op.launch_count()
    ys = op.forward_batched(items)
    assert op.launch_count() - n0 == 12                      # {3}, {2, 1}, {4}: three waves of 4 launches
    for (_, _, c, _), y in zip(items, ys):
        assert torch.equal(y, A.forward(xt, c))
    acc = torch.zeros_like(xt)
    op.adjoint_batched([(A, y, c, acc, True) for (_, _, c, _), y in zip(items, ys)])
    ref = torch.zeros_like(xt)
    for (_, _, c, _), y in zip(items, ys):
        A.adjoint(y, c, out=ref, accumulate=True)
    assert (torch.linalg.norm(acc - ref) / torch.linalg.norm(ref)).item() < 1e-6
    assert A.status() == 0
