"""GPU tests of the learned warm start: the CUDA network's forward pass and
gradients against the oracle's float64 PyTorch network on the same
(BF16-rounded) weights, training on collected pair solves, and the CG
started from the network's guesses finishing at the same solution as the
CG started from zero."""
import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

P3 = 32 ** 3


def _batch(rng, B):
    x = np.zeros((B, 2, 32, 32, 32), np.float32)
    x[:, 0] = rng.standard_normal((B, 32, 32, 32))
    x[:, 1, 4:27, 6:25, 3:29] = 1.0  # a box
    t = rng.standard_normal((B, 32, 32, 32)).astype(np.float32)
    return x, t


@pytest.fixture(scope="module")
def net():
    from paper_2208_06097_gb300 import sea
    n = sea.WarmStartNet(width=4, seed=7)
    yield n
    n.close()


def test_weight_count(net):
    assert net.num_weights() == U.num_weights(4)


def test_forward_matches_oracle(net, rng):
    x, _ = _batch(rng, 2)
    out = np.zeros((2, 32, 32, 32), np.float32)
    net.forward(x, out)
    w = net.get_weights()
    ref = U.forward(torch.as_tensor(x.astype(np.float64)), U.unpack(w, 4)).numpy()
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() <= 2e-5 * scale
    # device tensors give the same result
    xd = torch.from_numpy(x).cuda()
    od = torch.empty((2, 32, 32, 32), dtype=torch.float32, device="cuda")
    net.forward(xd, od)
    assert np.array_equal(od.cpu().numpy(), out)


def test_gradient_matches_oracle(net, rng):
    x, t = _batch(rng, 2)
    loss, g = net.loss_grad(x, t)
    w = net.get_weights()
    L, gref, _ = U.loss_and_grad(w, 4, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - L) <= 1e-5 * abs(L)
    off = 0
    for ci, co, k in U.layer_dims(4):
        for nw in (co * ci * (27 if k == 3 else 1), co):
            a, b = g[off:off + nw], gref[off:off + nw]
            assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max() + 1e-9, (ci, co, k, nw)
            off += nw
    # deterministic: the same call gives the same bits
    loss2, g2 = net.loss_grad(x, t)
    assert loss2 == loss and np.array_equal(g, g2)


@pytest.fixture(scope="module")
def trained(h2o8):
    """A width-8 network trained on the (H2O)8 pair solves (plain CG)."""
    from paper_2208_06097_gb300 import sea
    dev = torch.device("cuda:0")
    net = sea.WarmStartNet(width=8, seed=1)
    ctx = sea.Context(h2o8.cell, h2o8.grid, cg_tol=1e-12)
    phi = torch.from_numpy(h2o8.phi).to(dev)
    ctx.set_orbitals(phi)
    cold = torch.empty_like(phi)
    ecold = ctx.apply_vxx(cold)
    it_cold = ctx.plan()["iters"]
    n = net.collect(ctx)
    assert n == len(it_cold)
    first = net.train(1, batch=8, lr=2e-3, seed=3)
    last = net.train(300, batch=8, lr=2e-3, seed=4)
    yield dict(net=net, ctx=ctx, phi=phi, cold=cold.cpu().numpy(), ecold=ecold, it_cold=it_cold,
               first=first, last=last)
    ctx.close()
    net.close()


def test_training_reduces_loss(trained):
    assert trained["last"] < 0.5 * trained["first"], (trained["first"], trained["last"])


@pytest.mark.parametrize("precision", [0, 1], ids=["plain", "mixed"])
def test_warm_start_same_solution_fewer_iterations(trained, h2o8, precision):
    from paper_2208_06097_gb300 import sea
    net = trained["net"]
    ctx = sea.Context(h2o8.cell, h2o8.grid, cg_tol=1e-12, precision=precision, warm_start=1)
    net.attach(ctx)
    ctx.set_orbitals(trained["phi"])
    out = torch.empty_like(trained["phi"])
    e = ctx.apply_vxx(out)
    it_warm = ctx.plan()["iters"]
    scale = np.abs(trained["cold"]).max()
    assert np.abs(out.cpu().numpy() - trained["cold"]).max() <= 1e-9 * scale
    assert abs(e - trained["ecold"]) <= 1e-10 * abs(trained["ecold"])
    if precision == 0:
        assert it_warm.sum() < trained["it_cold"].sum(), (it_warm.sum(), trained["it_cold"].sum())
    sea.WarmStartNet.detach(ctx)
    ctx.close()


def test_warm_start_mixed_production_tolerance(trained, h2o8):
    # At cg_tol = 1e-8 the mixed form keeps x and the true residual in
    # double-float: the guess enters split into FP32 pairs and r = b - A x0 is
    # formed in double-float.  Same bound as the cold solve at that tolerance
    # (the stopping rule), against the tight FP64 solution.
    from paper_2208_06097_gb300 import sea
    net = trained["net"]
    ctx = sea.Context(h2o8.cell, h2o8.grid, cg_tol=1e-8, precision=1, warm_start=1)
    net.attach(ctx)
    ctx.set_orbitals(trained["phi"])
    out = torch.empty_like(trained["phi"])
    e = ctx.apply_vxx(out)
    scale = np.abs(trained["cold"]).max()
    assert np.abs(out.cpu().numpy() - trained["cold"]).max() <= 5e-8 * scale
    assert abs(e - trained["ecold"]) <= 1e-8 * abs(trained["ecold"])
    sea.WarmStartNet.detach(ctx)
    ctx.close()


def test_warm_start_needs_a_model(h2o8):
    from paper_2208_06097_gb300 import sea
    ctx = sea.Context(h2o8.cell, h2o8.grid, warm_start=1)
    ctx.set_orbitals(torch.from_numpy(h2o8.phi).cuda())
    with pytest.raises(sea.SeaError):
        ctx.apply_vxx(torch.empty((h2o8.n_orb,) + h2o8.phi.shape[1:], dtype=torch.float64,
                                  device="cuda"))
    ctx.close()
