"""sea_poisson_batch_noalloc: the box Poisson solver for callers that
cannot allocate device memory (host frameworks that own all device memory
through their own pool, processes with a device footprint fixed at
start-up).  It must give the same solutions as the allocating
sea_poisson_batch, on two calls in a row (the shared scratch keeps the
previous call's contents, which must not leak into the next), also with
the scratch filled to its capacity; and a caller that is capturing a CUDA
graph gets SEA_ERR_ARG with its capture left intact (the call is
synchronous, so it cannot be captured).

Collected last on purpose, so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

H = (0.25, 0.23, 0.27)


def _solve(exts, seed, noalloc, tol=1e-12):
    from paper_2208_06097_gb300 import sea
    rng = np.random.default_rng(seed)
    n = sum(e[0] * e[1] * e[2] for e in exts)
    rhs = torch.from_numpy(rng.normal(size=n)).cuda()
    x = torch.full_like(rhs, float("nan"))
    it, rc = sea.poisson_batch(H, exts, rhs, x, tol=tol, noalloc=noalloc)
    return x.cpu().numpy(), it, rc


@pytest.mark.parametrize("call", [0, 1])
def test_matches_allocating_entry_point_two_calls(call):
    # two different batches back to back: sizes and right-hand sides change
    exts = [[(13, 12, 11), (3, 5, 7), (16, 16, 16), (1, 1, 1)],
            [(9, 20, 6), (14, 14, 14), (2, 2, 30)]][call]
    for seed in (10 + call, 20 + call):
        xa, ita, rca = _solve(exts, seed, noalloc=False)
        xn, itn, rcn = _solve(exts, seed, noalloc=True)
        assert rca == 0 and rcn == 0
        assert np.all(np.isfinite(xn))
        assert np.abs(xn - xa).max() <= 1e-11 * max(1.0, np.abs(xa).max())
        np.testing.assert_array_equal(itn, ita)


def test_rejects_sizes_beyond_capacity():
    from paper_2208_06097_gb300 import sea
    rhs = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(sea.SeaError) as e:
        sea.poisson_batch(H, [(128, 128, 128)], rhs, rhs, noalloc=True)
    assert e.value.code == 9
    with pytest.raises(sea.SeaError) as e:
        sea.poisson_batch(H, [(1, 1, 1)] * 4097, rhs, rhs, noalloc=True)
    assert e.value.code == 9


@pytest.mark.parametrize("exts", [[(16, 64, 64)] * 16, [(2, 2, 2)] * 4096],
                         ids=["max_unknowns", "max_boxes"])
def test_exactly_at_capacity(exts):
    # 1,048,576 unknowns in 16 boxes, and exactly 4096 boxes: the vectors
    # and the box records fill their regions of the fixed layout
    for seed in (31, 32):
        xa, ita, rca = _solve(exts, seed, noalloc=False, tol=1e-8)
        xn, itn, rcn = _solve(exts, seed, noalloc=True, tol=1e-8)
        assert rca == 0 and rcn == 0
        assert np.all(np.isfinite(xn))
        assert np.abs(xn - xa).max() <= 1e-11 * max(1.0, np.abs(xa).max())
        np.testing.assert_array_equal(itn, ita)


def test_refused_under_stream_capture():
    from paper_2208_06097_gb300 import sea
    exts = [(5, 6, 7)]
    _solve(exts, 3, noalloc=True)  # the device's first call: address look-up
    rhs = torch.ones(5 * 6 * 7, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(rhs)
    y = torch.zeros(4, dtype=torch.float64, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=torch.cuda.Stream()):
        y.add_(1.0)
        with pytest.raises(sea.SeaError) as e:
            sea.poisson_batch(H, exts, rhs, x, noalloc=True,
                              stream=torch.cuda.current_stream().cuda_stream)
        y.add_(1.0)
    assert e.value.code == 1
    g.replay()  # the capture survived: both adds replay, nothing was solved
    torch.cuda.synchronize()
    assert torch.all(y == 2.0)
    assert torch.all(x == 0.0)
    # and the entry point works again outside the capture
    xa, _, _ = _solve(exts, 4, noalloc=False)
    xn, _, rcn = _solve(exts, 4, noalloc=True)
    assert rcn == 0 and np.abs(xn - xa).max() <= 1e-11 * max(1.0, np.abs(xa).max())
