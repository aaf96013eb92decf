"""Host-buffer calls run in chunks with the copies overlapped on separate
streams; every chunk runs the same kernels on the same data, so the
results equal the device-buffer calls bit for bit.  Covered: orbitals from
host memory (orbital ranges), V_xx phi into host memory (orbital ranges),
ACE apply with host psi/out over several ragged vector chunks, page-locked
and pageable host memory, both precision forms; the device results are
checked against the oracle."""
import numpy as np
import pytest

from oracle import ace as OA
from oracle import oracle as O
from paper_2208_06097_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.fixture(scope="module", params=[0, 1], ids=["plain", "mixed"])
def device_run(request, h2o8):
    """Device-buffer reference run of one form."""
    from paper_2208_06097_gb300 import sea
    dev = torch.device("cuda:0")
    ctx = sea.Context(h2o8.cell, h2o8.grid, cg_tol=1e-12, precision=request.param)
    phi = torch.from_numpy(h2o8.phi).to(dev)
    out = torch.empty_like(phi)
    ctx.set_orbitals(phi)
    exx = ctx.apply_vxx(out)
    ctx.build_ace()
    psi = synth.random_trial_vectors(77, h2o8.grid, 31)
    pd = torch.from_numpy(psi).to(dev)
    y = torch.empty_like(pd)
    ctx.apply_ace(pd, y)
    torch.cuda.synchronize()
    res = dict(precision=request.param, vxx=out.cpu().numpy(), exx=exx, psi=psi,
               y=y.cpu().numpy())
    ctx.close()
    return res


def test_device_run_matches_oracle(device_run, h2o8):
    ref = O.apply_vxx(h2o8.phi, h2o8.cell, O.Params(cg_tol=1e-12))
    scale = np.abs(ref["vxx"]).max()
    assert np.abs(device_run["vxx"] - ref["vxx"]).max() <= 1e-9 * scale
    F = h2o8.phi.reshape(h2o8.n_orb, -1)
    a = OA.build_ace(F, ref["vxx"].reshape(h2o8.n_orb, -1), h2o8.dV)
    yr = OA.apply_ace(a["Xi"], device_run["psi"].reshape(77, -1), h2o8.dV)
    assert np.abs(device_run["y"].reshape(77, -1) - yr).max() <= 1e-8 * np.abs(yr).max()


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_host_calls_equal_device_calls(device_run, h2o8, pinned):
    from paper_2208_06097_gb300 import sea
    wrap = _pinned if pinned else (lambda a: np.ascontiguousarray(a).copy())
    ctx = sea.Context(h2o8.cell, h2o8.grid, cg_tol=1e-12, precision=device_run["precision"])
    ctx.set_orbitals(wrap(h2o8.phi))
    vxx = wrap(np.full(h2o8.phi.shape, np.nan))
    exx = ctx.apply_vxx(vxx)
    assert exx == device_run["exx"]
    assert np.array_equal(vxx, device_run["vxx"])
    ctx.build_ace()
    y = wrap(np.full(device_run["psi"].shape, np.nan))
    ctx.apply_ace(wrap(device_run["psi"]), y)
    assert np.array_equal(y, device_run["y"])
    # a single-vector host call (one chunk shorter than the chunk size)
    y1 = wrap(np.full((1,) + h2o8.phi.shape[1:], np.nan))
    ctx.apply_ace(wrap(device_run["psi"][40:41]), y1)
    assert np.array_equal(y1[0], device_run["y"][40])
    ctx.close()


def test_host_apply_many_chunks(h2o8):
    """More vectors than 64 chunks of 32: the chunk size grows, nothing is
    dropped (ragged last chunk)."""
    from paper_2208_06097_gb300 import sea
    dev = torch.device("cuda:0")
    ctx = sea.Context(h2o8.cell, h2o8.grid, cg_tol=1e-10, precision=1)
    ctx.set_orbitals(torch.from_numpy(h2o8.phi).to(dev))
    ctx.apply_vxx(torch.empty(h2o8.phi.shape, dtype=torch.float64, device=dev))
    ctx.build_ace()
    nv = 64 * 32 + 45
    psi = _pinned(synth.random_trial_vectors(nv, h2o8.grid, 77))
    y = _pinned(np.full(psi.shape, np.nan))
    ctx.apply_ace(psi, y)
    pd = torch.from_numpy(psi).to(dev)
    yd = torch.empty_like(pd)
    ctx.apply_ace(pd, yd)
    assert np.array_equal(y, yd.cpu().numpy())
    ctx.close()
