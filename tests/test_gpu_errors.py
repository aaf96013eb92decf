"""Error statuses of the C ABI, triggered from the host (no GPU fault):
non-finite or unnormalized orbitals, call-order violations, a CG iteration
cap, a spent CG time budget, and a non-positive-definite -Mbar (App. A:
Cholesky fails) from an orbital that is identically zero."""
import numpy as np
import pytest

from oracle import ace as OA
from paper_2208_06097_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def small():
    return synth.make_waters(2, 6.21, 32, seed=77)


def _ctx(s, **kw):
    from paper_2208_06097_gb300 import sea
    return sea.Context(s.cell, s.grid, **kw)


def test_nonfinite_orbitals_rejected(small):
    from paper_2208_06097_gb300 import sea
    phi = small.phi.copy()
    phi[1, 3, 4, 5] = np.nan
    with _ctx(small) as ctx:
        with pytest.raises(sea.SeaError) as e:
            ctx.set_orbitals(phi)
        assert e.value.code == 8
        # the context is still usable
        ctx.set_orbitals(np.ascontiguousarray(small.phi))
        out = np.empty_like(small.phi)
        ctx.apply_vxx(out)


def test_call_order(small):
    from paper_2208_06097_gb300 import sea
    with _ctx(small) as ctx:
        out = np.empty_like(small.phi)
        with pytest.raises(sea.SeaError) as e:
            ctx.apply_vxx(out)
        assert e.value.code == 2
        ctx.set_orbitals(np.ascontiguousarray(small.phi))
        with pytest.raises(sea.SeaError) as e:
            ctx.build_ace()
        assert e.value.code == 2
        with pytest.raises(sea.SeaError) as e:
            ctx.apply_ace(np.ascontiguousarray(small.phi), out)
        assert e.value.code == 2


def test_bad_arguments(small):
    from paper_2208_06097_gb300 import sea
    with pytest.raises(sea.SeaError) as e:
        sea.Context(small.cell, (4, 32, 32))
    assert e.value.code == 1
    with pytest.raises(sea.SeaError) as e:
        sea.Context(small.cell, small.grid, lmax=7)
    assert e.value.code == 1
    with pytest.raises(sea.SeaError) as e:
        sea.Context((0.0, 1.0, 1.0), small.grid)
    assert e.value.code == 1


def test_cg_cap_reported_results_written(small):
    with _ctx(small, cg_max_iter=2) as ctx:
        ctx.set_orbitals(np.ascontiguousarray(small.phi))
        out = np.full_like(small.phi, np.nan)
        ctx.apply_vxx(out, allow_cap=True)
        assert np.all(np.isfinite(out))
        plan = ctx.plan()
        assert np.all(plan["iters"] == -2)


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_orbital_makes_mbar_singular(small, precision):
    # Cholesky only (ace_decomp = 1): the zero pivot is reported, by the
    # FP64 kernel chain and by the mixed form's one-launch block tasks
    from paper_2208_06097_gb300 import sea
    phi = np.ascontiguousarray(small.phi.copy())
    phi[0] = 0.0
    with _ctx(small, ace_decomp=1, orth_tol=0.0, precision=precision) as ctx:  # norm 0
        ctx.set_orbitals(phi)
        out = np.empty_like(phi)
        ctx.apply_vxx(out)
        assert np.all(out[0] == 0)
        with pytest.raises(sea.SeaError) as e:
            ctx.build_ace()
        assert e.value.code == 6
    F = phi.reshape(phi.shape[0], -1)
    with pytest.raises(OA.NotPositiveDefinite):
        OA.build_ace(F, out.reshape(phi.shape[0], -1), small.dV)


def test_unnormalized_orbital_rejected(small):
    from paper_2208_06097_gb300 import sea
    phi = np.ascontiguousarray(small.phi.copy())
    phi[2] *= 1.0 + 1e-5  # <phi|phi> = 1 + 2e-5
    for dev in (False, True):
        arg = torch.from_numpy(phi).cuda() if dev else phi
        with _ctx(small) as ctx:
            with pytest.raises(sea.SeaError) as e:
                ctx.set_orbitals(arg)
            assert e.value.code == 8
            ctx.set_orbitals(np.ascontiguousarray(small.phi))  # still usable
    # within the tolerance, and with the check switched off, accepted
    phi[2] = small.phi[2] * (1.0 + 2e-7)
    with _ctx(small) as ctx:
        ctx.set_orbitals(phi)
    phi[2] = small.phi[2] * 2.0
    with _ctx(small, orth_tol=0.0) as ctx:
        ctx.set_orbitals(phi)


def test_cg_time_budget(small):
    # a budget of 1 ns is spent before the CTAs take their next pair: the
    # call reports SEA_ERR_TIMEOUT and the context stays usable
    from paper_2208_06097_gb300 import sea
    out = np.empty_like(small.phi)
    for precision in (0, 1):
        with _ctx(small, timeout_ms=1e-6, precision=precision) as ctx:
            ctx.set_orbitals(np.ascontiguousarray(small.phi))
            for _ in range(2):
                with pytest.raises(sea.SeaError) as e:
                    ctx.apply_vxx(out)
                assert e.value.code == 7
            with pytest.raises(sea.SeaError) as e:
                ctx.build_ace()  # no valid V_xx result
            assert e.value.code == 2
        with _ctx(small, timeout_ms=60000.0, precision=precision) as ctx:
            ctx.set_orbitals(np.ascontiguousarray(small.phi))
            ctx.apply_vxx(out)
            assert np.all(np.isfinite(out))
    with pytest.raises(sea.SeaError) as e:
        _ctx(small, timeout_ms=-1.0)
    assert e.value.code == 1
