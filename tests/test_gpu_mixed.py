"""The mixed-precision form (precision = 1: FP32 stencil sweeps and CG
vectors inside an FP64 iterative refinement) against the FP64 oracle.

Its stopping rule is applied to the true FP64 residual, so it meets the same
bounds as the FP64 path: at cg_tol = 1e-12 the spec bar
(max|dV_xx phi| <= 1e-9 Ha, rel|dE_xx| <= 1e-10), at 1e-8 the bound from
the stopping rule, and |dE_xx| <= 1e-6 Ha per molecule at the three
densities of the precision workload."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_06097_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(s, **prm):
    from paper_2208_06097_gb300 import sea
    with sea.Context(s.cell, s.grid, precision=1, **prm) as ctx:
        phi = torch.from_numpy(np.ascontiguousarray(s.phi)).cuda()
        out = torch.empty_like(phi)
        ctx.set_orbitals(phi)
        exx = ctx.apply_vxx(out)
        plan = ctx.plan()
        st = ctx.stats()
    return out.cpu().numpy(), exx, plan, st


def test_mixed_tight(h2o8):
    ref = O.apply_vxx(h2o8.phi, h2o8.cell, O.Params(cg_tol=1e-12))
    v, exx, plan, st = _run(h2o8, cg_tol=1e-12)
    np.testing.assert_array_equal(plan["pair"], ref["pair"])
    assert np.abs(v - ref["vxx"]).max() <= 1e-9
    assert abs(exx - ref["exx"]) <= 1e-10 * abs(ref["exx"])


def test_mixed_production(h2o8):
    ref = O.apply_vxx(h2o8.phi, h2o8.cell, O.Params())
    v, exx, plan, st = _run(h2o8)
    assert np.abs(v - ref["vxx"]).max() <= 5e-8 * np.abs(ref["vxx"]).max()
    assert abs(exx - ref["exx"]) <= 1e-8 * abs(ref["exx"])
    assert np.all(plan["iters"] > 0)


@pytest.mark.parametrize("name", ["h2o64_d04_128", "h2o64_d10_96", "h2o64_d17_80"])
def test_mixed_precision_workload_per_density(name):
    s = synth.make_config(name)
    ref = O.apply_vxx(s.phi, s.cell, O.Params())
    v, exx, plan, st = _run(s)
    n_mol = s.n_orb // 4
    assert abs(exx - ref["exx"]) / n_mol <= 1e-6
    assert np.abs(v - ref["vxx"]).max() <= 5e-8 * np.abs(ref["vxx"]).max()


def test_mixed_ace_matches_fp64_oracle(h2o8):
    # the mixed form's ACE contractions use FP32 error-free transformations;
    # their results must stay within FP64-class error of the dense oracle
    from oracle import ace as OA
    from paper_2208_06097_gb300 import sea
    ref = O.apply_vxx(h2o8.phi, h2o8.cell, O.Params(cg_tol=1e-12))
    F = h2o8.phi.reshape(h2o8.n_orb, -1)
    a = OA.build_ace(F, ref["vxx"].reshape(h2o8.n_orb, -1), h2o8.dV)
    with sea.Context(h2o8.cell, h2o8.grid, precision=1, cg_tol=1e-12) as ctx:
        phi = torch.from_numpy(h2o8.phi).cuda()
        out = torch.empty_like(phi)
        ctx.set_orbitals(phi)
        ctx.apply_vxx(out)
        ctx.build_ace()
        M, L = ctx.ace_matrices()
        psi = synth.random_trial_vectors(4, h2o8.grid, 12)
        y = np.empty_like(psi)
        ctx.apply_ace(psi, y)
        xi = torch.empty_like(phi)
        ctx.ace_vectors(xi)
        e_ace = ctx.stats()["exx_ace"]
    assert abs(e_ace - OA.exx_ace(F, a["Xi"], h2o8.dV)) <= 1e-10 * abs(e_ace)
    assert np.abs(M - a["M"]).max() <= 1e-9
    assert np.abs(L - a["L"]).max() <= 1e-9
    yr = OA.apply_ace(a["Xi"], psi.reshape(4, -1), h2o8.dV)
    assert np.abs(y.reshape(4, -1) - yr).max() <= 1e-9 * np.abs(yr).max()
    assert np.abs(xi.cpu().numpy().reshape(h2o8.n_orb, -1) - a["Xi"]).max() <= 1e-8 * np.abs(a["Xi"]).max()


def _mixed_ace_vs_oracle(s, n_vec=4):
    """Mixed-form M, L and V_ace psi against the FP64 oracle; returns the
    context statistics of the build."""
    from oracle import ace as OA
    from paper_2208_06097_gb300 import sea
    ref = O.apply_vxx(s.phi, s.cell, O.Params(cg_tol=1e-12))
    F = s.phi.reshape(s.n_orb, -1)
    a = OA.build_ace(F, ref["vxx"].reshape(s.n_orb, -1), s.dV)
    with sea.Context(s.cell, s.grid, precision=1, cg_tol=1e-12) as ctx:
        phi = torch.from_numpy(np.ascontiguousarray(s.phi)).cuda()
        out = torch.empty_like(phi)
        ctx.set_orbitals(phi)
        ctx.apply_vxx(out)
        ctx.build_ace()
        M, L = ctx.ace_matrices()
        psi = synth.random_trial_vectors(n_vec, s.grid, 21)
        y = np.empty_like(psi)
        ctx.apply_ace(psi, y)
        st = ctx.stats()
    assert np.abs(M - a["M"]).max() <= 1e-9 * max(1.0, np.abs(a["M"]).max())
    assert np.abs(L - a["L"]).max() <= 1e-9 * max(1.0, np.abs(a["L"]).max())
    yr = OA.apply_ace(a["Xi"], psi.reshape(n_vec, -1), s.dV)
    assert np.abs(y.reshape(n_vec, -1) - yr).max() <= 1e-9 * np.abs(yr).max()
    return st


def test_mixed_ace_odd_grid():
    # odd nx: rows are not 16-byte strided, so the contraction takes the
    # per-thread-load kernel instead of the TMA one; partial tiles on every axis
    s = synth.make_waters(4, 7.5, (41, 36, 44), seed=42)
    _mixed_ace_vs_oracle(s)


def test_mixed_ace_partial_blocks():
    # 40 orbitals: two 32 x 32 block columns in the Cholesky block tasks, the
    # second padded (8 rows of M, the identity beyond them in -Mbar)
    s = synth.make_waters(10, 8.5, 36, seed=77)
    assert s.n_orb == 40
    _mixed_ace_vs_oracle(s)


def test_mixed_ace_long_tile_lists():
    # a coarse grid puts more than 32 W rows on some tiles: those tiles are
    # expanded by the FP32 kernel, the others on the tensor cores
    s = synth.make_waters(64, 12.42, 32, seed=1001)
    st = _mixed_ace_vs_oracle(s, n_vec=40)
    assert st["ace_max_tile_list"] > 32, st["ace_max_tile_list"]
