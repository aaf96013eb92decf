"""The C ABI library loads and exports every entry point that
include/sea.h declares (no GPU work: only symbol lookup)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sea.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sea_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libsea():
    from paper_2208_06097_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("sea_create", "sea_set_orbitals", "sea_apply_vxx", "sea_build_ace",
                 "sea_apply_ace", "sea_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(libsea):
    missing = [n for n in _declared() if not hasattr(libsea, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2208_06097_gb300 import sea
    assert sorted(sea.EXPORTS) == _declared()


def test_default_params_without_gpu(libsea):
    from paper_2208_06097_gb300 import sea
    p = sea.default_params()
    assert p.lmax == 6 and p.fd_order == 12 and abs(p.eps - 10 ** -3.5) < 1e-18
    assert p.delta == 1e-3 and p.cg_tol == 1e-8


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2208_06097_gb300 import sea
    monkeypatch.setattr(sea, "_LIB", None)
    monkeypatch.setattr(sea, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        sea.lib()
