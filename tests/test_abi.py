"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point (no GPU needed)."""
import ctypes

import pytest

from tests._helpers import ensure_built, header_functions


def test_library_builds_and_exports_every_declared_symbol():
    path = ensure_built()
    lib = ctypes.CDLL(path)
    names = header_functions()
    assert "lobpcg_create" in names and "lobpcg_solve" in names and "lobpcg_apply_H" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_0707_3405_gb300 as lg
    ensure_built()
    assert lg.load() is not None
    monkeypatch.setattr(lg, "_lib", None)
    monkeypatch.setattr(lg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        lg.load()


def test_default_options_without_gpu():
    import paper_0707_3405_gb300 as lg
    ensure_built()
    o = lg.default_options()
    assert o.block_size == 64 and o.nline == 4 and o.precision == lg.FP64 and abs(o.tol - 1e-8) < 1e-20
    assert o.fp64_gemm == 0 and abs(o.mixed_early - 1e-3) < 1e-20
