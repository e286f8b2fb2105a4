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


def _raw_create(lib, lg, cell=True, a=10.0, N=16, ecut=5.0, nk=1, kpts=None, vloc=None, nproj=0, proj_E=None,
                opt=None):
    import numpy as np
    h = ctypes.c_void_p(12345)
    kp = np.zeros((max(nk, 1), 3)) if kpts is None else np.ascontiguousarray(kpts, dtype=np.float64)
    v = np.zeros((N, N, N)) if vloc is None else np.ascontiguousarray(vloc, dtype=np.float64)
    E = None if proj_E is None else np.ascontiguousarray(proj_E, dtype=np.float64)
    c = lg.Cell(a, N, ecut)
    rc = lib.lobpcg_create(ctypes.byref(h), ctypes.byref(c) if cell else None, nk, kp.ctypes.data,
                           v.ctypes.data, nproj, None if E is None else E.ctypes.data, None,
                           ctypes.byref(opt) if opt is not None else None, None)
    msg = (lib.lobpcg_last_error(None) or b"").decode()
    return rc, h.value, msg


def test_create_rejects_bad_arguments_before_any_device_call():
    """Argument errors come back as status codes with a message and a NULL handle, before the
    library touches a device (this runs without a GPU)."""
    import numpy as np
    import paper_0707_3405_gb300 as lg
    ensure_built()
    lib = lg.load()
    ERR_ARG, ERR_UNSUPPORTED = -1, -6

    def bad_opt(**kw):
        o = lg.default_options()
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    cases = [
        (dict(cell=False), ERR_ARG, "must not be NULL"),
        (dict(a=0.0), ERR_ARG, "a and ecut"),
        (dict(ecut=-1.0), ERR_ARG, "a and ecut"),
        (dict(nk=0), ERR_ARG, "nk must be"),
        (dict(nproj=3), ERR_ARG, "projector"),
        (dict(N=7), ERR_UNSUPPORTED, "product of 2, 3 and 5"),
        (dict(N=512), ERR_UNSUPPORTED, "product of 2, 3 and 5"),
        (dict(vloc=np.full((16, 16, 16), np.nan)), ERR_ARG, "vloc_r"),
        (dict(kpts=np.array([[0.0, np.inf, 0.0]])), ERR_ARG, "k-point"),
        (dict(nproj=2, proj_E=np.array([1.0, np.nan])), ERR_ARG, "proj_E"),
        (dict(opt=bad_opt(block_size=0)), ERR_ARG, "block_size"),
        (dict(opt=bad_opt(block_size=2000)), ERR_ARG, "block_size too large"),
        (dict(opt=bad_opt(nline=0)), ERR_ARG, "nline"),
        (dict(opt=bad_opt(precision=7)), ERR_ARG, "precision"),
        (dict(opt=bad_opt(tol=0.0)), ERR_ARG, "tol"),
        (dict(opt=bad_opt(tol=float("nan"))), ERR_ARG, "tol"),
        (dict(opt=bad_opt(nbuf=-1)), ERR_ARG, "nbuf"),
        (dict(opt=bad_opt(gemm_split=1)), ERR_UNSUPPORTED, "BF16x3"),
        (dict(opt=bad_opt(gemm_split=5)), ERR_ARG, "gemm_split"),
        (dict(opt=bad_opt(mixed_early=-1.0)), ERR_ARG, "mixed_early"),
        (dict(opt=bad_opt(fp64_gemm=4)), ERR_ARG, "fp64_gemm"),
    ]
    for kw, code, text in cases:
        rc, handle, msg = _raw_create(lib, lg, **kw)
        assert rc == code, (kw, rc, msg)
        assert handle is None, kw
        assert text in msg, (kw, msg)
    assert lib.lobpcg_create(None, None, 1, None, None, 0, None, None, None, None) == ERR_ARG


def test_handle_calls_reject_null_handle():
    import paper_0707_3405_gb300 as lg
    ensure_built()
    lib = lg.load()
    assert lib.lobpcg_npw(None, 0) == -1
    assert lib.lobpcg_set_stream(None, None) == -1
    assert lib.lobpcg_set_options(None, None) == -1
    assert lib.lobpcg_set_projectors(None, 0, None) == -1
    assert lib.lobpcg_solve(None, 64, None, None, None, None) == -1
    assert lib.lobpcg_apply_H(None, 0, None, None, 1, 0) == -1
    lib.lobpcg_destroy(None)


def test_kernel_entry_points_check_arguments_without_a_device():
    """The lobpcg_k_* calls reject bad precisions, sizes, pointers and leading dimensions
    with ERR_ARG before any device work; empty GEMM outputs are no-ops."""
    import paper_0707_3405_gb300 as lg
    ensure_built()
    lib = lg.load()
    C128, DF32, C64, ERR_ARG = 0, 2, 1, -1
    p = ctypes.c_void_p(0x1000)   # never dereferenced: every call below fails or returns first

    def msg():
        return (lib.lobpcg_k_last_error() or b"").decode()

    assert lib.lobpcg_k_gemm_cn(9, 4, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None) == ERR_ARG and "precision" in msg()
    assert lib.lobpcg_k_gemm_cn(9, 0, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None) == ERR_ARG
    assert lib.lobpcg_k_gemm_cn(C128, -1, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None) == ERR_ARG and "negative" in msg()
    assert lib.lobpcg_k_gemm_cn(C64, 4, 4, 8, 1.0, p, 7, p, 8, 0.0, p, 4, None) == ERR_ARG and "leading" in msg()
    assert lib.lobpcg_k_gemm_cn(DF32, 4, 4, 8, 1.0, None, 8, p, 8, 0.0, p, 4, None) == ERR_ARG
    assert lib.lobpcg_k_gemm_cn(C128, 0, 4, 8, 1.0, None, 0, None, 0, 0.0, None, 0, None) == 0
    assert lib.lobpcg_k_gram_lower(C64, 4, 8, p, 8, p, 8, p, 4, None) == ERR_ARG and "precision" in msg()
    assert lib.lobpcg_k_gram_lower(C128, 4, 8, p, 8, p, 8, p, 3, None) == ERR_ARG
    assert lib.lobpcg_k_gram_lower(DF32, 0, 8, None, 8, None, 8, None, 0, None) == 0
    assert lib.lobpcg_k_gemm_nn(9, 4, 4, 4, 1.0, p, 4, p, 4, 0.0, None, 0, p, 4, None) == ERR_ARG
    assert lib.lobpcg_k_gemm_nn(C128, 4, 4, 4, 1.0, p, 4, p, 4, 1.0, None, 0, p, 4, None) == ERR_ARG
    assert lib.lobpcg_k_gemm_nn(C64, 8, 4, 4, 1.0, p, 7, p, 4, 0.0, None, 0, p, 8, None) == ERR_ARG
    assert lib.lobpcg_k_gemm_nn(DF32, 8, 0, 4, 1.0, None, 0, None, 0, 0.0, None, 0, None, 0, None) == 0
    th = ctypes.c_void_p(0x2000)
    for fn in (lib.lobpcg_k_rayleigh_ritz, lib.lobpcg_k_rayleigh_ritz_df32, lib.lobpcg_k_rayleigh_ritz32):
        assert fn(4, 5, p, p, 1e-12, th, p, None, None) == ERR_ARG and "m <= n" in msg()
        assert fn(5000, 5, p, p, 1e-12, th, p, None, None) == ERR_ARG
        assert fn(4, 2, None, p, 1e-12, th, p, None, None) == ERR_ARG and "NULL" in msg()
    assert lib.lobpcg_k_heev(0, p, th, p, None) == ERR_ARG
    assert lib.lobpcg_k_heev(4, p, None, p, None) == ERR_ARG
    assert lib.lobpcg_k_set_gemm_mode(1) == ERR_ARG and "gemm mode" in msg()
    assert lib.lobpcg_k_set_gemm_mode(7) == ERR_ARG


def test_binding_structs_match_the_library_layout():
    """lobpcg_cell, lobpcg_options and lobpcg_stats as compiled have the sizes of the binding's
    ctypes structures (load() refuses a library that disagrees)."""
    import paper_0707_3405_gb300 as lg
    ensure_built()
    lib = lg.load()
    sizes = [ctypes.c_int64() for _ in range(3)]
    assert lib.lobpcg_struct_sizes(*[ctypes.byref(x) for x in sizes]) == 0
    assert [x.value for x in sizes] == [ctypes.sizeof(lg.Cell), ctypes.sizeof(lg.Options),
                                        ctypes.sizeof(lg.Stats)]
    assert lib.lobpcg_struct_sizes(None, None, None) == 0
