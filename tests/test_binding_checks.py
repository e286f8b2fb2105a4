"""The Python binding rejects operands whose type, shape, layout or residency does not match what
the C entry points will read or write, before any pointer reaches the library (CPU; no GPU
needed). A valid call passes through to the library, which here sees a NULL handle and returns
LOBPCG_ERR_ARG."""
import ctypes

import numpy as np
import pytest

from tests._helpers import ensure_built


@pytest.fixture(scope="module")
def lg():
    import paper_0707_3405_gb300 as lg
    ensure_built()
    lg.load()
    return lg


@pytest.fixture
def fake_solver(lg, monkeypatch):
    """A Solver object without a device handle: one k-point of 10 plane waves."""
    s = lg.Solver.__new__(lg.Solver)
    s._lib = lg.load()
    s.handle = ctypes.c_void_p()
    s.nk, s.nproj, s.N = 1, 0, 8
    monkeypatch.setattr(s, "npw", lambda k=0: 10)
    return s


def _z(*shape, dtype=np.complex128):
    return np.zeros(shape, dtype=dtype)


def test_solve_checks_every_start_block(lg, fake_solver):
    import torch
    s = fake_solver
    with pytest.raises(ValueError):
        s.solve([_z(4, 9)])                                   # wrong plane-wave count
    with pytest.raises(ValueError):
        s.solve([_z(4, 10)], nbands=8)                        # fewer rows than bands
    with pytest.raises(TypeError):
        s.solve([_z(4, 10, dtype=np.complex64)])
    with pytest.raises(ValueError):
        s.solve([np.asfortranarray(_z(4, 10))])               # not row-major contiguous
    with pytest.raises(ValueError):
        s.solve([torch.zeros((10, 4), dtype=torch.complex128).t()])
    with pytest.raises(TypeError):
        s.solve([[0j] * 10])
    with pytest.raises(ValueError):
        s.solve([_z(4, 10), _z(4, 10)])                       # one block per k-point
    with pytest.raises(lg.LobpcgError) as e:                  # valid: reaches the library
        s.solve([_z(4, 10)])
    assert e.value.code == lg.ERR_ARG
    with pytest.raises(lg.LobpcgError):
        s.solve([torch.zeros((8, 10), dtype=torch.complex128)], nbands=4)


def test_apply_h_checks_the_output_block(lg, fake_solver):
    import torch
    s = fake_solver
    X = _z(3, 10)
    with pytest.raises(TypeError):
        s.apply_H(0, X, _z(3, 9))
    with pytest.raises(TypeError):
        s.apply_H(0, X, _z(3, 10, dtype=np.complex64))
    with pytest.raises(TypeError):
        s.apply_H(0, X, torch.zeros((3, 10), dtype=torch.complex128))
    with pytest.raises(ValueError):
        s.apply_H(0, _z(10))
    Xt = torch.zeros((3, 10), dtype=torch.complex64)
    with pytest.raises(TypeError):
        s.apply_H(0, Xt, torch.zeros((3, 10), dtype=torch.complex128))
    with pytest.raises(TypeError):
        s.apply_H(0, Xt, torch.zeros((10, 3), dtype=torch.complex64).t())
    with pytest.raises(ValueError):
        s.apply_H(0, _z(3, 9))
    with pytest.raises(lg.LobpcgError) as e:
        s.apply_H(0, X, _z(3, 10))
    assert e.value.code == lg.ERR_ARG


def test_dense_building_blocks_check_operands(lg):
    import torch
    c128, c64 = torch.complex128, torch.complex64
    z = lambda *sh, dt=c128: torch.zeros(sh, dtype=dt)
    with pytest.raises(TypeError):
        lg.gemm_cn(torch.zeros((4, 8)), torch.zeros((4, 8)))  # real operands
    with pytest.raises(TypeError):
        lg.gemm_cn(z(4, 8), z(4, 8, dt=c64))                 # mixed precisions
    with pytest.raises(ValueError):
        lg.gemm_cn(z(4, 8), z(5, 7))                          # reduction lengths differ
    with pytest.raises(ValueError):
        lg.gemm_cn(z(4, 8), z(5, 8), C=z(4, 5))               # C must be (n, m)
    with pytest.raises(ValueError):
        lg.gemm_cn(z(8, 4).t(), z(5, 8))                      # not contiguous
    with pytest.raises(TypeError):
        lg.gemm_cn(z(4, 8), z(5, 8), C=z(5, 4))               # host memory
    with pytest.raises(ValueError):
        lg.gemm_nn(z(6, 20), z(3, 5))                         # B must be (n, k)
    with pytest.raises(ValueError):
        lg.gemm_nn(z(6, 20), z(3, 6), beta=1.0, C=z(3, 19))
    with pytest.raises(ValueError):
        lg.gemm_nn(z(6, 20), z(3, 6), D=z(20, 3))
    with pytest.raises(TypeError):
        lg.gemm_nn(z(6, 20), z(3, 6), D=z(3, 20))             # host memory
    with pytest.raises(ValueError):
        lg.gram_lower(z(4, 8), z(4, 8), C=z(4, 5))
    with pytest.raises(ValueError):
        lg.gram_lower(z(4, 8), z(4, 7))
    with pytest.raises(ValueError):
        lg.rayleigh_ritz(z(4, 5), z(4, 5), 2)                 # not square
    with pytest.raises(TypeError):
        lg.rayleigh_ritz(z(4, 4), z(4, 4, dt=c64), 2)
    with pytest.raises(TypeError):
        lg.rayleigh_ritz32(z(4, 4), z(4, 4), 2)               # complex64 only
    with pytest.raises(TypeError):
        lg.rayleigh_ritz(z(4, 4), z(4, 4), 2)                 # host memory
    with pytest.raises(ValueError):
        lg.heev(z(3, 4))
    with pytest.raises(TypeError):
        lg.heev(z(4, 4, dt=c64))
