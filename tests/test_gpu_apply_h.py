"""Parity of lobpcg_apply_H (H = T + V_loc + V_KB, Sec. 2.2 items iii-iv) with the
CPU FP64 oracle, element by element, on seeded synthetic cells.

Tolerances (relative to max |H x|):
  complex128 / FP64 FFT and GEMMs  1e-12
  complex128 / double-FP32         5e-12  (~2^-47 per operation, same growth)
  complex64  / FP32 FFT and GEMMs  5e-6   (FP32 unit roundoff 6e-8 times the
                                         ~log2(N^3) + nproj-term growth)
"""
import numpy as np
import pytest

import synth
from tests._helpers import ensure_built, make_solver, oracle_for

pytestmark = pytest.mark.gpu

TOL64, TOL32, TOLDF = 1e-12, 5e-6, 5e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _rand_block(seed, nb, npw):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nb, npw)) + 1j * rng.standard_normal((nb, npw))) / np.sqrt(2)


def _compare(solver, H, k, X, dtype, tol, df32=False):
    torch = _torch()
    Xt = torch.tensor(X.astype(dtype), device="cuda")
    Yt = solver.apply_H(k, Xt, df32=df32)
    torch.cuda.synchronize()
    Y = Yt.cpu().numpy().astype(np.complex128)
    ref = H.apply(X.astype(dtype).astype(np.complex128).T).T
    err = np.abs(Y - ref).max() / np.abs(ref).max()
    assert err < tol, err
    return err


CASES = [
    dict(a=5.0, N=8, natoms=1, kb=False, kpt=(0.0, 0.0, 0.0)),
    dict(a=6.0, N=12, natoms=2, kb=True, kpt=(0.0, 0.0, 0.0)),
    dict(a=6.0, N=12, natoms=2, kb=True, kpt=(0.25, 0.125, -0.375)),
    dict(a=7.0, N=16, natoms=3, kb=True, kpt=(0.5, 0.0, -0.5)),
    dict(a=9.0, N=20, natoms=2, kb=True, kpt=(0.1, 0.2, 0.3)),
    dict(a=10.0, N=24, natoms=4, kb=False, kpt=(0.0, 0.0, 0.0)),
    dict(a=11.0, N=30, natoms=2, kb=True, kpt=(-0.25, 0.25, 0.0)),
    dict(a=12.0, N=36, natoms=2, kb=True, kpt=(0.375, 0.0, 0.125)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c['N']}_kb{int(c['kb'])}_k{c['kpt'][0]}")
@pytest.mark.parametrize("prec", ["c128", "c64", "c128_df32"])
def test_apply_h_matches_oracle_small(case, prec):
    w = synth.tiny_workload(**case)
    with make_solver(w, block_size=4) as s:
        H = oracle_for(w, s)
        # 37 bands: several FFT band batches would be needed only for big grids;
        # an odd count exercises ragged GEMM tiles
        X = _rand_block(1, 37, s.npw())
        if prec == "c128":
            _compare(s, H, 0, X, np.complex128, TOL64)
        elif prec == "c128_df32":
            _compare(s, H, 0, X, np.complex128, TOLDF, df32=True)
        else:
            _compare(s, H, 0, X, np.complex64, TOL32)


def test_apply_h_dense_definition_tiny():
    """On a tiny cell compare with the explicitly assembled H (direct DFT, no FFT)."""
    w = synth.tiny_workload(a=5.0, N=8, natoms=2, kb=True, kpt=(0.25, -0.25, 0.125))
    torch = _torch()
    with make_solver(w, block_size=4) as s:
        H = oracle_for(w, s)
        Hd = H.dense()
        X = _rand_block(2, 5, s.npw())
        Y = s.apply_H(0, torch.tensor(X, device="cuda")).cpu().numpy()
        ref = (Hd @ X.T).T
        assert np.abs(Y - ref).max() / np.abs(ref).max() < TOL64


def test_apply_h_host_pointers_and_edge_cases():
    import paper_0707_3405_gb300 as lg
    torch = _torch()
    w = synth.tiny_workload(a=6.0, N=12, natoms=2, kb=True, kpt=(0.25, 0.0, 0.0))
    with make_solver(w, block_size=4) as s:
        H = oracle_for(w, s)
        X = _rand_block(3, 3, s.npw())
        Yh = s.apply_H(0, X)                              # numpy in/out (staged)
        Yd = s.apply_H(0, torch.tensor(X, device="cuda")).cpu().numpy()
        assert np.array_equal(Yh, Yd)
        ref = H.apply(X.T).T
        assert np.abs(Yh - ref).max() / np.abs(ref).max() < TOL64
        # nb = 0 is a no-op; nb = 1 works
        s.apply_H(0, np.zeros((0, s.npw()), dtype=np.complex128))
        Y1 = s.apply_H(0, X[:1].copy())
        assert np.abs(Y1 - ref[:1]).max() / np.abs(ref).max() < TOL64
        with pytest.raises(lg.LobpcgError) as e:
            s.apply_H(1, X)
        assert e.value.code == lg.ERR_ARG
        Xt = torch.tensor(X, device="cuda")
        with pytest.raises(lg.LobpcgError) as e:
            s.apply_H(0, Xt, Xt)                          # overlapping in/out
        assert e.value.code == lg.ERR_ARG


def test_apply_h_translation_invariance_gpu():
    """A uniform shift of the potential shifts H x by c x exactly (to rounding)."""
    torch = _torch()
    w = synth.tiny_workload(a=6.0, N=12, natoms=2, kb=True)
    w2 = synth.tiny_workload(a=6.0, N=12, natoms=2, kb=True)
    w2._vloc = w.vloc() + 0.5
    with make_solver(w, block_size=4) as s1, make_solver(w2, block_size=4) as s2:
        X = torch.tensor(_rand_block(4, 6, s1.npw()), device="cuda")
        d = (s2.apply_H(0, X) - s1.apply_H(0, X) - 0.5 * X).abs().max().item()
        assert d < 1e-12


@pytest.mark.parametrize("prec", ["c128", "c64", "c128_df32"])
def test_apply_h_full_size_k96(prec):
    """The 96^3 / 57925 plane-wave cell with 256 KB projectors, k = (1/4,1/4,1/4):
    a ragged block of 19 bands against the oracle's FFT route."""
    w = synth.make_workload("k96")
    with make_solver(w, block_size=64) as s:
        assert s.npw() == 57925
        H = oracle_for(w, s)
        X = _rand_block(5, 19, s.npw())
        _compare(s, H, 0, X, np.complex64 if prec == "c64" else np.complex128,
                 {"c128": TOL64, "c64": TOL32, "c128_df32": TOLDF}[prec], df32=prec == "c128_df32")


def test_apply_h_multi_kpoint_uneven_spheres():
    """Several k-points with different sphere sizes in one handle."""
    torch = _torch()
    w = synth.tiny_workload(a=8.0, N=16, natoms=2, kb=True)
    w.kpts = np.array([[0.0, 0.0, 0.0], [0.375, -0.125, 0.25], [-0.375, 0.375, 0.125]])
    with make_solver(w, block_size=4) as s:
        sizes = [s.npw(k) for k in range(3)]
        assert len(set(sizes)) > 1
        for k in range(3):
            H = oracle_for(w, s, k)
            X = _rand_block(10 + k, 7, s.npw(k))
            Y = s.apply_H(k, torch.tensor(X, device="cuda")).cpu().numpy()
            ref = H.apply(X.T).T
            assert np.abs(Y - ref).max() / np.abs(ref).max() < TOL64
