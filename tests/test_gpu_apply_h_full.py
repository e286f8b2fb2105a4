"""Parity of lobpcg_apply_H (H = T + V_loc + V_KB, Sec. 2.2 items iii-iv) with the
CPU FP64 oracle, element by element, on every grid edge the FP32 register
FFT passes are compiled for and at the full size of each benchmark cell:

* the 72^3 cell with 10 k-points (two k-points with different sphere sizes),
* the 120^3 Gamma cell (113081 plane waves, 432 projectors),
* the 160^3 cell at its Gamma point (267761 plane waves, 1024 projectors),
* small cells on the 48^3, 64^3 and 128^3 grids.

Each case compares complex128 (FP64), complex128 in double-FP32 arithmetic and
complex64 (FP32) applications of a ragged block of bands with the oracle's
FFT route on the same inputs.  Tolerances as in test_gpu_apply_h.py (relative
to max |H x|): 1e-12 FP64, 5e-12 double-FP32, 5e-6 FP32.
"""
import numpy as np
import pytest

import synth
from tests._helpers import ensure_built, make_solver, oracle_for

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c128_df32": 5e-12, "c64": 5e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _rand_block(seed, nb, npw):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((nb, npw)) + 1j * rng.standard_normal((nb, npw))) / np.sqrt(2)


def _check(s, H, k, X, prec):
    import torch
    dt = np.complex64 if prec == "c64" else np.complex128
    Xt = torch.tensor(X.astype(dt), device="cuda")
    Y = s.apply_H(k, Xt, df32=prec == "c128_df32")
    torch.cuda.synchronize()
    got = Y.cpu().numpy().astype(np.complex128)
    ref = H.apply(X.astype(dt).astype(np.complex128).T).T
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < TOL[prec], (prec, err)
    return err


@pytest.fixture(scope="module")
def mp72():
    w = synth.make_workload("mp72x10")
    s = make_solver(w, block_size=64)
    yield w, s
    s.close()


@pytest.mark.parametrize("k", [0, 1])
@pytest.mark.parametrize("prec", ["c128", "c128_df32", "c64"])
def test_apply_h_mp72x10(mp72, k, prec):
    w, s = mp72
    assert s.npw(0) != s.npw(1)               # uneven spheres
    H = oracle_for(w, s, k)
    _check(s, H, k, _rand_block(70 + k, 9, s.npw(k)), prec)


@pytest.fixture(scope="module")
def g120():
    w = synth.make_workload("gamma120")
    s = make_solver(w, block_size=128)
    H = oracle_for(w, s)
    yield w, s, H
    s.close()


@pytest.mark.parametrize("prec", ["c128", "c128_df32", "c64"])
def test_apply_h_gamma120(g120, prec):
    w, s, H = g120
    assert s.npw() == 113081
    _check(s, H, 0, _rand_block(120, 8, s.npw()), prec)


@pytest.fixture(scope="module")
def l160():
    w = synth.make_workload("large160")
    w.kpts = w.kpts[:1]                       # the Gamma point (267761 plane waves)
    s = make_solver(w, block_size=256)
    H = oracle_for(w, s)
    yield w, s, H
    s.close()


@pytest.mark.parametrize("prec", ["c128", "c128_df32", "c64"])
def test_apply_h_large160_gamma(l160, prec):
    w, s, H = l160
    assert s.npw() == 267761 and w.nproj == 1024
    _check(s, H, 0, _rand_block(160, 4, s.npw()), prec)


@pytest.mark.parametrize("N,a,kpt", [(48, 14.0, (0.25, -0.125, 0.0)), (64, 16.0, (0.0, 0.0, 0.0)),
                                     (128, 26.0, (0.125, 0.375, -0.25))])
@pytest.mark.parametrize("prec", ["c128", "c128_df32", "c64"])
def test_apply_h_other_register_grids(N, a, kpt, prec):
    w = synth.tiny_workload(a=a, N=N, natoms=3, kb=True, kpt=kpt, seed=N)
    with make_solver(w, block_size=4) as s:
        H = oracle_for(w, s)
        _check(s, H, 0, _rand_block(N, 5, s.npw()), prec)
