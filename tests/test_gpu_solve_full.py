"""Full-size solves of the benchmark cells against the oracle's golden eigenvalues
(tests/golden, written by tests/golden/make_golden.py from the oracle's LOBPCG and
confirmed by its Lanczos route), every returned band re-checked with the oracle's H.

Targets (Algorithm 1, Sec. 3.2): every requested eigenvalue within 1e-9 Ha of the
oracle's, every residual ||H x - eps x|| <= 1e-8 Ha recomputed by the oracle on the
returned vectors, the library's own residuals equal to that recomputation, and the
returned block orthonormal.
"""
import os

import numpy as np
import pytest

import synth
from oracle import checks
from tests._helpers import ensure_built, make_solver, oracle_for

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _start(w, s, k=0, M=None, kglobal=None):
    import torch
    return torch.tensor(w.x0(s.npw(k), k if kglobal is None else kglobal, M).T.copy(), device="cuda")


def _check_all(w, s, k, X, eig, resid, ref, orth):
    H = oracle_for(w, s, k)
    M = X.shape[0]
    d = np.abs(eig - ref[:M]).max()
    assert d < 1e-9, d
    Xn = X.cpu().numpy().T
    r = checks.residuals(H, Xn, eig)
    assert r.max() <= 1e-8, r.max()
    assert np.abs(resid - r).max() < 1e-9
    assert checks.orthonormality_error(Xn) < orth
    return d, r.max()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_solve_k96_all_bands_vs_oracle(precision):
    """The 96^3 cell: 256 bands in blocks of 64 plus 64 buffer bands, k = (1/4,1/4,1/4)."""
    w = synth.make_workload("k96")
    ref = np.loadtxt(os.path.join(GOLDEN, "k96_eig.txt"))
    with make_solver(w, block_size=64, nline=4, max_sweeps=40, precision=precision, tol=1e-8, nbuf=64) as s:
        X = _start(w, s)
        res = s.solve([X])
        assert res.status == 0, res.stats
        _check_all(w, s, 0, X, res.eig[0], res.resid[0], ref, 1e-12 if precision == "fp64" else 1e-10)


def test_solve_mp72x10_all_kpoints_vs_oracle():
    """The 10-k-point 72^3 cell in one call (concurrent k-point lanes), mixed schedule: every
    k-point's 128 eigenvalues match its golden and meet 1e-8 with the oracle's H."""
    w = synth.make_workload("mp72x10")
    refs = {k: np.loadtxt(os.path.join(GOLDEN, f"mp72x10_k{k}_eig.txt")) for k in range(w.nk)}
    with make_solver(w, block_size=64, nline=4, max_sweeps=40, precision="mixed", tol=1e-8, nbuf=64) as s:
        Xs = [_start(w, s, k) for k in range(w.nk)]
        res = s.solve(Xs)
        assert res.status == 0, res.stats
        for k in range(w.nk):
            H = oracle_for(w, s, k)
            Xn = Xs[k].cpu().numpy().T
            r = checks.residuals(H, Xn, res.eig[k])
            assert r.max() <= 1e-8, (k, r.max())
            assert checks.orthonormality_error(Xn) < 1e-10
            assert np.abs(res.eig[k] - refs[k]).max() < 1e-9, (k, np.abs(res.eig[k] - refs[k]).max())


@pytest.mark.parametrize("real", [False, True])
def test_solve_gamma120_all_bands_vs_oracle(real):
    """The 120^3 Gamma cell the mixed-vs-FP64 comparison is made on: 1024 bands in blocks of
    128 plus 128 buffer bands, mixed schedule, complex orbitals and the real-orbital form."""
    w = synth.make_workload("gamma120")
    ref = np.loadtxt(os.path.join(GOLDEN, "gamma120_eig.txt"))
    with make_solver(w, block_size=128, nline=4, max_sweeps=30, precision="mixed", tol=1e-8, nbuf=128,
                     gamma_real=real) as s:
        X = _start(w, s)
        res = s.solve([X])
        assert res.status == 0, res.stats
        _check_all(w, s, 0, X, res.eig[0], res.resid[0], ref, 1e-10)
