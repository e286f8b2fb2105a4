"""The Gamma-point real-orbital form of lobpcg_solve (options.gamma_real): packed half-sphere
storage, real coefficient matrices, H applied to two real bands at once.  Against the oracle
(oracle/gamma.py states the real form; its spectrum is the complex one): golden and dense
eigenvalues within 1e-9 Ha, every returned band real-form (c(-G) = conj(c(G))), orthonormal,
and with residual <= 1e-8 Ha recomputed by the oracle's H."""
import os

import numpy as np
import pytest

import synth
from oracle import checks, gamma as ogamma
from tests._helpers import ensure_built, make_solver, oracle_for

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _start(w, s, M, k=0):
    import torch
    return torch.tensor(w.x0(s.npw(k), k, M).T.copy(), device="cuda")


def _check_real_form(s, X, k=0):
    mil = s.gvectors(k)
    zero, plus, minus = ogamma.half_set(mil)
    Xn = X.cpu().numpy().T
    sym = np.abs(Xn[minus] - Xn[plus].conj()).max()
    assert sym < 1e-13, sym
    assert np.abs(Xn[zero].imag).max() < 1e-13
    return Xn


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gamma_real_gamma24_golden(precision):
    w = synth.make_workload("gamma24")
    ref = np.loadtxt(os.path.join(GOLDEN, "gamma24_eig.txt"))
    with make_solver(w, block_size=16, nline=4, max_sweeps=60, precision=precision, tol=1e-8, nbuf=16,
                     gamma_real=True) as s:
        X = _start(w, s, 16)
        res = s.solve([X])
        assert res.status == 0, res.stats
        assert np.abs(res.eig[0] - ref).max() < 1e-9, np.abs(res.eig[0] - ref).max()
        Xn = _check_real_form(s, X)
        H = oracle_for(w, s)
        r = checks.residuals(H, Xn, res.eig[0])
        assert r.max() <= 1e-8, r.max()
        assert np.abs(res.resid[0] - r).max() < 1e-9
        assert checks.orthonormality_error(Xn) < (1e-12 if precision == "fp64" else 1e-10)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gamma_real_with_projectors_vs_dense(precision):
    """A Gamma cell with KB projectors (s and p: real in r space up to a sign), several
    blocks and an odd block size (the last pair of an H application has one band)."""
    w = synth.tiny_workload(a=10.0, N=24, natoms=3, kb=True, ecut=0.5 * (2 * np.pi / 10.0 * 7.2) ** 2)
    with make_solver(w, block_size=5, nline=4, max_sweeps=100, precision=precision, tol=1e-8, nbuf=5,
                     gamma_real=True) as s:
        H = oracle_for(w, s)
        exact = np.linalg.eigvalsh(H.dense())[:15]
        X = _start(w, s, 15)
        res = s.solve([X])
        assert res.status == 0, res.stats
        assert np.abs(res.eig[0] - exact).max() < 1e-9
        Xn = _check_real_form(s, X)
        assert checks.residuals(H, Xn, res.eig[0]).max() <= 1e-8


def test_gamma_real_only_at_gamma():
    """In a handle with Gamma and a general k-point, only the Gamma point takes the real form;
    both match dense diagonalisation."""
    import dataclasses
    base = synth.tiny_workload(a=6.0, N=12, natoms=2, kb=True)
    w = dataclasses.replace(base, kpts=np.array([[0.0, 0.0, 0.0], [0.25, 0.125, -0.375]]))
    with make_solver(w, block_size=4, nline=4, max_sweeps=100, tol=1e-8, nbuf=4, gamma_real=True) as s:
        Xs = [_start(w, s, 8, k) for k in range(2)]
        res = s.solve(Xs)
        assert res.status == 0
        for k in range(2):
            H = oracle_for(w, s, k)
            exact = np.linalg.eigvalsh(H.dense())[:8]
            assert np.abs(res.eig[k] - exact).max() < 1e-9
        _check_real_form(s, Xs[0], 0)


def test_gamma_real_gamma120_matches_complex_solve():
    """The 120^3 Gamma cell, mixed schedule, real form against the complex-orbital solve of
    the same cell: the same 1024 eigenvalues within 1e-9 Ha; sampled residuals re-checked by
    the oracle's H."""
    import torch
    w = synth.make_workload("gamma120")
    kw = dict(block_size=128, nline=4, max_sweeps=30, precision="mixed", tol=1e-8, nbuf=128)
    with make_solver(w, gamma_real=True, **kw) as s:
        X = _start(w, s, 1024)
        res = s.solve([X])
        assert res.status == 0, res.stats
        s.set_options(gamma_real=False, **kw)
        Xc = _start(w, s, 1024)
        rc = s.solve([Xc])
        assert rc.status == 0
        assert np.abs(res.eig[0] - rc.eig[0]).max() < 1e-9
        Xn = _check_real_form(s, X)
        H = oracle_for(w, s)
        pick = np.array([0, 1, 127, 128, 511, 700, 1022, 1023])
        r = checks.residuals(H, Xn[:, pick], res.eig[0][pick])
        assert r.max() <= 1e-8, r.max()
        G = (X.conj() @ X.T).cpu().numpy()
        assert np.abs(G - np.eye(1024)).max() < 1e-10
