"""The electron density rho(r) = sum_b f_b |psi_b(r)|^2 (Sec. 2.1, first step of the SC
loop; by the inverse FFT, Sec. 2.2 item iii) through lobpcg_density, against the oracle's
density (oracle/density.py, itself pinned by the plain sum, Parseval and plane-wave closed
forms), element by element on the N^3 grid.

Tolerances, relative to max rho: 1e-12 for FP64 and double-FP32 transforms, 2e-6 for the
FP32 register transforms (FP32 sums over each band batch).
"""
import numpy as np
import pytest

import synth
from oracle import density as odens
from tests._helpers import ensure_built, make_solver

pytestmark = pytest.mark.gpu
TOL = {"c128": 1e-12, "c128_df32": 1e-12, "c64": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _bands(seed, nb, npw):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((npw, nb)) + 1j * rng.standard_normal((npw, nb))
    Q, _ = np.linalg.qr(X)                       # orthonormal bands
    return Q


def _run(s, w, k, Q, f, prec):
    import torch
    dt = torch.complex64 if prec == "c64" else torch.complex128
    X = torch.tensor(np.ascontiguousarray(Q.T), dtype=dt, device="cuda")
    rho = s.density(k, X, f, df32=prec == "c128_df32")
    torch.cuda.synchronize()
    return rho.cpu().numpy()


CASES = [
    dict(a=6.0, N=12, kpt=(0.25, 0.125, -0.375)),         # register grid
    dict(a=9.0, N=20, kpt=(0.0, 0.0, 0.0)),                # register grid, Gamma
    dict(a=10.0, N=30, kpt=(0.1, -0.2, 0.3)),              # shared-memory passes only (30 = 2 3 5)
    dict(a=16.0, N=72, kpt=(0.375, -0.125, 0.125)),        # two-lane register lines
    dict(a=20.0, N=96, kpt=(0.25, 0.25, 0.25)),            # four-lane register lines
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"N{c['N']}")
@pytest.mark.parametrize("prec", ["c128", "c128_df32", "c64"])
def test_density_matches_oracle(case, prec):
    w = synth.tiny_workload(natoms=2, kb=False, **case)
    with make_solver(w, block_size=4) as s:
        mil = s.gvectors(0)
        nb = 13
        Q = _bands(case["N"], nb, s.npw())
        f = np.linspace(2.0, 0.5, nb)
        got = _run(s, w, 0, Q, f, prec)
        Qd = Q.astype(np.complex64).astype(np.complex128) if prec == "c64" else Q
        ref = odens.density(w.a, w.N, mil, Qd, f)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < TOL[prec], err
        # Parseval on the grid: the density integrates to the occupations
        assert odens.electron_count(w.a, got) == pytest.approx(f.sum(), rel=1e-12 if prec != "c64" else 1e-6)


def test_density_accumulates_over_calls_and_kpoints():
    """rho is accumulated: two calls with halves of the bands equal one call with all of
    them, and a second k-point adds its own bands' density."""
    import torch
    w = synth.tiny_workload(a=8.0, N=16, natoms=2, kb=False)
    w.kpts = np.array([[0.0, 0.0, 0.0], [0.25, -0.125, 0.375]])
    with make_solver(w, block_size=4) as s:
        Q0 = _bands(1, 10, s.npw(0))
        Q1 = _bands(2, 6, s.npw(1))
        f0, f1 = np.full(10, 2.0), np.full(6, 0.5)
        X0 = torch.tensor(np.ascontiguousarray(Q0.T), device="cuda")
        X1 = torch.tensor(np.ascontiguousarray(Q1.T), device="cuda")
        full = s.density(0, X0, f0).cpu().numpy()
        rho = s.density(0, X0[:4].contiguous(), f0[:4])
        s.density(0, X0[4:].contiguous(), f0[4:], rho=rho)
        assert np.abs(rho.cpu().numpy() - full).max() < 1e-13 * np.abs(full).max()
        s.density(1, X1, f1, rho=rho)
        ref = odens.density(w.a, w.N, s.gvectors(0), Q0, f0) + odens.density(w.a, w.N, s.gvectors(1), Q1, f1)
        assert np.abs(rho.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()
        # bitwise reproducible
        again = s.density(0, X0, f0).cpu().numpy()
        assert np.array_equal(again, full)


def test_density_of_the_k96_eigenvectors_vs_oracle():
    """Full size: the density of the 256 lowest bands of the 96^3 cell (57925 plane waves),
    each doubly occupied, from the library's FP64 solve, against the oracle's density of the
    same vectors; the electron count is 512."""
    import torch
    w = synth.make_workload("k96")
    with make_solver(w, block_size=64, nline=4, max_sweeps=40, precision="mixed", tol=1e-8, nbuf=64) as s:
        X = torch.tensor(w.x0(s.npw(), 0).T.copy(), device="cuda")
        res = s.solve([X])
        assert res.status == 0
        f = np.full(w.nbands, 2.0)
        got = s.density(0, X, f, df32=True).cpu().numpy()
        ref = odens.density(w.a, w.N, s.gvectors(0), X.cpu().numpy().T, f)
        assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12
        assert odens.electron_count(w.a, got) == pytest.approx(512.0, rel=1e-10)


def test_density_argument_errors():
    import torch
    import paper_0707_3405_gb300 as lg
    w = synth.tiny_workload(a=6.0, N=12, natoms=1, kb=False)
    with make_solver(w, block_size=4) as s:
        X = torch.zeros((2, s.npw()), dtype=torch.complex128, device="cuda")
        with pytest.raises(lg.LobpcgError) as e:
            s.density(1, X, [1.0, 1.0])
        assert e.value.code == lg.ERR_ARG
        with pytest.raises(lg.LobpcgError) as e:
            s.density(0, X, [1.0, float("nan")])
        assert e.value.code == lg.ERR_ARG
        with pytest.raises(lg.LobpcgError) as e:
            s.density(0, X.cpu(), [1.0, 1.0], rho=torch.zeros((12, 12, 12), dtype=torch.float64, device="cuda"))
        assert e.value.code == lg.ERR_ARG
