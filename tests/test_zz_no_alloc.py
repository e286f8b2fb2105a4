"""The allocation-free entry point lobpcg_apply_local_noalloc, called through
the C ABI.

It exists for callers that cannot allocate device memory while they run
(code inside another framework's memory pool or under a fixed device-memory
budget, loops that must not touch the allocator because allocation can
synchronise the device); its FFT half-box lives in a fixed file-scope device
array that every call shares.

Checks: on two calls in a row, its output equals the allocating
lobpcg_apply_H on cells without KB projectors (where H = T + V_loc exactly)
and the oracle's T + V_loc; a call on a fresh handle leaves the device's free
memory unchanged; a complex64 band just under the 32 MiB limit works, and
oversized grids, host pointers and mistyped outputs are refused.  This file is
named to be collected last."""
import numpy as np
import pytest

import synth
from tests._helpers import ensure_built, make_solver, oracle_for

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 5e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _oracle_local(H, X):
    """(T + V_loc) X with the oracle's operator, X given as (nb, npw)."""
    Xc = np.asarray(X, dtype=np.complex128).T
    return (H.T[:, None] * Xc + H.apply_local(Xc)).T


CELLS = [
    ("gamma24", lambda: synth.make_workload("gamma24")),                       # 24^3, shared-memory/register passes
    ("n72", lambda: synth.tiny_workload(a=16.0, N=72, natoms=3, kb=False,      # 72^3, two-lane register lines
                                        kpt=(0.375, -0.125, 0.125))),
]


@pytest.mark.parametrize("cell", CELLS, ids=lambda c: c[0])
@pytest.mark.parametrize("dtype,tol", [("complex128", TOL64), ("complex64", TOL32)])
def test_noalloc_matches_apply_h_and_oracle_twice(cell, dtype, tol):
    import torch
    w = cell[1]()
    assert w.nproj == 0
    dt = getattr(torch, dtype)
    with make_solver(w, block_size=4) as s:
        H = oracle_for(w, s)
        rng = np.random.default_rng(21)
        for call in range(2):                  # the shared array keeps the last call's contents
            nb = 19 if call == 0 else 6
            Xn = (rng.standard_normal((nb, s.npw())) + 1j * rng.standard_normal((nb, s.npw()))) / np.sqrt(2)
            X = torch.tensor(Xn, dtype=dt, device="cuda")
            ref = s.apply_H(0, X)
            got = torch.empty_like(X)
            s.apply_local_noalloc(0, X, got)
            torch.cuda.synchronize()
            err = (got - ref).abs().max().item() / ref.abs().max().item()
            assert err < tol, (call, err)
            ora = _oracle_local(H, X.cpu().numpy())
            g = got.cpu().numpy().astype(np.complex128)
            err_o = np.abs(g - ora).max() / np.abs(ora).max()
            assert err_o < tol, (call, err_o)


def test_noalloc_allocates_nothing_on_a_fresh_handle():
    import torch
    w = synth.make_workload("gamma24")
    rng = np.random.default_rng(3)
    with make_solver(w, block_size=16) as s:
        X = torch.tensor(rng.standard_normal((8, s.npw())) + 1j * rng.standard_normal((8, s.npw())),
                         dtype=torch.complex128, device="cuda")
        Y = torch.empty_like(X)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(2):
            s.apply_local_noalloc(0, X, Y)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)


def _big_cell():
    # 256^3 grid with a sphere of radius 24.5 (49 x-planes): one band's half-box is
    # 49 * 256^2 * 8 B = 25.7 MB in complex64 (under 32 MiB) and 51 MB in complex128 (over)
    a, N = 20.0, 256
    ecut = 0.5 * (2 * np.pi / a * 24.5) ** 2
    rng = np.random.default_rng(9)
    pos = rng.uniform(0.0, a, size=(2, 3))
    return synth.Workload("big256", a, N, ecut, np.zeros((1, 3)), pos, np.array([-2.0, -1.5]),
                          np.array([1.0, 0.9]), np.zeros(0), 4, 4, kb=False)


def test_noalloc_near_the_limit_and_refusals():
    import torch
    import paper_0707_3405_gb300 as lg
    w = _big_cell()
    with make_solver(w, block_size=4) as s:
        H = oracle_for(w, s)
        rng = np.random.default_rng(17)
        Xn = rng.standard_normal((2, s.npw())) + 1j * rng.standard_normal((2, s.npw()))
        X = torch.tensor(Xn, dtype=torch.complex64, device="cuda")
        got = torch.empty_like(X)
        s.apply_local_noalloc(0, X, got)       # one complex64 band per batch, 25.7 MB of 32 MiB
        torch.cuda.synchronize()
        ora = _oracle_local(H, X.cpu().numpy())
        err = np.abs(got.cpu().numpy().astype(np.complex128) - ora).max() / np.abs(ora).max()
        assert err < TOL32, err
        X2 = X.to(torch.complex128)
        with pytest.raises(lg.LobpcgError) as e:
            s.apply_local_noalloc(0, X2, torch.empty_like(X2))
        assert e.value.code == lg.ERR_ARG and "exceeds" in str(e.value)
        with pytest.raises(TypeError):
            s.apply_local_noalloc(0, X2, torch.empty_like(X))   # output of the wrong dtype
    w = synth.tiny_workload(a=8.0, N=16, natoms=1, kb=False)
    with make_solver(w, block_size=4) as s:
        X = np.zeros((2, s.npw()), dtype=np.complex128)
        with pytest.raises(lg.LobpcgError) as e:
            s.apply_local_noalloc(0, torch.from_numpy(X), torch.from_numpy(X.copy()))
        assert e.value.code == lg.ERR_ARG
