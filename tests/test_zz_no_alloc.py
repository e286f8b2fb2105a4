"""The allocation-free entry point lobpcg_apply_local_noalloc, called through
the C ABI, against the allocating lobpcg_apply_H on a cell without KB
projectors (where H = T + V_loc exactly), on two calls in a row.

It exists for callers that cannot allocate device memory while they run; its
FFT half-box lives in a fixed file-scope device array.  This file is named to
be collected last."""
import numpy as np
import pytest

import synth
from tests._helpers import ensure_built, make_solver

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 5e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.mark.parametrize("dtype,tol", [("complex128", TOL64), ("complex64", TOL32)])
def test_noalloc_matches_apply_h_twice(dtype, tol):
    import torch
    w = synth.make_workload("gamma24")          # 24^3 grid, 925 plane waves, no projectors
    dt = getattr(torch, dtype)
    with make_solver(w, block_size=16) as s:
        rng = np.random.default_rng(21)
        for call in range(2):                  # the shared array keeps the last call's contents
            X = torch.tensor(rng.standard_normal((19, s.npw())) + 1j * rng.standard_normal((19, s.npw())),
                             dtype=dt, device="cuda")
            ref = s.apply_H(0, X)
            got = torch.empty_like(X)
            s.apply_local_noalloc(0, X, got)
            torch.cuda.synchronize()
            err = (got - ref).abs().max().item() / ref.abs().max().item()
            assert err < tol, (call, err)


def test_noalloc_rejects_oversized_grid_and_host_pointers():
    import torch
    import paper_0707_3405_gb300 as lg
    w = synth.tiny_workload(a=8.0, N=16, natoms=1, kb=False)
    with make_solver(w, block_size=4) as s:
        X = np.zeros((2, s.npw()), dtype=np.complex128)
        with pytest.raises(lg.LobpcgError) as e:
            s.apply_local_noalloc(0, torch.from_numpy(X), torch.from_numpy(X.copy()))
        assert e.value.code == lg.ERR_ARG
    # 256^3 grid with a sphere of radius 24.5 (49 x-planes): one complex128 band's
    # half-box is 49 * 256^2 * 16 B = 51 MB > 32 MiB
    a, N = 20.0, 256
    ecut = 0.5 * (2 * np.pi / a * 24.5) ** 2
    with make_solver(synth.Workload("big", a, N, ecut, np.zeros((1, 3)),
                                    np.zeros((1, 3)), np.array([-1.0]), np.array([1.0]), np.zeros(0), 4, 4,
                                    kb=False, _vloc=np.zeros((N, N, N))), block_size=4) as s:
        X = torch.zeros((1, s.npw()), dtype=torch.complex128, device="cuda")
        with pytest.raises(lg.LobpcgError) as e:
            s.apply_local_noalloc(0, X, torch.empty_like(X))
        assert e.value.code == lg.ERR_ARG and "exceeds" in str(e.value)
