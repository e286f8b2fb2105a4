"""The bounded-wait path of the tensor-core GEMMs, driven without hanging or
faulting the GPU: the poll limit of their ring waits is set to zero, so the
first wait for a stage's MMAs gives up at once.  The CTA then stops issuing,
waits with the full limit for the MMAs it already issued, frees its tensor
memory and returns with the device flag set; the host sees LOBPCG_ERR_TIMEOUT
from lobpcg_k_check_timeouts and from a solve (which checks the flag after
every sweep).  After the limit is restored the same calls succeed."""
import numpy as np
import pytest

import synth
from tests._helpers import ensure_built, make_solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


@pytest.fixture()
def zero_spin():
    import paper_0707_3405_gb300 as lg
    lg.set_spin_limit(0)
    try:
        yield
    finally:
        lg.set_spin_limit(-1)
        try:
            lg.check_timeouts()       # clear a flag left by a failed test
        except lg.LobpcgError:
            pass


def test_gemm_wait_runs_out_and_returns(zero_spin):
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(4)
    K, m, n = 8192, 64, 64          # 512 stages of 16: every CTA refills its ring
    A = torch.tensor(rng.standard_normal((m, K)) + 1j * rng.standard_normal((m, K)), dtype=torch.complex64,
                     device="cuda")
    B = torch.tensor(rng.standard_normal((n, K)) + 1j * rng.standard_normal((n, K)), dtype=torch.complex64,
                     device="cuda")
    lg.set_gemm_mode(2)
    lg.gemm_cn(A, B)                 # returns: the kernel gave up instead of waiting
    with pytest.raises(lg.LobpcgError) as e:
        lg.check_timeouts()
    assert e.value.code == lg.ERR_TIMEOUT
    lg.check_timeouts()              # the flag was read and cleared
    lg.set_spin_limit(-1)
    C = lg.gemm_cn(A, B)
    lg.check_timeouts()
    ref = A.cpu().numpy().astype(np.complex128).conj() @ B.cpu().numpy().astype(np.complex128).T
    got = C.cpu().numpy().T
    scale = np.abs(A.cpu().numpy()).astype(np.float64) @ np.abs(B.cpu().numpy()).astype(np.float64).T
    assert (np.abs(got - ref) / scale).max() < 2e-6


def test_solve_reports_timeout(zero_spin):
    import torch
    import paper_0707_3405_gb300 as lg
    # about 17k plane waves: the mixed schedule's Grams run on the tensor cores with K splits of
    # more stages than the ring holds, so their CTAs wait to refill it
    w = synth.tiny_workload(a=16.0, N=64, natoms=2, kb=True, nbands=8, block=4)
    with make_solver(w, block_size=4, precision="mixed", max_sweeps=3) as s:
        X = torch.tensor(w.x0(s.npw(), 0, 8).T.copy(), device="cuda")
        with pytest.raises(lg.LobpcgError) as e:
            s.solve([X.clone()])
        assert e.value.code == lg.ERR_TIMEOUT
        lg.set_spin_limit(-1)
        r = s.solve([X.clone()])
        assert r.status in (lg.OK, lg.NOT_CONVERGED)
