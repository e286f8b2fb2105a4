"""FP64-class complex128 GEMMs on the tensor cores (exact 8-bit BF16 digit slices,
exact FP32 accumulation per 64 terms, double-FP32 sums; LOBPCG_C128_TC) against FP64
numpy, on odd shapes and at the solve's shapes.

Bound: 2e-12 relative to sum |a||b| per entry, the bound the double-FP32 engine is
held to.  The digit scheme's own bound is about 2^-44 of sum |a||b| (slices of 48
bits per 64-term chunk scale, level sums exact); the extreme-digit cases check that
no level accumulator exceeds FP32's exact integer range.
"""
import numpy as np
import pytest

from tests._helpers import ensure_built

pytestmark = pytest.mark.gpu
TOL = 2e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _dev(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("m,n,K", [(1, 1, 1), (16, 16, 925), (64, 37, 5000), (192, 192, 57925), (432, 19, 3001),
                                   (7, 130, 100), (320, 128, 113081), (129, 65, 64), (33, 200, 129)])
def test_oz_gemm_cn(m, n, K):
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(m * 13 + n + K)
    A, B, C0 = _c(rng, K, m), _c(rng, K, n), _c(rng, m, n)
    Ct = _dev(C0.T)
    lg.gemm_cn(_dev(A.T), _dev(B.T), alpha=0.5, beta=-2.0, C=Ct, tc=True)
    lg.check_timeouts()
    got = Ct.cpu().numpy().T
    ref = 0.5 * A.conj().T @ B - 2.0 * C0
    scale = 0.5 * np.abs(A).T @ np.abs(B) + 2.0 * np.abs(C0)
    assert (np.abs(got - ref) / scale).max() < TOL


@pytest.mark.parametrize("n,K", [(1, 1), (64, 925), (65, 5000), (200, 57925), (320, 3001), (33, 100),
                                 (1152, 8192)])
def test_oz_gram_lower(n, K):
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(n * 3 + K)
    A, B = _c(rng, K, n), _c(rng, K, n)
    Ct = _dev(np.zeros((n, n), dtype=np.complex128))
    lg.gram_lower(_dev(A.T), _dev(B.T), C=Ct, tc=True)
    lg.check_timeouts()
    got = Ct.cpu().numpy().T
    ref = A.conj().T @ B
    scale = np.abs(A).T @ np.abs(B)
    il = np.tril_indices(n)
    assert (np.abs(got - ref)[il] / scale[il]).max() < TOL


@pytest.mark.parametrize("M,n,k", [(57925, 320, 320), (1000, 64, 5), (130, 7, 100), (113081, 128, 384),
                                   (64, 1, 1), (4097, 130, 1152)])
@pytest.mark.parametrize("beta", [0.0, -0.5])
def test_oz_gemm_nn(M, n, k, beta):
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(M + 7 * n + k)
    A, B, C0 = _c(rng, M, k), _c(rng, k, n), _c(rng, M, n)
    Dt = lg.gemm_nn(_dev(A.T), _dev(B.T), alpha=1.5, beta=beta, C=_dev(C0.T) if beta else None, tc=True)
    lg.check_timeouts()
    got = Dt.cpu().numpy().T
    ref = 1.5 * A @ B + beta * C0
    scale = 1.5 * np.abs(A) @ np.abs(B) + abs(beta) * np.abs(C0)
    assert (np.abs(got - ref) / scale).max() < TOL


def test_oz_in_place_accumulate():
    """D = C - A B with D and C the same buffer (the constraint update X <- X - Y G)."""
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(5)
    M, n, k = 20000, 64, 256
    A, B, X0 = _c(rng, M, k), _c(rng, k, n), _c(rng, M, n)
    Xt = _dev(X0.T)
    lg.gemm_nn(_dev(A.T), _dev(B.T), alpha=-1.0, beta=1.0, C=Xt, D=Xt, tc=True)
    got = Xt.cpu().numpy().T
    ref = X0 - A @ B
    scale = np.abs(A) @ np.abs(B) + np.abs(X0)
    assert (np.abs(got - ref) / scale).max() < TOL


@pytest.mark.parametrize("val", [0.999, -0.999, 1.0, 3.0e-7])
def test_oz_extreme_digits_are_exact(val):
    """Constant operands whose leading digit is the largest allowed (|d_1| = 256 for
    0.999): every level sum sits at the top of FP32's exact integer range; the result
    must still be the exact product to the scheme's precision."""
    import paper_0707_3405_gb300 as lg
    K, m, n = 4096, 128, 64
    A = np.full((K, m), val * (1 + 1j))
    B = np.full((K, n), val * (1 - 1j))
    C = lg.gemm_cn(_dev(A.T), _dev(B.T), tc=True).cpu().numpy().T
    ref = A.conj().T @ B
    assert (np.abs(C - ref) / (np.abs(A).T @ np.abs(B))).max() < TOL
    D = lg.gemm_nn(_dev(np.full((K, m), val).T + 0j), _dev(np.full((m, n), -val).T + 0j), tc=True).cpu().numpy().T
    refd = np.full((K, n), -val * val * m)
    assert np.abs(D - refd).max() / (val * val * m) < TOL


def test_oz_matches_double_fp32_engine_on_grams():
    """The two FP64-class engines agree on a Gram of nearly orthonormal vectors (entries
    from 1 down to ~1e-12), well inside either one's bound."""
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(_c(rng, 20000, 96))
    X = Q + 1e-9 * _c(rng, 20000, 96)
    Xt = _dev(X.T)
    Gt = lg.gram_lower(Xt, Xt, tc=True).cpu().numpy().T
    Gd = lg.gram_lower(Xt, Xt, df32=True).cpu().numpy().T
    ref = X.conj().T @ X
    il = np.tril_indices(96)
    assert np.abs(Gt - ref)[il].max() < 1e-13
    assert np.abs(Gt - Gd)[il].max() < 1e-13
