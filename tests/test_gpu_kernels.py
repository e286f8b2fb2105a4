"""Parity of the dense building blocks (GEMMs, FP64 Rayleigh-Ritz, Hermitian
eigensolver) with FP64 numpy/scipy on odd shapes.

Tolerances: FP64 GEMMs 1e-13 relative to sum |a||b|; FP32 GEMMs 1e-5 relative;
eigenvalues 1e-12 relative to ||A||; eigenvector residuals 1e-11 ||A||;
orthonormality 1e-12.
"""
import numpy as np
import pytest
import scipy.linalg

from tests._helpers import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("m,n,K", [(1, 1, 1), (16, 16, 925), (64, 37, 5000), (192, 192, 57925), (432, 19, 3001),
                                   (7, 130, 100)])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_gemm_cn(m, n, K, prec):
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(m * 7 + n)
    A, B, C0 = _c(rng, K, m), _c(rng, K, n), _c(rng, m, n)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    At = torch.tensor(A.T.copy(), dtype=dt, device="cuda")
    Bt = torch.tensor(B.T.copy(), dtype=dt, device="cuda")
    Ct = torch.tensor(C0.T.copy(), dtype=dt, device="cuda")
    lg.gemm_cn(At, Bt, alpha=0.5, beta=-2.0, C=Ct)
    got = Ct.cpu().numpy().T
    ref = 0.5 * A.conj().T @ B - 2.0 * C0
    scale = 0.5 * np.abs(A).T @ np.abs(B) + 2.0 * np.abs(C0)
    tol = 1e-13 if prec == "c128" else 1e-5
    assert (np.abs(got - ref) / scale).max() < tol


# double-FP32 engine: ~2^-47 per product, the pair accumulator renormalised every 16 terms;
# bound 2e-12 relative to sum |a||b| (the FP64 engine: 1e-13)
DF32_TOL = 2e-12


@pytest.mark.parametrize("n,K", [(1, 1), (64, 925), (65, 5000), (200, 57925), (320, 3001), (33, 100)])
@pytest.mark.parametrize("df32", [False, True])
def test_gram_lower(n, K, df32):
    """Lower triangle of A^H B (complex128); tiles strictly above the diagonal untouched."""
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(n * 3 + K)
    A, B = _c(rng, K, n), _c(rng, K, n)
    At = torch.tensor(A.T.copy(), device="cuda")
    Bt = torch.tensor(B.T.copy(), device="cuda")
    sentinel = 12345.0 + 0j
    Ct = torch.full((n, n), sentinel, dtype=torch.complex128, device="cuda")
    lg.gram_lower(At, Bt, C=Ct, df32=df32)
    got = Ct.cpu().numpy().T
    ref = A.conj().T @ B
    scale = np.abs(A).T @ np.abs(B)
    i, j = np.tril_indices(n)
    assert (np.abs(got[i, j] - ref[i, j]) / scale[i, j]).max() < (DF32_TOL if df32 else 1e-13)
    # 64 x 64 (or 32 x 32 for small FP64 products) tiles strictly above the diagonal keep the sentinel
    bt = 32 if n * n <= 512 * 512 and K <= 8192 and not df32 else 64
    ti, tj = np.meshgrid(np.arange(n) // bt, np.arange(n) // bt, indexing="ij")
    up = ti < tj
    assert np.all(got[up] == sentinel)
    assert np.allclose(got[~up], ref[~up], rtol=0, atol=(1e-11 if df32 else 1e-12) * scale.max())


@pytest.mark.parametrize("m,n,K", [(1, 1, 1), (16, 16, 925), (64, 37, 5000), (192, 192, 57925), (256, 320, 57925),
                                   (7, 130, 100)])
def test_gemm_cn_df32(m, n, K):
    """Double-FP32 A^H B against FP64 numpy, with a planted-cancellation column: a Gram entry
    that is tiny next to sum |a||b| must still come out to FP64 class (an FP32 accumulator
    would leave ~1e-7 of sum |a||b| there)."""
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(m * 11 + n + K)
    A, B, C0 = _c(rng, K, m), _c(rng, K, n), _c(rng, m, n)
    if K > 1 and n > 1:
        B[:, 0] = B[:, 0] - A[:, 0] * (A[:, 0].conj() @ B[:, 0]) / (A[:, 0].conj() @ A[:, 0])  # a0 ^H b0 ~ 0
    At = torch.tensor(A.T.copy(), device="cuda")
    Bt = torch.tensor(B.T.copy(), device="cuda")
    Ct = torch.tensor(C0.T.copy(), device="cuda")
    lg.gemm_cn(At, Bt, alpha=0.5, beta=-2.0, C=Ct, df32=True)
    got = Ct.cpu().numpy().T
    ref = 0.5 * A.conj().T @ B - 2.0 * C0
    scale = 0.5 * np.abs(A).T @ np.abs(B) + 2.0 * np.abs(C0)
    assert (np.abs(got - ref) / scale).max() < DF32_TOL


@pytest.mark.parametrize("M,n,k", [(1, 1, 1), (925, 16, 16), (57925, 64, 128), (57925, 320, 320), (3001, 7, 432),
                                   (100, 130, 65)])
def test_gemm_nn_df32(M, n, k):
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(M + 5 * n + k)
    A, B, C0 = _c(rng, M, k), _c(rng, k, n), _c(rng, M, n)
    At = torch.tensor(A.T.copy(), device="cuda")
    Bt = torch.tensor(B.T.copy(), device="cuda")
    Ct = torch.tensor(C0.T.copy(), device="cuda")
    D = lg.gemm_nn(At, Bt, alpha=-1.0, beta=1.0, C=Ct, D=Ct, df32=True)   # in-place accumulate
    got = D.cpu().numpy().T
    ref = -A @ B + C0
    scale = np.abs(A) @ np.abs(B) + np.abs(C0)
    assert (np.abs(got - ref) / scale).max() < DF32_TOL


@pytest.mark.parametrize("M,n,k", [(1, 1, 1), (925, 16, 16), (57925, 64, 128), (3001, 7, 432), (100, 130, 65)])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_gemm_nn(M, n, k, prec):
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(M + n + k)
    A, B, C0 = _c(rng, M, k), _c(rng, k, n), _c(rng, M, n)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    At = torch.tensor(A.T.copy(), dtype=dt, device="cuda")
    Bt = torch.tensor(B.T.copy(), dtype=dt, device="cuda")
    Ct = torch.tensor(C0.T.copy(), dtype=dt, device="cuda")
    D = lg.gemm_nn(At, Bt, alpha=-1.0, beta=1.0, C=Ct, D=Ct)   # in-place accumulate
    got = D.cpu().numpy().T
    ref = -A @ B + C0
    scale = np.abs(A) @ np.abs(B) + np.abs(C0)
    tol = 1e-13 if prec == "c128" else 1e-5
    assert (np.abs(got - ref) / scale).max() < tol


@pytest.fixture
def gemm_mode():
    import paper_0707_3405_gb300 as lg
    yield lg.set_gemm_mode
    lg.set_gemm_mode(0)


# complex64 on the tensor cores (3xTF32): shapes of the projector, Gram, constraint and update
# products, plus ragged edges (partial M / N tiles, K tails, N above one tile)
@pytest.mark.parametrize("m,n,K", [(256, 256, 57925), (192, 128, 57925), (64, 64, 5000), (130, 7, 3001),
                                   (17, 300, 2000), (1, 1, 1024), (129, 65, 1031)])
@pytest.mark.parametrize("mode", [0, 3])
def test_gemm_cn_c64_engines(m, n, K, mode, gemm_mode):
    import torch
    import paper_0707_3405_gb300 as lg
    gemm_mode(mode)
    rng = np.random.default_rng(m * 13 + n + K)
    A, B, C0 = _c(rng, K, m), _c(rng, K, n), _c(rng, m, n)
    At = torch.tensor(A.T.copy(), dtype=torch.complex64, device="cuda")
    Bt = torch.tensor(B.T.copy(), dtype=torch.complex64, device="cuda")
    Ct = torch.tensor(C0.T.copy(), dtype=torch.complex64, device="cuda")
    lg.gemm_cn(At, Bt, alpha=0.75, beta=0.5, C=Ct)
    lg.check_timeouts()
    A32 = At.cpu().numpy().T.astype(np.complex128)   # the inputs as the GPU sees them (rounded to FP32)
    B32 = Bt.cpu().numpy().T.astype(np.complex128)
    C32 = C0.astype(np.complex64).astype(np.complex128)
    ref = 0.75 * A32.conj().T @ B32 + 0.5 * C32
    scale = 0.75 * np.abs(A32).T @ np.abs(B32) + 0.5 * np.abs(C32)
    got = Ct.cpu().numpy().T
    assert (np.abs(got - ref) / scale).max() < 2e-6


@pytest.mark.parametrize("M,n,k", [(57925, 256, 256), (57925, 64, 192), (3001, 7, 432), (1500, 300, 17),
                                   (1024, 1, 1), (2049, 129, 65)])
@pytest.mark.parametrize("mode", [0, 3])
def test_gemm_nn_c64_engines(M, n, k, mode, gemm_mode):
    import torch
    import paper_0707_3405_gb300 as lg
    gemm_mode(mode)
    rng = np.random.default_rng(M + 3 * n + k)
    A, B, C0 = _c(rng, M, k), _c(rng, k, n), _c(rng, M, n)
    At = torch.tensor(A.T.copy(), dtype=torch.complex64, device="cuda")
    Bt = torch.tensor(B.T.copy(), dtype=torch.complex64, device="cuda")
    Ct = torch.tensor(C0.T.copy(), dtype=torch.complex64, device="cuda")
    D = lg.gemm_nn(At, Bt, alpha=-1.5, beta=1.0, C=Ct, D=Ct)
    lg.check_timeouts()
    A32 = At.cpu().numpy().T.astype(np.complex128)
    B32 = Bt.cpu().numpy().T.astype(np.complex128)
    C32 = C0.astype(np.complex64).astype(np.complex128)
    ref = -1.5 * A32 @ B32 + C32
    scale = 1.5 * np.abs(A32) @ np.abs(B32) + np.abs(C32)
    got = D.cpu().numpy().T
    assert (np.abs(got - ref) / scale).max() < 2e-6
    # beta = 0 writes D without reading it
    D2 = lg.gemm_nn(At, Bt, alpha=1.0, beta=0.0)
    lg.check_timeouts()
    assert (np.abs(D2.cpu().numpy().T - A32 @ B32) / (np.abs(A32) @ np.abs(B32))).max() < 2e-6


def test_gemm_mode_rejects_unknown():
    import paper_0707_3405_gb300 as lg
    with pytest.raises(lg.LobpcgError):
        lg.set_gemm_mode(1)
    lg.set_gemm_mode(0)


def _herm(rng, n):
    A = _c(rng, n, n)
    return A + A.conj().T


@pytest.mark.parametrize("n", [1, 2, 5, 33, 48, 192, 193, 257, 384, 416, 417])
def test_heev(n):
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(n)
    A = _herm(rng, n)
    w, V = lg.heev(torch.tensor(A.T.copy(), device="cuda"))
    w = w.cpu().numpy()
    V = V.cpu().numpy().T                  # columns = eigenvectors
    nrm = np.abs(A).sum(1).max()
    assert np.abs(w - np.linalg.eigvalsh(A)).max() < 1e-12 * nrm
    assert np.abs(A @ V - V * w[None, :]).max() < 1e-11 * nrm
    assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-12


def test_heev_degenerate_clusters():
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(5)
    n = 60
    U, _ = np.linalg.qr(_c(rng, n, n))
    ev = np.concatenate([[0.0] * 6, [1.0] * 12, np.linspace(2, 5, n - 18)])
    A = (U * ev) @ U.conj().T
    w, V = lg.heev(torch.tensor(A.T.copy(), device="cuda"))
    w = w.cpu().numpy()
    V = V.cpu().numpy().T
    assert np.abs(w - ev).max() < 1e-12 * 5
    assert np.abs(A @ V - V * w[None, :]).max() < 1e-11 * 5
    assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-12


@pytest.mark.parametrize("n,m", [(3, 1), (48, 16), (192, 64), (384, 128), (416, 100), (640, 200)])
@pytest.mark.parametrize("df32", [False, True])
def test_rayleigh_ritz_generalized(n, m, df32):
    """FP64 Rayleigh-Ritz against scipy's generalized eigh; df32 = the double-FP32 variant
    (Cholesky diagonal blocks, tridiagonalisation column work, small products), same bounds."""
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(n + m)
    Z = _c(rng, 4 * n, n)
    H = _herm(rng, 4 * n)
    S = Z.conj().T @ Z
    A = Z.conj().T @ H @ Z
    theta, C, nd = lg.rayleigh_ritz(torch.tensor(S.T.copy(), device="cuda"), torch.tensor(A.T.copy(), device="cuda"), m,
                                    df32=df32)
    theta = theta.cpu().numpy()
    C = C.cpu().numpy().T
    ref = scipy.linalg.eigh(A, S, eigvals_only=True)[:m]
    sc = np.abs(ref).max()
    assert int(nd.item()) == 0
    assert np.abs(theta - ref).max() < 1e-10 * sc
    assert np.abs(C.conj().T @ S @ C - np.eye(m)).max() < 1e-10
    assert np.abs(A @ C - S @ C * theta[None, :]).max() < 1e-9 * sc * np.abs(S).max()


def test_rayleigh_ritz_drops_dependent_columns():
    """A basis with two (nearly) repeated columns: they are dropped and the Ritz
    pairs of the remaining subspace are returned."""
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(9)
    npw = 300
    X = _c(rng, npw, 6)
    Z = np.hstack([X, X[:, :2] + 1e-9 * _c(rng, npw, 2), _c(rng, npw, 3)])
    H = _herm(rng, npw)
    S = Z.conj().T @ Z
    A = Z.conj().T @ H @ Z
    keep = [0, 1, 2, 3, 4, 5, 8, 9, 10]
    ref = scipy.linalg.eigh(A[np.ix_(keep, keep)], S[np.ix_(keep, keep)], eigvals_only=True)[:4]
    for df32 in (False, True):
        theta, C, nd = lg.rayleigh_ritz(torch.tensor(S.T.copy(), device="cuda"),
                                        torch.tensor(A.T.copy(), device="cuda"), 4, drop_tol=1e-10, df32=df32)
        assert int(nd.item()) == 2
        assert np.abs(theta.cpu().numpy() - ref).max() < 1e-8 * np.abs(ref).max()
        Cn = C.cpu().numpy().T
        assert np.abs(Cn[[6, 7]]).max() < 1e-12 * np.abs(Cn).max()
    theta, C, nd = lg.rayleigh_ritz(torch.tensor(S.T.copy(), device="cuda"), torch.tensor(A.T.copy(), device="cuda"),
                                    4, drop_tol=1e-10)
    assert int(nd.item()) == 2
    assert np.abs(theta.cpu().numpy() - ref).max() < 1e-8 * np.abs(ref).max()
    C = C.cpu().numpy().T
    assert np.abs(C[[6, 7]]).max() < 1e-12 * np.abs(C).max()


@pytest.mark.parametrize("n,m", [(3, 1), (48, 16), (128, 64), (192, 64)])
def test_rayleigh_ritz_fp32(n, m):
    """The FP32 Rayleigh-Ritz used inside the mixed-precision block iterations:
    Ritz values to ~1e-5 relative, C^H S C = I to ~1e-4."""
    import torch
    import paper_0707_3405_gb300 as lg
    rng = np.random.default_rng(100 + n + m)
    Z = _c(rng, 4 * n, n)
    H = _herm(rng, 4 * n)
    S = Z.conj().T @ Z
    A = Z.conj().T @ H @ Z
    theta, C, nd = lg.rayleigh_ritz32(torch.tensor(S.T.copy(), dtype=torch.complex64, device="cuda"),
                                      torch.tensor(A.T.copy(), dtype=torch.complex64, device="cuda"), m)
    theta = theta.cpu().numpy().astype(float)
    C = C.cpu().numpy().T.astype(complex)
    ref = scipy.linalg.eigh(A, S, eigvals_only=True)[:m]
    sc = np.abs(ref).max()
    assert int(nd.item()) == 0
    assert np.abs(theta - ref).max() < 2e-5 * sc
    assert np.abs(C.conj().T @ S @ C - np.eye(m)).max() < 1e-3
