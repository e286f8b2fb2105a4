"""Pins of the oracle's eigensolvers: Jacobi against LAPACK and a 2x2 closed
form; block LOBPCG (Algorithm 1 with the block constraint and the final
Rayleigh-Ritz) against dense diagonalisation, Courant-Fischer bounds and its
special cases m = M and m = 1 (the single-band method of Eq. 2)."""
import numpy as np
import pytest

import synth
from oracle import basis, checks, hamiltonian, jacobi, lanczos, lobpcg


def _rand_herm(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return A + A.conj().T


@pytest.mark.parametrize("n", [1, 2, 7, 40])
def test_jacobi_matches_lapack(n):
    A = _rand_herm(n, n)
    w, V = jacobi.jacobi_eigh(A)
    assert np.abs(w - np.linalg.eigvalsh(A)).max() < 1e-12 * max(1.0, np.abs(A).max())
    assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-13
    assert np.abs(A @ V - V * w[None, :]).max() < 1e-12 * max(1.0, np.abs(A).max())


def test_jacobi_2x2_closed_form():
    a, d, b = 0.3, -1.1, 0.4 - 0.7j
    w, _ = jacobi.jacobi_eigh(np.array([[a, b], [np.conj(b), d]]))
    r = np.sqrt(((a - d) / 2) ** 2 + abs(b) ** 2)
    assert np.allclose(w, [(a + d) / 2 - r, (a + d) / 2 + r], atol=1e-15)


def test_jacobi_on_dense_hamiltonian():
    w = synth.tiny_workload(a=5.0, N=8, natoms=1)
    H = hamiltonian.for_workload(w)
    Hd = H.dense()
    ev, _ = jacobi.jacobi_eigh(Hd)
    assert np.abs(ev - np.linalg.eigvalsh(Hd)).max() < 1e-12


def _tiny(kpt=(0.0, 0.0, 0.0), nb=8, m=4, seed=11):
    w = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=kpt, nbands=nb, block=m, seed=seed)
    H = hamiltonian.for_workload(w)
    return w, H


@pytest.mark.parametrize("kpt", [(0.0, 0.0, 0.0), (0.25, 0.125, -0.375)])
def test_lobpcg_matches_dense(kpt):
    w, H = _tiny(kpt)
    ref = np.linalg.eigvalsh(H.dense())[:8]
    r = lobpcg.solve(H, w.x0(H.npw), block=4, nline=4, tol=1e-10)
    assert r.converged
    assert np.abs(r.eig - ref).max() < 1e-10
    assert checks.orthonormality_error(r.X) < 1e-12
    assert checks.residuals(H, r.X, r.eig).max() < 1e-10


@pytest.mark.parametrize("kpt", [(0.0, 0.0, 0.0), (0.25, 0.125, -0.375)])
def test_lanczos_route_matches_dense(kpt):
    """The second route to the lowest eigenpairs (ARPACK's Lanczos on the matrix-free H, used to
    confirm the full-size goldens) against the dense H diagonalised by LAPACK: the lowest 12
    eigenvalues in ascending order, unit eigenvectors with small residuals, the right spectral
    projectors."""
    w, H = _tiny(kpt)
    ev, V = np.linalg.eigh(H.dense())
    el, X = lanczos.lowest(H, 12)
    assert np.abs(el - ev[:12]).max() < 1e-10
    assert np.all(np.diff(el) >= 0.0)
    assert np.abs(np.linalg.norm(X, axis=0) - 1.0).max() < 1e-12
    assert checks.residuals(H, X, el).max() < 1e-8
    assert checks.projector_distance(X, V[:, :12], ev[:12]) < 1e-8


def test_lobpcg_single_block_is_plain_rayleigh_ritz_iteration():
    """m = M: one block, the constraint is empty; converges to the same pairs."""
    w, H = _tiny(nb=6, m=6)
    ref = np.linalg.eigvalsh(H.dense())[:6]
    r = lobpcg.solve(H, w.x0(H.npw, M=6), block=6, nline=4, tol=1e-10)
    assert r.converged and np.abs(r.eig - ref).max() < 1e-10


def test_lobpcg_block_size_one_band_by_band():
    """m = 1: the single-band locally optimal method of Eq. 2, band by band."""
    w, H = _tiny(nb=4, m=1)
    ref = np.linalg.eigvalsh(H.dense())[:4]
    r = lobpcg.solve(H, w.x0(H.npw, M=4), block=1, nline=4, tol=1e-10, max_sweeps=400)
    assert r.converged and np.abs(r.eig - ref).max() < 1e-10


def test_lobpcg_with_buffer_bands_converges_the_wanted_ones():
    """Buffer bands: 8 wanted bands plus one block of 4 iterated along. The convergence test
    looks at the wanted bands only; they match the dense eigenvalues and meet the tolerance,
    and the buffer bands still bound the next eigenvalues from above (Courant-Fischer)."""
    w, H = _tiny(nb=12, m=4)
    ev = np.linalg.eigvalsh(H.dense())
    r = lobpcg.solve(H, w.x0(H.npw, M=12), block=4, nline=4, tol=1e-10, nconv=8)
    assert r.converged
    assert np.abs(r.eig[:8] - ev[:8]).max() < 1e-10
    assert r.resid[:8].max() <= 1e-10
    assert r.history[-1] == pytest.approx(r.resid[:8].max(), rel=1e-12)
    assert np.all(r.eig[8:] >= ev[8:12] - 1e-10)


def test_lobpcg_ritz_values_bound_and_decrease():
    """Courant-Fischer: the k-th Ritz value of the first block is >= the k-th
    eigenvalue, and within a block visit it never increases."""
    w, H = _tiny(nb=8, m=4)
    exact = np.linalg.eigvalsh(H.dense())
    r = lobpcg.solve(H, w.x0(H.npw), block=4, nline=4, tol=1e-9, keep_trace=True)
    nblk = 2
    for visit, trace in enumerate(r.ritz_trace):
        b = visit % nblk
        for th in trace:
            if b == 0:
                assert np.all(th >= exact[:4] - 1e-11)
        for t0, t1 in zip(trace[:-1], trace[1:]):
            assert np.all(t1 <= t0 + 1e-10)


def test_lobpcg_free_electrons_degenerate_shells():
    """V = 0: the lowest shells of 1/2|G|^2 are highly degenerate; the solver must
    return the closed-form eigenvalues and the right spectral projectors."""
    a, N = 6.0, 12
    k = np.zeros(3)
    miller = basis.sphere(a, N, synth.default_ecut(a, N), k)
    H = hamiltonian.Hamiltonian(a, N, k, miller, np.zeros((N, N, N)))
    T = np.sort(H.T)
    X0 = synth.start_vectors(5, H.npw, 8)
    r = lobpcg.solve(H, X0, block=4, nline=4, tol=1e-10)
    assert r.converged
    assert np.abs(r.eig - T[:8]).max() < 1e-10
    evals, evecs = np.linalg.eigh(H.dense())
    assert checks.projector_distance(r.X, evecs[:, :8], evals[:8]) < 1e-8


def test_lobpcg_workload_gamma24_matches_dense():
    """The 24^3 / 925 plane-wave cell, 16 bands in one block, to 1e-10."""
    w = synth.make_workload("gamma24")
    H = hamiltonian.for_workload(w)
    ref = np.linalg.eigvalsh(H.dense())[:16]
    r = lobpcg.solve(H, w.x0(H.npw), block=16, nline=4, tol=1e-10)
    assert r.converged and np.abs(r.eig - ref).max() < 1e-10


def test_lobpcg_block_stays_orthogonal_to_the_earlier_blocks():
    """Sec. 3.2 multiband-by-multiband: with the constraint block Y spanning the m lowest exact
    eigenvectors, a block visit returns a block orthogonal to Y, and by Courant-Fischer on the
    complement of Y its k-th Ritz value is at least the (m + k)-th eigenvalue."""
    w, H = _tiny(nb=8, m=4)
    ev, V = np.linalg.eigh(H.dense())
    Y = V[:, :4]
    X0 = w.x0(H.npw)[:, 4:8]
    Xb, _, theta = lobpcg.block_lobpcg(H, X0, H.T, Y, nline=4)
    assert np.abs(Y.conj().T @ Xb).max() < 1e-12
    assert np.all(theta >= ev[4:8] - 1e-10)
    assert np.all(theta < ev[4:8] + 0.5 * (ev[8] - ev[4]))    # and it made progress


class _Dense:
    def __init__(self, A):
        self.A = A

    def apply(self, X):
        return self.A @ X


@pytest.mark.parametrize("m", [1, 3])
def test_lobpcg_first_two_steps_are_block_krylov_rayleigh_ritz(m):
    """With a preconditioner that is a multiple of the identity (all kinetic energies equal, so
    the Teter ratio is K(1) everywhere), span[X, W] after the first step and span[X, W, P] after
    the second are the block Krylov spaces span[X0, H X0] and span[X0, H X0, H^2 X0] (P holds
    the previous step's W and P parts, Alg. 1 step 5). So the Ritz values after one and two
    iterations are the lowest Ritz values of H on those Krylov spaces, and the block returned
    after the second is the matching orthonormal Ritz block: it lies in the third Krylov space
    and its residual is orthogonal to it (the Galerkin condition). Dropping P, mixing up the
    coefficient blocks, or taking W from anything but the residual breaks one of these."""
    rng = np.random.default_rng(21 + m)
    n = 40
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = 0.5 * (A + A.conj().T) + np.diag(np.arange(n, dtype=float))
    X0 = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    trace = []
    X2, _, theta = lobpcg.block_lobpcg(_Dense(A), X0, np.ones(n), None, nline=2, trace=trace)

    def krylov(p):
        blocks, B = [], X0
        for _ in range(p):
            blocks.append(B)
            B = A @ B
        Q, _ = np.linalg.qr(np.hstack(blocks))
        return Q, np.linalg.eigvalsh(Q.conj().T @ A @ Q)[:m]

    assert np.abs(trace[0] - krylov(1)[1]).max() < 1e-10
    assert np.abs(trace[1] - krylov(2)[1]).max() < 1e-10
    Q3, ritz3 = krylov(3)
    assert np.abs(trace[2] - ritz3).max() < 1e-10
    assert np.all(trace[2] < trace[1] - 1e-6)
    assert np.abs(X2.conj().T @ X2 - np.eye(m)).max() < 1e-10
    assert np.abs(X2 - Q3 @ (Q3.conj().T @ X2)).max() < 1e-10
    assert np.abs(Q3.conj().T @ (A @ X2 - X2 * theta[None, :])).max() < 1e-9


@pytest.mark.parametrize("m", [1, 3])
def test_lobpcg_p_spans_what_the_previous_iterate_spans(m):
    """Sec. 3.1: replacing the previous iterate X^(i-1) by P^(i) in the basis of the subspace does
    not change the subspace. So at every later iteration the Ritz values the oracle records equal
    the lowest Ritz values of H on span[X^(i), W^(i), X^(i-1)], built here from the iterates of
    shorter runs from the same start (the iteration is deterministic)."""
    rng = np.random.default_rng(31 + m)
    n = 40
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = 0.5 * (A + A.conj().T) + np.diag(np.arange(n, dtype=float))
    X0 = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    T = np.ones(n)
    iters, trace = [X0], []
    for nl in range(1, 4):
        iters.append(lobpcg.block_lobpcg(_Dense(A), X0, T, None, nline=nl)[0])
    lobpcg.block_lobpcg(_Dense(A), X0, T, None, nline=4, trace=trace)
    for i in (2, 3):
        Xi, Xp = iters[i], iters[i - 1]
        th = np.real(np.diag(Xi.conj().T @ A @ Xi))
        Wi = A @ Xi - Xi * th[None, :]          # a multiple of K(R) when all kinetic energies are equal
        Q, _ = np.linalg.qr(np.hstack([Xi, Wi, Xp]))
        ritz = np.linalg.eigvalsh(Q.conj().T @ A @ Q)[:m]
        assert np.abs(trace[i + 1] - ritz).max() < 1e-9, i


def test_residuals_are_taken_on_unit_columns():
    """||H x - eps x|| of the normalised column: zero for a scaled eigenvector, and the same for
    a block and any positive multiple of it."""
    w, H = _tiny()
    ev, V = np.linalg.eigh(H.dense())
    assert checks.residuals(H, 3.7 * V[:, :3], ev[:3]).max() < 1e-12
    X = w.x0(H.npw)[:, :3]
    r1 = checks.residuals(H, X, ev[:3])
    np.testing.assert_allclose(checks.residuals(H, 5.0 * X, ev[:3]), r1, rtol=1e-12)
    assert np.all(r1 > 1e-3)


def test_orthonormality_error_is_the_largest_gram_deviation():
    """max |X^H X - I|: zero for an orthonormal complex block; scaling one column by (1 + e)
    gives exactly (1 + e)^2 - 1 on its diagonal, and mixing one column into another by a
    complex amount c gives |c| off the diagonal (Gram matrix of [q0, q1 + c q0])."""
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 5)) + 1j * rng.standard_normal((30, 5)))
    assert checks.orthonormality_error(Q) < 1e-14
    Q1 = Q.copy()
    Q1[:, 2] *= 1.0 + 1e-3
    assert checks.orthonormality_error(Q1) == pytest.approx((1.0 + 1e-3) ** 2 - 1.0, rel=1e-9)
    c = 0.02 - 0.05j
    Q2 = Q.copy()
    Q2[:, 1] = Q[:, 1] + c * Q[:, 0]
    assert checks.orthonormality_error(Q2) == pytest.approx(max(abs(c), abs(c) ** 2), rel=1e-9)


def test_map_by_miller_recovers_a_permutation():
    """The index map between two orders of the same plane-wave set is the permutation that
    reorders one into the other (brute force over a shuffled sphere); different sets raise."""
    mil = basis.sphere(6.0, 12, synth.default_ecut(6.0, 12), [0.25, 0.125, -0.375])
    rng = np.random.default_rng(3)
    p_src, p_dst = rng.permutation(len(mil)), rng.permutation(len(mil))
    src, dst = mil[p_src], mil[p_dst]
    p = checks.map_by_miller(src, dst)
    assert np.array_equal(src[p], dst)
    assert np.array_equal(p, np.argsort(p_src)[p_dst])
    other = dst.copy()
    other[0] = [99, 0, 0]
    with pytest.raises(ValueError):
        checks.map_by_miller(src, other)


def test_clusters_split_where_the_gap_is_exceeded():
    eig = np.array([0.0, 1e-8, 2e-8, 1.0, 2.0, 2.0 + 5e-7])
    assert checks.clusters(eig, 1e-6) == [(0, 3), (3, 4), (4, 6)]
    assert checks.clusters(eig, 1e-9) == [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6)]
    assert checks.clusters(np.array([3.0]), 1e-6) == [(0, 1)]
    assert checks.clusters(np.array([0.0, 3e-6, 3.5e-6]), 1e-6) == [(0, 1), (1, 3)]


def test_projector_distance_detects_wrong_subspace():
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 6)) + 1j * rng.standard_normal((20, 6)))
    eig = np.array([0, 0, 1, 1, 2, 3.0])
    assert checks.projector_distance(Q, Q @ np.diag(np.exp(1j * np.arange(6))), eig) < 1e-12
    Q2 = Q.copy()
    Q2[:, 2] = Q[:, 4]
    assert checks.projector_distance(Q2, Q, eig) > 0.5


def test_golden_files_reproduce():
    """The stored expected eigenvalues are what the oracle computes today."""
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    w = synth.make_workload("gamma24")
    ev = np.linalg.eigvalsh(hamiltonian.for_workload(w).dense())[:16]
    assert np.abs(np.loadtxt(os.path.join(here, "gamma24_eig.txt")) - ev).max() < 1e-12
    t = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=(0.25, 0.125, -0.375))
    ev = np.linalg.eigvalsh(hamiltonian.for_workload(t).dense())[:24]
    assert np.abs(np.loadtxt(os.path.join(here, "tiny_kb_eig.txt")) - ev).max() < 1e-12


def test_multi_k_goldens_respect_time_reversal():
    """Each stored golden of the 10-k-point 72^3 cell comes from its own LOBPCG run from its own
    start vectors. Where two of its k-points are time-reversal partners (k_i + k_j a reciprocal
    lattice vector; real V and KB projectors), the spectra must coincide: eps(k) = eps(-k)."""
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    w = synth.make_workload("mp72x10")
    pairs = [(i, j) for i in range(w.nk) for j in range(i + 1, w.nk)
             if np.allclose(w.kpts[i] + w.kpts[j], np.round(w.kpts[i] + w.kpts[j]))]
    assert pairs
    for i, j in pairs:
        ei = np.loadtxt(os.path.join(here, f"mp72x10_k{i}_eig.txt"))
        ej = np.loadtxt(os.path.join(here, f"mp72x10_k{j}_eig.txt"))
        assert np.abs(ei - ej).max() < 1e-11, (i, j)


def test_teter_preconditioner_limits_and_shape():
    """The Teter-Payne-Allan ratio K(x) passes low-energy components unchanged to fourth order,
    K = 1 - (16/27) x^4 + (32/81) x^5 + O(x^6), and acts like the inverse kinetic energy at high
    energy, 1/K = 2x - 2 + O(1/x); in between it decreases monotonically inside (0, 1]."""
    K = lobpcg.teter
    assert K(np.array([0.0]))[0] == 1.0
    for x in (0.01, 0.02):
        lead = (1.0 - K(np.array([x]))[0]) / x ** 4
        assert lead == pytest.approx(16.0 / 27.0 - 32.0 / 81.0 * x, abs=1e-6)
    for x in (1e3, 1e4):
        inv = 1.0 / K(np.array([x]))[0]
        assert inv - 2.0 * x == pytest.approx(-2.0, abs=10.0 / x)
    xs = np.linspace(0.0, 200.0, 20001)
    k = K(xs)
    assert np.all(k > 0.0) and np.all(k <= 1.0)
    assert np.all(np.diff(k[1:]) < 0.0)


def test_precondition_uses_the_band_kinetic_energy():
    """W = K(T / Ekin) R column by column, Ekin the kinetic expectation of the band: a band made
    of two plane waves has Ekin = (T_a + T_b) / 2 whatever its norm and phases."""
    rng = np.random.default_rng(5)
    T = np.abs(rng.standard_normal(12)) * 3.0
    X = np.zeros((12, 2), complex)
    X[[2, 7], 0] = 2.5 * np.exp(1j * np.array([0.3, -1.1]))    # two plane waves, equal weight
    X[4, 1] = -0.7j                                           # one plane wave
    R = rng.standard_normal((12, 2)) + 1j * rng.standard_normal((12, 2))
    W = lobpcg.precondition(R, X, T)
    e0 = 0.5 * (T[2] + T[7])
    np.testing.assert_allclose(W[:, 0], lobpcg.teter(T / e0) * R[:, 0], rtol=1e-14)
    np.testing.assert_allclose(W[:, 1], lobpcg.teter(T / T[4]) * R[:, 1], rtol=1e-14)
    # at the band's own plane wave the ratio is K(1) = 65/81
    assert W[4, 1] / R[4, 1] == pytest.approx(65.0 / 81.0, rel=1e-14)
