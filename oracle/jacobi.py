"""Cyclic two-sided Jacobi for Hermitian matrices (oracle; test infrastructure).

Used on tiny dense bases as an eigen-solver that does not depend on LAPACK.
Each sweep visits every pair (p, q) once, in the round-robin ("tournament")
order of Brent and Luk: in each of the n-1 rounds the n indices form n/2
disjoint pairs, so all rotations of a round commute and are applied together.

For a pair with ``A[p,p] = a``, ``A[q,q] = d``, ``A[p,q] = b = |b| e^{i phi}``
the unitary ``U = diag(1, e^{-i phi}) [[c, s], [-s, c]]`` with
``t = s/c`` the smaller root of ``t^2 + 2 tau t - 1 = 0``,
``tau = (d - a) / (2 |b|)``, makes ``(U^H A U)[p, q] = 0`` (classical Jacobi
rotation after removing the phase of the off-diagonal element).
"""
from __future__ import annotations

import numpy as np


def _round_robin(n: int):
    """Yield the n-1 rounds of disjoint pairs covering all pairs of range(n) (n even)."""
    players = list(range(n))
    for _ in range(n - 1):
        yield [(players[i], players[n - 1 - i]) for i in range(n // 2)]
        players = [players[0], players[-1]] + players[1:-1]


def jacobi_eigh(A: np.ndarray, tol: float = 1e-14, max_sweeps: int = 60):
    """Eigen-decomposition ``A = V diag(w) V^H`` of a Hermitian matrix.

    Returns ascending eigenvalues ``w`` and the unitary ``V`` (columns are
    eigenvectors).  Sweeps stop when the off-diagonal Frobenius norm is below
    ``tol * ||A||_F``.
    """
    A = np.array(A, dtype=np.complex128)
    n0 = A.shape[0]
    n = n0 + (n0 % 2)
    if n != n0:                                   # pad with an isolated index
        B = np.zeros((n, n), dtype=np.complex128)
        B[:n0, :n0] = A
        A = B
    V = np.eye(n, dtype=np.complex128)
    scale = np.linalg.norm(A)
    if scale == 0.0:
        return np.zeros(n0), np.eye(n0, dtype=np.complex128)
    for _ in range(max_sweeps):
        off = np.linalg.norm(A - np.diag(np.diag(A)))
        if off <= tol * scale:
            break
        for pairs in _round_robin(n):
            P = np.array([p for p, _ in pairs])
            Q = np.array([q for _, q in pairs])
            b = A[P, Q]
            absb = np.abs(b)
            act = absb > 0.0
            a_ = A[P, P].real
            d_ = A[Q, Q].real
            tau = np.where(act, (d_ - a_) / (2.0 * np.where(act, absb, 1.0)), 0.0)
            t = np.where(tau >= 0, 1.0, -1.0) / (np.abs(tau) + np.sqrt(1.0 + tau * tau))
            t = np.where(act, t, 0.0)
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = t * c
            ph = np.where(act, b / np.where(act, absb, 1.0), 1.0)     # e^{i phi}
            # U = [[c, s], [-s e^{-i phi}, c e^{-i phi}]]  (columns p, q)
            u_pp, u_pq = c, s
            u_qp, u_qq = -s * np.conj(ph), c * np.conj(ph)
            # A <- A U  (columns)
            Ap, Aq = A[:, P].copy(), A[:, Q].copy()
            A[:, P] = Ap * u_pp + Aq * u_qp
            A[:, Q] = Ap * u_pq + Aq * u_qq
            # A <- U^H A  (rows)
            Ap, Aq = A[P, :].copy(), A[Q, :].copy()
            A[P, :] = np.conj(u_pp)[:, None] * Ap + np.conj(u_qp)[:, None] * Aq
            A[Q, :] = np.conj(u_pq)[:, None] * Ap + np.conj(u_qq)[:, None] * Aq
            # V <- V U
            Vp, Vq = V[:, P].copy(), V[:, Q].copy()
            V[:, P] = Vp * u_pp + Vq * u_qp
            V[:, Q] = Vp * u_pq + Vq * u_qq
            A[P, Q] = 0.0
            A[Q, P] = 0.0
    w = np.diag(A).real[:n0]
    V = V[:n0, :n0] if n != n0 else V
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]
