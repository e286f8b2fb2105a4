"""Comparisons of a solver's output with the oracle (test infrastructure)."""
from __future__ import annotations

import numpy as np


def residuals(H, X: np.ndarray, eig: np.ndarray) -> np.ndarray:
    """``||H x_i - eps_i x_i||_2`` of unit-normalised columns, with the oracle's H."""
    X = np.asarray(X, dtype=np.complex128)
    X = X / np.linalg.norm(X, axis=0)[None, :]
    return np.linalg.norm(H.apply(X) - X * np.asarray(eig)[None, :], axis=0)


def orthonormality_error(X: np.ndarray) -> float:
    """``max |X^H X - I|``."""
    X = np.asarray(X, dtype=np.complex128)
    return float(np.abs(X.conj().T @ X - np.eye(X.shape[1])).max())


def clusters(eig: np.ndarray, gap: float) -> list:
    """Index ranges of eigenvalues closer than ``gap`` to a neighbour."""
    out, start = [], 0
    for i in range(1, len(eig) + 1):
        if i == len(eig) or eig[i] - eig[i - 1] > gap:
            out.append((start, i))
            start = i
    return out


def projector_distance(X: np.ndarray, Xref: np.ndarray, eig_ref: np.ndarray, gap: float = 1e-6) -> float:
    """Largest ``||X_c X_c^H - R_c R_c^H||_2`` over clusters of (near) equal eigenvalues.

    Eigenvectors are unique only up to a unitary mixing within a degenerate
    cluster (and a phase), so the spectral projectors are compared instead.
    The last cluster is skipped when it may be cut by the end of the band range.
    """
    worst = 0.0
    cl = clusters(np.asarray(eig_ref), gap)
    for (s, e) in cl[:-1] if len(cl) > 1 else cl:
        A = np.asarray(X[:, s:e], dtype=np.complex128)
        B = np.asarray(Xref[:, s:e], dtype=np.complex128)
        # ||A A^H - B B^H||_2 = sin of the largest principal angle = ||(I - B B^H) A||_2
        s_ = np.linalg.svd(A - B @ (B.conj().T @ A), compute_uv=False)
        worst = max(worst, float(s_.max()))
    return worst


def map_by_miller(miller_src: np.ndarray, miller_dst: np.ndarray) -> np.ndarray:
    """Permutation ``p`` with ``miller_src[p] == miller_dst`` (row-wise)."""
    key = lambda m: (np.asarray(m, dtype=np.int64) + 4096) @ np.array([1 << 26, 1 << 13, 1], dtype=np.int64)
    ks, kd = key(miller_src), key(miller_dst)
    order = np.argsort(ks)
    pos = np.searchsorted(ks[order], kd)
    if np.any(pos >= len(ks)) or np.any(ks[order][np.minimum(pos, len(ks) - 1)] != kd):
        raise ValueError("plane-wave sets differ")
    return order[pos]
