"""Plane-wave basis of the oracle (test infrastructure; see oracle/__init__.py).

Sec. 2.1 expands each orbital as ``psi_nk(r) = sum_G c_nk(G) exp(i(k+G).r)``.
For a cubic cell of side ``a`` the reciprocal vectors are ``G_n = (2 pi/a) n``
for integer triplets ``n``; the basis at k-point ``k`` (reduced coordinates)
is every ``n`` with ``1/2 |q_n|^2 <= Ecut``, ``q_n = (2 pi/a)(n + k)``.

Reading used for the sphere edge: the test is done in index units,
``|n + k|^2 <= 2 Ecut (a / 2 pi)^2 + 1e-9``, so that lattice points lying
exactly on the sphere (they exist for the default cutoff) are always kept.
"""
from __future__ import annotations

import math

import numpy as np


def sphere(a: float, N: int, ecut: float, kpt) -> np.ndarray:
    """Miller indices (npw, 3) int64 of the sphere, sorted by (n_x, n_y, n_z).

    Every index must lie in the FFT box ``[-N/2, N/2-1]``; a cutoff too large
    for the grid raises ``ValueError``.
    """
    k = np.asarray(kpt, dtype=np.float64)
    r2 = 2.0 * ecut * (a / (2.0 * math.pi)) ** 2
    lim = int(math.ceil(math.sqrt(r2))) + 2
    rng = np.arange(-lim, lim + 1)
    nx, ny, nz = np.meshgrid(rng, rng, rng, indexing="ij")
    n = np.stack([nx.ravel(), ny.ravel(), nz.ravel()], axis=1)
    d = n + k[None, :]
    keep = np.einsum("ij,ij->i", d, d) <= r2 + 1e-9
    n = n[keep]
    if n.size and (n.min() < -(N // 2) or n.max() > N - N // 2 - 1):
        raise ValueError("plane-wave sphere does not fit in the FFT box")
    order = np.lexsort((n[:, 2], n[:, 1], n[:, 0]))
    return n[order].astype(np.int64)


def kinetic(miller: np.ndarray, kpt, a: float) -> np.ndarray:
    """Kinetic diagonal ``T(n) = 1/2 |q_n|^2`` (Ha) of each plane wave."""
    q = (2.0 * math.pi / a) * (np.asarray(miller, dtype=np.float64) + np.asarray(kpt, dtype=np.float64)[None, :])
    return 0.5 * np.einsum("ij,ij->i", q, q)


def box_index(miller: np.ndarray, N: int) -> tuple:
    """FFT-box position ``n mod N`` of every plane wave, as an index tuple."""
    m = np.mod(np.asarray(miller), N)
    return (m[:, 0], m[:, 1], m[:, 2])
