"""Electron density on the real-space grid (oracle; test infrastructure).

The first step of the self-consistent loop (Sec. 2.1) builds the density from
the orbitals; in the norm-conserving case (O = I, no compensation charge) it
is ``rho(r) = sum_{k,n} w_k f_nk |psi_nk(r)|^2``.  The same 3D FFT that applies
the local potential takes each band to real space for it (Sec. 2.2 item iii;
Sec. 4.1, last paragraph, where the per-band contributions are summed over
bands).  So the density needs only the first half of the H-application
machinery (sphere -> box, inverse FFT) and a weighted sum of squared moduli.

Conventions (the same as the Hamiltonian's):

* ``psi(r) = Omega^-1/2 sum_G c(G) exp(i (k+G).r)`` with orthonormal
  coefficient vectors, ``Omega = a^3``;
* on the grid ``r_j = a j / N`` the factor ``exp(i G.r_j)`` is
  ``exp(2 pi i n.j / N)``; the Bloch phase ``exp(i k.r)`` has modulus one and
  drops out of ``|psi|^2``.

``density_direct`` is the definition written out as a plain sum over plane
waves at every grid point; ``density`` takes the inverse FFT route.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

from . import basis


def density_direct(a: float, N: int, miller: np.ndarray, C: np.ndarray, f: np.ndarray) -> np.ndarray:
    """``rho(r_j) = Omega^-1 sum_n f_n |sum_G c_n(G) exp(2 pi i n_G.j/N)|^2`` on the
    ``N^3`` grid, ``[x][y][z]``, by the plain sum (tiny grids only)."""
    n = np.asarray(miller, dtype=np.float64)
    g = np.arange(N)
    j = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3).astype(np.float64)
    E = np.exp(2j * np.pi * (j @ n.T) / N)              # (N^3, npw)
    psi = E @ np.asarray(C, dtype=np.complex128)        # (N^3, nb), without Omega^-1/2
    rho = (np.abs(psi) ** 2) @ np.asarray(f, dtype=np.float64)
    return rho.reshape(N, N, N) / a ** 3


def density(a: float, N: int, miller: np.ndarray, C: np.ndarray, f: np.ndarray) -> np.ndarray:
    """The same density through the inverse FFT: each band placed at box index
    ``n mod N``, summed over ``exp(+2 pi i n.j/N)`` (no 1/N^3), squared modulus,
    weighted by ``f_n`` and divided by ``Omega``."""
    C = np.asarray(C, dtype=np.complex128)
    idx = basis.box_index(miller, N)
    rho = np.zeros((N, N, N))
    for b in range(C.shape[1]):
        box = np.zeros((N, N, N), dtype=np.complex128)
        box[idx] = C[:, b]
        psi = scipy.fft.ifftn(box, norm="forward")
        rho += float(f[b]) * (psi.real ** 2 + psi.imag ** 2)
    return rho / a ** 3


def electron_count(a: float, rho: np.ndarray) -> float:
    """``int rho dr`` by the grid rule ``(Omega / N^3) sum_j rho(r_j)`` (exact for a
    density of band-limited orbitals whose sphere fits the box)."""
    N = rho.shape[0]
    return float(rho.sum()) * a ** 3 / N ** 3
