"""Kohn-Sham Hamiltonian on the plane-wave sphere (oracle; test infrastructure).

Sec. 2.1 / 2.2 of the paper: for a fixed potential the eigenproblem solved
inside the self-consistent loop is ``H c = eps c`` on the plane-wave sphere
(norm-conserving case, overlap O = I).  ``H`` has three parts:

* kinetic ``1/2 |k+G|^2`` on the diagonal;
* the local potential ``v_loc`` (Sec. 2.2 item iii, applied by FFT in the
  paper): with the potential given on the grid ``r_j = a j/N``, its matrix
  element between plane waves ``n`` and ``n'`` is the discrete Fourier
  coefficient ``Vt((n - n') mod N)`` with
  ``Vt(n) = N^-3 sum_j V(r_j) exp(-2 pi i n.j / N)``;
  this is exactly what "inverse FFT, multiply by V(r), forward FFT" on an
  ``N^3`` box computes, so the dense matrix and the FFT route define the same
  operator;
* the non-local Kleinman-Bylander part ``v_nl`` (Sec. 2.2 item iv, Sec. 4.3):
  ``sum_p E_p |beta_p><beta_p|``.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

from . import basis


def direct_dft(v: np.ndarray) -> np.ndarray:
    """``Vt(n) = N^-3 sum_j V(r_j) exp(-2 pi i n.j/N)`` evaluated as a plain sum.

    The triple sum is written as three successive sums over j_z, j_y, j_x of
    the same exponentials (the exponential factorises); no FFT is used.
    Output index is ``n mod N``.
    """
    N = v.shape[0]
    j = np.arange(N)
    F = np.exp(-2j * np.pi * np.outer(j, j) / N)      # F[n, j]
    t = np.einsum("ck,ijk->ijc", F, v.astype(np.complex128))
    t = np.einsum("bj,ijc->ibc", F, t)
    t = np.einsum("ai,ibc->abc", F, t)
    return t / N ** 3


def dense_H(a: float, N: int, kpt, miller: np.ndarray, v: np.ndarray,
            beta: np.ndarray | None = None, E: np.ndarray | None = None) -> np.ndarray:
    """Assemble the npw x npw Hermitian matrix ``H`` element by element.

    ``H[i, j] = T_i delta_ij + Vt((n_i - n_j) mod N) + sum_p E_p beta[i,p] conj(beta[j,p])``.
    """
    vt = direct_dft(v)
    n = np.asarray(miller)
    d = np.mod(n[:, None, :] - n[None, :, :], N)
    H = vt[d[..., 0], d[..., 1], d[..., 2]]
    H = H + np.diag(basis.kinetic(n, kpt, a))
    if beta is not None and beta.shape[1] > 0:
        H = H + (beta * E[None, :]) @ beta.conj().T
    return H


class Hamiltonian:
    """Matrix-free ``H`` on the sphere of one k-point (library FFT for v_loc).

    ``apply(X)`` returns ``H X`` for an (npw, nb) complex block, in FP64.
    """

    def __init__(self, a: float, N: int, kpt, miller: np.ndarray, v: np.ndarray,
                 beta: np.ndarray | None = None, E: np.ndarray | None = None, workers: int = -1):
        self.a, self.N = a, N
        self.kpt = np.asarray(kpt, dtype=np.float64)
        self.miller = np.asarray(miller)
        self.v = np.asarray(v, dtype=np.float64)
        self.T = basis.kinetic(self.miller, self.kpt, a)
        self.idx = basis.box_index(self.miller, N)
        self.beta = beta if (beta is not None and beta.shape[1] > 0) else None
        self.E = None if self.beta is None else np.asarray(E, dtype=np.float64)
        self.workers = workers

    @property
    def npw(self) -> int:
        return self.miller.shape[0]

    def apply_local(self, X: np.ndarray, chunk: int = 8) -> np.ndarray:
        """``V_loc X``: place c(n) at box index n mod N, inverse FFT (sum of
        c(n) exp(+2 pi i n.j/N)), multiply by V(r_j), forward FFT, divide by
        N^3 and read back the sphere entries."""
        N = self.N
        X = np.asarray(X, dtype=np.complex128)
        out = np.empty_like(X)
        for s in range(0, X.shape[1], chunk):
            blk = X[:, s:s + chunk]
            box = np.zeros((N, N, N, blk.shape[1]), dtype=np.complex128)
            box[self.idx] = blk
            psi = scipy.fft.ifftn(box, axes=(0, 1, 2), norm="forward", workers=self.workers)
            psi *= self.v[..., None]
            Vpsi = scipy.fft.fftn(psi, axes=(0, 1, 2), norm="forward", workers=self.workers)
            out[:, s:s + chunk] = Vpsi[self.idx]
        return out

    def apply_nonlocal(self, X: np.ndarray) -> np.ndarray:
        """``sum_p E_p beta_p (beta_p^H X)``."""
        if self.beta is None:
            return np.zeros_like(X, dtype=np.complex128)
        B = self.beta.conj().T @ X
        return self.beta @ (self.E[:, None] * B)

    def apply(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.complex128)
        one = X.ndim == 1
        if one:
            X = X[:, None]
        Y = self.T[:, None] * X + self.apply_local(X) + self.apply_nonlocal(X)
        return Y[:, 0] if one else Y

    def dense(self) -> np.ndarray:
        """The same operator as an explicit matrix (direct DFT, no FFT)."""
        return dense_H(self.a, self.N, self.kpt, self.miller, self.v, self.beta, self.E)


def for_workload(w, k_index: int = 0, workers: int = -1) -> Hamiltonian:
    """Oracle Hamiltonian of k-point ``k_index`` of a ``synth.Workload``."""
    kpt = w.kpts[k_index]
    miller = basis.sphere(w.a, w.N, w.ecut, kpt)
    beta = w.beta(miller, k_index) if w.nproj else None
    return Hamiltonian(w.a, w.N, kpt, miller, w.vloc(), beta, w.proj_E if w.nproj else None, workers=workers)
