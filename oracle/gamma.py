"""Gamma-point real-wavefunction form of the eigenproblem (oracle; test infrastructure).

At k = 0 with a real local potential and real-space-real projectors, H
commutes with the antiunitary map ``(C c)(G) = conj(c(-G))``: its eigenvectors
can be taken with real ``psi(r)``, i.e. ``c(-G) = conj(c(G))``.  Plane-wave
codes then store only half of the sphere and do real arithmetic (the
"time-reversal" storage plane-wave codes use at Gamma; the paper's Sec. 2.1
expansion restricted to real orbitals).  Nothing about the spectrum changes;
this module states the real form exactly so that a half-sphere solver can be
checked against it.

Real orthonormal basis of the real-wavefunction space (dimension npw):

* ``e_0`` for G = 0;
* for every G in the half set ``S+`` (n_x > 0; or n_x = 0, n_y > 0; or
  n_x = n_y = 0, n_z > 0), ``u_G = (e_G + e_-G)/sqrt 2`` and
  ``v_G = i (e_G - e_-G)/sqrt 2``.

A real coordinate vector ``x = (x_0, x_u, x_v)`` is the sphere vector with
``c(0) = x_0``, ``c(G) = (x_u + i x_v)/sqrt 2`` and ``c(-G) = conj(c(G))``.
Half-sphere storage keeps ``h(0) = c(0)`` and ``h(G) = c(G)`` for G in S+; then
``<a, b> = a_0 b_0 + 2 sum_{S+} Re(conj(h_a(G)) h_b(G))``.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian, lobpcg


def half_set(miller: np.ndarray):
    """Index of G = 0, indices of S+ and of the matching -G, for a sphere
    symmetric under n -> -n (the Gamma-point sphere)."""
    n = np.asarray(miller)
    pos = {tuple(v): i for i, v in enumerate(n)}
    zero = pos.get((0, 0, 0))
    if zero is None:
        raise ValueError("the sphere has no G = 0 (not a Gamma-point sphere)")
    plus, minus = [], []
    for i, (x, y, z) in enumerate(n):
        if x > 0 or (x == 0 and (y > 0 or (y == 0 and z > 0))):
            j = pos.get((-x, -y, -z))
            if j is None:
                raise ValueError("sphere is not symmetric under G -> -G")
            plus.append(i)
            minus.append(j)
    plus, minus = np.array(plus, dtype=np.int64), np.array(minus, dtype=np.int64)
    if 1 + 2 * len(plus) != len(n):
        raise ValueError("sphere is not symmetric under G -> -G")
    return zero, plus, minus


def real_basis(miller: np.ndarray) -> np.ndarray:
    """Unitary ``U`` (npw x npw complex) whose columns are ``e_0, u_G..., v_G...``
    (G over S+ in sphere order)."""
    zero, plus, minus = half_set(miller)
    npw, h = len(miller), len(plus)
    U = np.zeros((npw, npw), dtype=np.complex128)
    s = 1.0 / np.sqrt(2.0)
    U[zero, 0] = 1.0
    cols = np.arange(h)
    U[plus, 1 + cols] = s
    U[minus, 1 + cols] = s
    U[plus, 1 + h + cols] = 1j * s
    U[minus, 1 + h + cols] = -1j * s
    return U


def to_sphere(miller: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Real coordinates (npw, nb) -> sphere coefficients (npw, nb) complex."""
    return real_basis(miller) @ np.asarray(x, dtype=np.float64)


def to_half(miller: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Sphere coefficients of real orbitals -> half storage (1 + |S+|, nb): G = 0 first,
    then S+ in sphere order."""
    zero, plus, _ = half_set(miller)
    c = np.asarray(c)
    return np.concatenate([c[zero:zero + 1], c[plus]], axis=0)


def from_half(miller: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Half storage -> sphere coefficients, filling ``c(-G) = conj(c(G))``."""
    zero, plus, minus = half_set(miller)
    h = np.asarray(h, dtype=np.complex128)
    c = np.zeros((len(miller),) + h.shape[1:], dtype=np.complex128)
    c[zero] = h[0].real
    c[plus] = h[1:]
    c[minus] = np.conj(h[1:])
    return c


def half_inner(ha: np.ndarray, hb: np.ndarray) -> np.ndarray:
    """``A^H B`` of two blocks of real orbitals from their half storage:
    ``h_a(0) h_b(0) + 2 Re(sum_{S+} conj(h_a) h_b)`` (a real matrix)."""
    ha, hb = np.asarray(ha), np.asarray(hb)
    return np.outer(ha[0].real, hb[0].real) + 2.0 * np.real(ha[1:].conj().T @ hb[1:])


class RealHamiltonian:
    """H in the real basis: ``apply(x) = Re(U^H H U x)`` for real coordinate blocks
    ``x`` (the imaginary part vanishes when H has the real form)."""

    def __init__(self, H: hamiltonian.Hamiltonian):
        if np.any(np.asarray(H.kpt) != 0.0):
            raise ValueError("the real form exists at the Gamma point only")
        self.H = H
        self.U = real_basis(H.miller)
        self.T = np.real(np.einsum("gi,g,gi->i", self.U.conj(), H.T, self.U))

    @property
    def npw(self) -> int:
        return self.H.npw

    def apply(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        y = self.U.conj().T @ self.H.apply(self.U @ x)
        return np.real(y)

    def dense(self) -> np.ndarray:
        """``U^H H U`` (complex; real up to rounding when H has the real form)."""
        return self.U.conj().T @ self.H.dense() @ self.U


def solve_real(H: hamiltonian.Hamiltonian, x0: np.ndarray, block: int, nline: int = 4, tol: float = 1e-10,
               max_sweeps: int = 200) -> lobpcg.Result:
    """The block LOBPCG sweeps of ``lobpcg.solve`` run in real arithmetic on the real
    form; ``x0`` real (npw, M).  The eigenvectors returned are real coordinates."""
    return lobpcg.solve(RealHamiltonian(H), np.asarray(x0, dtype=np.float64), block, nline=nline, tol=tol,
                        max_sweeps=max_sweeps, real=True)
