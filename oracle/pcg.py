"""Band-by-band preconditioned conjugate gradient for a fixed H (oracle; test infrastructure).

The paper compares its LOBPCG with the band-by-band PCG of Teter, Payne and
Allan (1989) in the iterative-diagonalisation form of Bylander et al. (1990)
(Sec. 1; Sec. 3.3).  It does not restate that method, so this module takes
the steps as those references define them, for a fixed Hamiltonian:

for every band n in order, kept orthogonal to the bands before it, ``nline``
iterations of

1. ``eps = <x|H|x>`` for the normalised band ``x``;
2. the steepest-descent direction ``xi = -(H x - eps x)``, orthogonalised to the
   earlier bands and to ``x``;
3. the preconditioned direction ``eta = K(xi)`` (the Teter ratio of the LOBPCG
   oracle, ``x = T(q)/Ekin(x)``), orthogonalised the same way;
4. the conjugate direction ``d = eta + gamma d_prev`` with
   ``gamma = <eta|xi> / <eta_prev|xi_prev>`` (0 on the first iteration);
5. ``d`` made orthogonal to ``x`` and normalised to ``d^``;
6. exact line minimisation of the Rayleigh quotient on
   ``x(theta) = cos(theta) x + sin(theta) d^`` (the two-dimensional
   Rayleigh-Ritz problem on span[x, d^]), and ``x <- x(theta*)``.

A sweep over all bands is closed by the same all-band Rayleigh-Ritz step as
the LOBPCG oracle (Sec. 2.1, subspace diagonalisation after the eigensolver),
and the same convergence test (every residual ``<= tol``) ends the run.
"""
from __future__ import annotations

import numpy as np

from .lobpcg import Result, orthonormalize, precondition, project_out, rayleigh_ritz


def line_minimum(A: float, B: float, C: float):
    """Minimiser of ``E(theta) = A cos^2 + B sin^2 + 2 C sin cos``.

    ``E = (A+B)/2 + (A-B)/2 cos(2 theta) + C sin(2 theta)`` is smallest where
    ``(cos 2theta, sin 2theta)`` points against ``((A-B)/2, C)``; returns
    ``(theta, E(theta))`` with ``theta`` in ``(-pi/2, pi/2]``.
    """
    theta = 0.5 * np.arctan2(-2.0 * C, B - A)
    c, s = np.cos(theta), np.sin(theta)
    return float(theta), float(A * c * c + B * s * s + 2.0 * C * s * c)


def band_pcg(H, x: np.ndarray, T: np.ndarray, Y: np.ndarray | None, nline: int, trace=None):
    """``nline`` PCG iterations on one band ``x`` kept orthogonal to the orthonormal
    block ``Y`` (the bands before it); returns the new band and its Rayleigh quotient."""
    x = project_out(Y, x.reshape(-1, 1))
    x = x / np.linalg.norm(x)
    hx = H.apply(x)
    eps = float(np.real(np.vdot(x, hx)))
    if trace is not None:
        trace.append(eps)
    d_prev, dot_prev = None, None
    for _ in range(nline):
        xi = -(hx - eps * x)                                   # step 2
        xi = project_out(Y, xi)
        xi = xi - x * np.vdot(x, xi)
        eta = precondition(xi, x, T)                           # step 3
        eta = project_out(Y, eta)
        eta = eta - x * np.vdot(x, eta)
        dot = float(np.real(np.vdot(eta, xi)))
        d = eta if d_prev is None or dot_prev == 0.0 else eta + (dot / dot_prev) * d_prev   # step 4
        d_prev, dot_prev = d, dot
        dh = d - x * np.vdot(x, d)                             # step 5
        nd = np.linalg.norm(dh)
        if nd == 0.0:
            break
        dh = dh / nd
        hd = H.apply(dh)
        B = float(np.real(np.vdot(dh, hd)))                    # step 6
        C = float(np.real(np.vdot(x, hd)))
        theta, _ = line_minimum(eps, B, C)
        c, s = np.cos(theta), np.sin(theta)
        x, hx = c * x + s * dh, c * hx + s * hd
        nx = np.linalg.norm(x)
        x, hx = x / nx, hx / nx
        eps = float(np.real(np.vdot(x, hx)))
        if trace is not None:
            trace.append(eps)
    return x[:, 0], eps


def solve_pcg(H, X0: np.ndarray, nline: int = 4, tol: float = 1e-10, max_sweeps: int = 500,
              keep_trace: bool = False) -> Result:
    """Lowest M = X0.shape[1] eigenpairs of H by band-by-band PCG sweeps, each closed
    by an all-band Rayleigh-Ritz step."""
    X = np.array(X0, dtype=np.complex128)
    M = X.shape[1]
    T = H.T
    res = Result(np.zeros(0), X, np.zeros(0), 0, False)
    for sweep in range(1, max_sweeps + 1):
        for n in range(M):
            trace = [] if keep_trace else None
            X[:, n], _ = band_pcg(H, X[:, n], T, X[:, :n] if n else None, nline, trace)
            if keep_trace:
                res.ritz_trace.append(trace)
        X = orthonormalize(X)
        HX = H.apply(X)
        theta, C = rayleigh_ritz(X, HX, M)
        X, HX = X @ C, HX @ C
        nrm = np.linalg.norm(X, axis=0)
        X, HX = X / nrm[None, :], HX / nrm[None, :]
        r = np.linalg.norm(HX - X * theta[None, :], axis=0)
        res.history.append(float(r.max()))
        res.eig, res.X, res.resid, res.sweeps = theta, X, r, sweep
        if r.max() <= tol:
            res.converged = True
            break
    return res
