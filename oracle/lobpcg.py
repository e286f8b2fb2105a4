"""Block LOBPCG of the paper, in plain numpy FP64 (oracle; test infrastructure).

Follows Sec. 3 of Bottin, Leroux, Knyazev, Zerah (2007):

* Algorithm 1 (Sec. 3.2) for one block Psi of m bands, P^(0) = 0, ``nline``
  iterations:
    1. Upsilon = Rayleigh quotients of Psi (Eq. 1),
    2. R = H Psi - Psi Upsilon            (O = I, norm-conserving case),
    3. W = K(R)                           (preconditioned residual),
    4. Rayleigh-Ritz on span[Psi, W, P]; Psi <- Psi Delta + W Lambda + P Gamma
       (the m lowest Ritz pairs),
    5. P <- W Lambda + P Gamma.
* The M bands are processed block after block; each block is kept orthogonal
  to the blocks before it (Sec. 3.2, "multiband-by-multiband"): the block and
  every W are projected out of the span of the earlier blocks.
* A sweep over all blocks is closed by a Rayleigh-Ritz step over all M bands
  (Sec. 3.2, last paragraph; Sec. 2.1 "subspace diagonalization").

Readings where the paper is silent:

* K is the Teter-Payne-Allan (1989) preconditioner the paper's introduction
  cites for plane-wave codes: ``K(x) = (27+18x+12x^2+8x^3) /
  (27+18x+12x^2+8x^3+16x^4)`` with ``x = T(q) / Ekin(psi_i)``, ``Ekin`` the
  kinetic energy of the current band.
* The Rayleigh-Ritz step on a possibly ill-conditioned basis is done by
  scaling the basis to unit norm, diagonalising its Gram matrix and dropping
  directions whose Gram eigenvalue is below ``1e-13`` of the largest (plain
  Rayleigh-Ritz on the retained, orthonormalised basis).
* The first iteration of a block has P = 0, so the subspace is span[Psi, W].
* Convergence: after the all-band Rayleigh-Ritz, every band has
  ``||H x_i - theta_i x_i||_2 <= tol`` with ``||x_i||_2 = 1``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg


def teter(x: np.ndarray) -> np.ndarray:
    """Teter-Payne-Allan preconditioner polynomial ratio K(x)."""
    p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x))
    return p / (p + 16.0 * x ** 4)


def precondition(R: np.ndarray, X: np.ndarray, T: np.ndarray) -> np.ndarray:
    """W = K(R) with ``x = T(q)/Ekin(x_i)`` column by column."""
    ekin = np.einsum("g,gi->i", T, np.abs(X) ** 2) / np.einsum("gi->i", np.abs(X) ** 2)
    return teter(T[:, None] / ekin[None, :]) * R


def project_out(Y: np.ndarray | None, V: np.ndarray) -> np.ndarray:
    """Remove span(Y) from V twice (classical Gram-Schmidt, repeated); Y orthonormal."""
    if Y is None or Y.shape[1] == 0:
        return V
    for _ in range(2):
        V = V - Y @ (Y.conj().T @ V)
    return V


def orthonormalize(V: np.ndarray) -> np.ndarray:
    """Orthonormal basis of span(V) with the same number of columns (Householder QR)."""
    Q, _ = np.linalg.qr(V)
    return Q


def rayleigh_ritz(Z: np.ndarray, HZ: np.ndarray, m: int, drop: float = 1e-13):
    """Lowest m Ritz pairs of H on span(Z): returns (theta, C) with Z C the Ritz vectors."""
    S = Z.conj().T @ Z
    A = Z.conj().T @ HZ
    S = 0.5 * (S + S.conj().T)
    A = 0.5 * (A + A.conj().T)
    d = 1.0 / np.sqrt(np.real(np.diag(S)))
    S = d[:, None] * S * d[None, :]
    A = d[:, None] * A * d[None, :]
    mu, U = np.linalg.eigh(S)
    keep = mu > drop * mu[-1]
    B = U[:, keep] / np.sqrt(mu[keep])[None, :]
    theta, Q = np.linalg.eigh(B.conj().T @ A @ B)
    C = d[:, None] * (B @ Q[:, :m])
    return theta[:m], C


@dataclass
class Result:
    eig: np.ndarray
    X: np.ndarray
    resid: np.ndarray
    sweeps: int
    converged: bool
    history: list = field(default_factory=list)   # max residual after each sweep
    ritz_trace: list = field(default_factory=list)  # per block visit: list of theta arrays


def block_lobpcg(H, X: np.ndarray, T: np.ndarray, Y: np.ndarray | None, nline: int, trace=None):
    """Algorithm 1 on one block X (npw x m), constrained to be orthogonal to Y.

    Returns the updated block, H times it and its Ritz values.
    """
    m = X.shape[1]
    X = orthonormalize(project_out(Y, X))
    HX = H.apply(X)
    # Rayleigh quotients / initial Ritz rotation of the block (step 1)
    theta, C = rayleigh_ritz(X, HX, m)
    X, HX = X @ C, HX @ C
    if trace is not None:
        trace.append(theta.copy())
    P = HP = None
    for _ in range(nline):
        R = HX - X * theta[None, :]                 # step 2
        W = precondition(R, X, T)                   # step 3
        W = project_out(Y, W)                       # constraint against earlier blocks
        HW = H.apply(W)
        if P is None:
            Z, HZ = np.hstack([X, W]), np.hstack([HX, HW])
        else:
            Z, HZ = np.hstack([X, W, P]), np.hstack([HX, HW, HP])
        theta, C = rayleigh_ritz(Z, HZ, m)         # step 4
        Cx, Cw = C[:m], C[m:2 * m]
        Pn, HPn = W @ Cw, HW @ Cw                   # step 5
        if P is not None:
            Cp = C[2 * m:]
            Pn, HPn = Pn + P @ Cp, HPn + HP @ Cp
        X, HX = X @ Cx + Pn, HX @ Cx + HPn
        P, HP = Pn, HPn
        if trace is not None:
            trace.append(theta.copy())
    return X, HX, theta


def solve(H, X0: np.ndarray, block: int, nline: int = 4, tol: float = 1e-10, max_sweeps: int = 200,
          nblocks_only: int | None = None, keep_trace: bool = False, real: bool = False,
          nconv: int | None = None) -> Result:
    """Lowest M = X0.shape[1] eigenpairs of H by block-by-block LOBPCG sweeps.

    ``nblocks_only`` restricts the run to the first blocks (their result does
    not depend on later blocks, which are constrained to be orthogonal to them).
    ``real``: H is a real symmetric operator on real vectors (the Gamma-point real
    form); the same steps then run in real arithmetic.
    ``nconv``: only the lowest ``nconv`` bands must meet ``tol`` (the rest are
    buffer bands iterated along to give the top wanted bands a gap to the
    unresolved spectrum; the paper is silent on them).  Default: all bands.
    """
    X = np.array(X0, dtype=np.float64 if real else np.complex128)
    M = X.shape[1]
    if M % block:
        raise ValueError("number of bands must be a multiple of the block size")
    nb = M // block if nblocks_only is None else nblocks_only
    X = X[:, :nb * block]
    T = H.T
    res = Result(np.zeros(0), X, np.zeros(0), 0, False)
    for sweep in range(1, max_sweeps + 1):
        for b in range(nb):
            Y = X[:, :b * block] if b else None
            trace = [] if keep_trace else None
            Xb, _, _ = block_lobpcg(H, X[:, b * block:(b + 1) * block], T, Y, nline, trace)
            X[:, b * block:(b + 1) * block] = Xb
            if keep_trace:
                res.ritz_trace.append(trace)
        # final Rayleigh-Ritz over all bands handled (Sec. 3.2)
        X = orthonormalize(X)
        HX = H.apply(X)
        theta, C = rayleigh_ritz(X, HX, X.shape[1])
        X, HX = X @ C, HX @ C
        nrm = np.linalg.norm(X, axis=0)
        X, HX = X / nrm[None, :], HX / nrm[None, :]
        r = np.linalg.norm(HX - X * theta[None, :], axis=0)
        rc = r if nconv is None else r[:nconv]
        res.history.append(float(rc.max()))
        res.eig, res.X, res.resid, res.sweeps = theta, X, r, sweep
        if rc.max() <= tol:
            res.converged = True
            break
    return res
