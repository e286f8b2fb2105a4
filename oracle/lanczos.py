"""Lowest eigenvalues of the plane-wave Hamiltonian by implicitly restarted
Lanczos (ARPACK through scipy) -- oracle; test infrastructure.

This is a second, independent route to the result the LOBPCG sweeps compute
(the M lowest eigenpairs of the Hermitian operator H of Sec. 2.1-2.2 on the
plane-wave sphere): a library eigensolver takes the oracle's matrix-free
``Hamiltonian.apply`` one vector at a time.  It shares no step with
``oracle.lobpcg`` (no blocks, no preconditioner, no Rayleigh-Ritz on
[X W P]), so agreement of the two pins the LOBPCG oracle at sizes where the
dense matrix no longer fits, and in particular shows that no eigenvalue was
skipped (a residual test alone cannot show that).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as sla


def lowest(H, nev: int, tol: float = 1e-13, ncv: int | None = None, seed: int = 5) -> tuple:
    """``(eig, X)``: the ``nev`` algebraically smallest eigenvalues (ascending) and
    unit eigenvectors (npw, nev) of ``H`` by ARPACK's Hermitian Lanczos driver."""
    n = H.npw
    op = sla.LinearOperator((n, n), matvec=lambda v: H.apply(np.asarray(v, dtype=np.complex128).reshape(-1)),
                            dtype=np.complex128)
    rng = np.random.default_rng(seed)
    v0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ncv = ncv if ncv is not None else min(n, max(2 * nev + 1, nev + 64))
    w, X = sla.eigsh(op, k=nev, which="SA", tol=tol, ncv=ncv, v0=v0)
    order = np.argsort(w)
    return w[order], X[:, order]
