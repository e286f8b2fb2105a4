"""Write the stored expected values under tests/golden/ (calls only oracle/ and synth).

Run from the repository root:  python tests/golden/make_golden.py

* gamma24_eig.txt -- the 16 lowest eigenvalues (Ha) of the 24^3 / a = 10 bohr
  Gamma-point cell with four Gaussian atoms (no KB part), from the oracle's
  dense Hamiltonian (direct DFT of V) diagonalised by LAPACK and confirmed by
  the oracle's Jacobi solver.
* tiny_kb_eig.txt -- the 24 lowest eigenvalues of a 12^3 / a = 6 bohr cell
  with two atoms and eight KB projectors at k = (1/4, 1/8, -3/8), same route.

Full-size cells (minutes to an hour of CPU each; ``python tests/golden/make_golden.py k96``
and so on):

* k96_eig.txt -- the 256 lowest eigenvalues of the 96^3 cell (57925 plane waves,
  64 atoms, 256 KB projectors, k = (1/4,1/4,1/4)): the oracle's block LOBPCG
  with 64 buffer bands to max residual 1e-10 Ha on the 256, confirmed by the
  oracle's Lanczos route (ARPACK) to 1e-10 Ha.
* mp72x10_k0_eig.txt, mp72x10_k1_eig.txt -- the 128 lowest eigenvalues of the
  first two k-points of the 10-k-point 72^3 cell, same two routes
  (``mp72x10``); ``mp72x10_k<j>`` writes the file of k-point j the same way.
* gamma120_eig.txt -- the 1024 lowest eigenvalues of the 120^3 Gamma cell
  (113081 plane waves, 108 atoms, 432 KB projectors): the oracle's block LOBPCG
  with 128 buffer bands to max residual 1e-10 Ha on the 1024.  The Lanczos
  route for it takes hours, so it runs apart on the stored file:
  ``python tests/golden/make_golden.py confirm gamma120`` (agreement 8.7e-13 Ha
  over all 1024, 11344 s on 8 host cores).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import hamiltonian, jacobi, lanczos, lobpcg  # noqa: E402


def _eigs(w, nev, use_jacobi):
    Hd = hamiltonian.for_workload(w).dense()
    ev = np.linalg.eigvalsh(Hd)[:nev]
    if use_jacobi:
        ej, _ = jacobi.jacobi_eigh(Hd)
        assert np.abs(ej[:nev] - ev).max() < 1e-11
    return ev


def _lobpcg_eigs(w, k, nev, nbuf, confirm):
    """Lowest nev eigenvalues of k-point k by the oracle's LOBPCG (buffer bands, tol 1e-10),
    optionally confirmed by the Lanczos route."""
    import time
    H = hamiltonian.for_workload(w, k)
    t0 = time.time()
    r = lobpcg.solve(H, w.x0(H.npw, k, nev + nbuf), block=w.block, nline=w.nline, tol=1e-10, nconv=nev)
    assert r.converged, r.history
    ev = r.eig[:nev]
    print(f"{w.name} k={k}: LOBPCG {r.sweeps} sweeps, max resid {r.resid[:nev].max():.2e}, "
          f"{time.time() - t0:.0f} s", flush=True)
    if confirm:
        t0 = time.time()
        el, _ = lanczos.lowest(H, nev)
        d = np.abs(el - ev).max()
        print(f"{w.name} k={k}: Lanczos agrees to {d:.2e} Ha, {time.time() - t0:.0f} s", flush=True)
        assert d < 1e-10, d
    return ev


def full_size(which):
    if which == "k96":
        w = synth.make_workload("k96")
        np.savetxt(os.path.join(HERE, "k96_eig.txt"), _lobpcg_eigs(w, 0, 256, 64, True), fmt="%.17e",
                   header="256 lowest eigenvalues (Ha), cell a=20 N=96 k=(1/4,1/4,1/4), 64 atoms + 256 KB, seed 1002; "
                          "oracle block LOBPCG (64 buffer bands, resid <= 1e-10) confirmed by oracle Lanczos")
    elif which == "mp72x10" or which.startswith("mp72x10_k"):
        w = synth.make_workload("mp72x10")
        for k in ((0, 1) if which == "mp72x10" else (int(which[len("mp72x10_k"):]),)):
            np.savetxt(os.path.join(HERE, f"mp72x10_k{k}_eig.txt"), _lobpcg_eigs(w, k, 128, 64, True), fmt="%.17e",
                       header=f"128 lowest eigenvalues (Ha), cell a=16 N=72 k-point {k} = {tuple(w.kpts[k])}, 32 atoms + "
                              f"128 KB, seed 1004; oracle block LOBPCG (64 buffer bands, resid <= 1e-10) confirmed by "
                              f"oracle Lanczos")
    elif which == "gamma120":
        w = synth.make_workload("gamma120")
        np.savetxt(os.path.join(HERE, "gamma120_eig.txt"), _lobpcg_eigs(w, 0, 1024, 128, False), fmt="%.17e",
                   header="1024 lowest eigenvalues (Ha), cell a=25 N=120 Gamma, 108 atoms + 432 KB, seed 1003; "
                          "oracle block LOBPCG (128 buffer bands, resid <= 1e-10)")
    else:
        raise SystemExit(f"unknown cell {which}")


def confirm(which):
    """Compare a stored full-size golden with the oracle's Lanczos route (no LOBPCG rerun)."""
    import time
    files = {"gamma120": ("gamma120_eig.txt", 0)}
    name, k = files[which]
    w = synth.make_workload(which)
    ev = np.loadtxt(os.path.join(HERE, name))
    H = hamiltonian.for_workload(w, k)
    t0 = time.time()
    el, _ = lanczos.lowest(H, len(ev))
    d = np.abs(el - ev).max()
    print(f"{which} k={k}: Lanczos ({len(ev)} eigenvalues) agrees with {name} to {d:.2e} Ha, "
          f"{time.time() - t0:.0f} s", flush=True)
    assert d < 1e-10, d


def main():
    if len(sys.argv) > 2 and sys.argv[1] == "confirm":
        for which in sys.argv[2:]:
            confirm(which)
        return
    if len(sys.argv) > 1:
        for which in sys.argv[1:]:
            full_size(which)
        return
    w = synth.make_workload("gamma24")
    np.savetxt(os.path.join(HERE, "gamma24_eig.txt"), _eigs(w, 16, False), fmt="%.17e",
               header="16 lowest eigenvalues (Ha), cell a=10 N=24 Gamma, 4 Gaussian atoms, seed 1001; oracle dense H + LAPACK")
    t = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=(0.25, 0.125, -0.375))
    np.savetxt(os.path.join(HERE, "tiny_kb_eig.txt"), _eigs(t, 24, True), fmt="%.17e",
               header="24 lowest eigenvalues (Ha), cell a=6 N=12 k=(1/4,1/8,-3/8), 2 atoms + 8 KB, seed 7; oracle dense H + LAPACK, Jacobi-confirmed")


if __name__ == "__main__":
    main()
