"""Write the stored expected values under tests/golden/ (calls only oracle/ and synth).

Run from the repository root:  python tests/golden/make_golden.py

* gamma24_eig.txt -- the 16 lowest eigenvalues (Ha) of the 24^3 / a = 10 bohr
  Gamma-point cell with four Gaussian atoms (no KB part), from the oracle's
  dense Hamiltonian (direct DFT of V) diagonalised by LAPACK and confirmed by
  the oracle's Jacobi solver.
* tiny_kb_eig.txt -- the 24 lowest eigenvalues of a 12^3 / a = 6 bohr cell
  with two atoms and eight KB projectors at k = (1/4, 1/8, -3/8), same route.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import hamiltonian, jacobi  # noqa: E402


def _eigs(w, nev, use_jacobi):
    Hd = hamiltonian.for_workload(w).dense()
    ev = np.linalg.eigvalsh(Hd)[:nev]
    if use_jacobi:
        ej, _ = jacobi.jacobi_eigh(Hd)
        assert np.abs(ej[:nev] - ev).max() < 1e-11
    return ev


def main():
    w = synth.make_workload("gamma24")
    np.savetxt(os.path.join(HERE, "gamma24_eig.txt"), _eigs(w, 16, False), fmt="%.17e",
               header="16 lowest eigenvalues (Ha), cell a=10 N=24 Gamma, 4 Gaussian atoms, seed 1001; oracle dense H + LAPACK")
    t = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=(0.25, 0.125, -0.375))
    np.savetxt(os.path.join(HERE, "tiny_kb_eig.txt"), _eigs(t, 24, True), fmt="%.17e",
               header="24 lowest eigenvalues (Ha), cell a=6 N=12 k=(1/4,1/8,-3/8), 2 atoms + 8 KB, seed 7; oracle dense H + LAPACK, Jacobi-confirmed")


if __name__ == "__main__":
    main()
