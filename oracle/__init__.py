"""CPU FP64 oracle for the plane-wave LOBPCG eigensolver -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything from here.  The
product path (the CUDA library and its Python binding) never does, and this
package never imports the product: the two share only the seeded input
generators in ``synth``.

What it computes (Bottin, Leroux, Knyazev, Zerah 2007):

* ``basis``       -- the plane-wave sphere ``1/2 |k+G|^2 <= Ecut`` (Sec. 2.1,
                     expansion of the Kohn-Sham orbitals) and the kinetic diagonal.
* ``hamiltonian`` -- the Hamiltonian ``H = T + V_loc + V_KB`` restricted to the
                     sphere: a dense matrix built from a direct (non-FFT) DFT of
                     the grid potential, and a matrix-free application through a
                     library FFT (Sec. 2.2 items iii and iv).
* ``jacobi``      -- cyclic two-sided Jacobi eigensolver in round-robin
                     (parallel) order, for tiny dense bases.
* ``lobpcg``      -- the block LOBPCG iteration of Algorithm 1 (Sec. 3.2), run
                     block by block with the orthogonality constraint against the
                     previous blocks and closed by a Rayleigh-Ritz step over all M
                     bands (Sec. 3.2, last paragraph).
* ``checks``      -- residual norms, orthonormality and cluster-projector
                     distances used to compare any solver against the oracle.

For the rows beside the LOBPCG path:

* ``density``     -- rho(r) = sum_n f_n |psi_n(r)|^2 on the grid (first step
                     of the SC loop, Sec. 2.1; by FFT, Sec. 2.2 item iii),
                     as a plain sum and by the inverse FFT.
* ``gamma``       -- the Gamma-point real-wavefunction form: half-sphere
                     storage, its inner products, H in a real orthonormal
                     basis, and the LOBPCG sweeps in real arithmetic.
* ``pcg``         -- band-by-band PCG with exact line minimisation (the
                     method Sec. 3.3 compares LOBPCG with).  Its conjugacy
                     coefficient changes the speed, not the converged result,
                     so it is pinned only through convergence.

Pins (tests/test_oracle_*.py): V=0 closed form and cubic-lattice shell counts,
lattice-point counts with points on the sphere's edge, constant-V shift,
rank-one KB secular equation, direct DFT vs analytic Fourier coefficients,
Hermiticity, translation invariance, time reversal, Jacobi vs LAPACK,
Courant-Fischer bounds, LOBPCG vs dense diagonalisation, the block constraint
against exact eigenvectors, the first two LOBPCG steps as Rayleigh-Ritz on
block Krylov spaces, the Teter-Payne-Allan ratio's small- and large-x
expansions and the band kinetic energy it is scaled by
(tests/test_oracle_next.py: density Parseval, plane-wave closed forms,
translation and unitary invariance; real form unitary, real, same spectrum;
PCG line minimum vs brute force, exact two-plane-wave step, monotone Rayleigh
quotient, dense and free-electron limits).  tests/test_oracle_mutants.py
plants one plausible mistake at a time in these modules and checks that a pin
fails for each.
"""
