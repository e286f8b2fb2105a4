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

Pins (tests/test_oracle_*.py): V=0 closed form, constant-V shift, rank-one KB
secular equation, direct DFT vs analytic Fourier coefficients, Hermiticity,
translation invariance, time reversal, Jacobi vs LAPACK, Courant-Fischer
bounds, LOBPCG vs dense diagonalisation, the Teter-Payne-Allan ratio's small-
and large-x expansions and the band kinetic energy it is scaled by.
"""
