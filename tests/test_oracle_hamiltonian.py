"""Pins of the oracle's basis and Hamiltonian against closed forms and invariants.

None of these compares the oracle with itself: each expected value comes from
mathematics the paper's setting fixes (Sec. 2.1 plane-wave expansion, a real
local potential, a Hermitian KB projector sum) or from an independent library
routine.
"""
import math

import numpy as np
import pytest
import scipy.optimize

import synth
from oracle import basis, hamiltonian


def _ham(w, v=None, with_kb=True, k_index=0):
    kpt = w.kpts[k_index]
    miller = basis.sphere(w.a, w.N, w.ecut, kpt)
    beta = w.beta(miller, k_index) if (with_kb and w.nproj) else None
    return hamiltonian.Hamiltonian(w.a, w.N, kpt, miller, w.vloc() if v is None else v,
                                   beta, w.proj_E if beta is not None else None)


# ---------------------------------------------------------------- sphere
@pytest.mark.parametrize("name,approx", [("gamma24", 900), ("k96", 58e3), ("gamma120", 113e3),
                                         ("mp72x10", 24e3), ("large160", 268e3)])
def test_sphere_size_matches_stated_and_volume(name, approx):
    """npw agrees with the stated approximate sizes and with the sphere volume."""
    w = synth.make_workload(name)
    for k in w.kpts:
        n = basis.sphere(w.a, w.N, w.ecut, k).shape[0]
        assert abs(n - approx) / approx < 0.03
        vol = 4.0 / 3.0 * math.pi * (w.N / 4.0) ** 3     # |n+k| <= N/4 in index units
        assert abs(n - vol) / vol < 0.03


def test_sphere_brute_force_tiny():
    """Every box point inside the cutoff is present exactly once, none outside."""
    a, N, ecut, k = 5.0, 12, 3.1, np.array([0.125, -0.375, 0.25])
    got = {tuple(r) for r in basis.sphere(a, N, ecut, k)}
    want = set()
    for i in range(-N // 2, N // 2):
        for j in range(-N // 2, N // 2):
            for l in range(-N // 2, N // 2):
                qx, qy, qz = (2 * math.pi / a) * (i + k[0]), (2 * math.pi / a) * (j + k[1]), (2 * math.pi / a) * (l + k[2])
                if 0.5 * (qx * qx + qy * qy + qz * qz) <= ecut:
                    want.add((i, j, l))
    assert got == want


def test_sphere_keeps_lattice_points_on_the_edge():
    """The cutoff is inclusive (1/2 |k+G|^2 <= Ecut): with a = 2 pi and Ecut = R/2 the sphere at
    k = 0 is every integer point with |n|^2 <= R, whose count is the number of cubic-lattice
    points in a ball of squared radius R, sum_{j <= R} r_3(j) (r_3(j): ways of writing j as a
    sum of three squares): 1, 7, 19, 27, 33, 57, 81, 81, 93, 123, 147 for R = 0 ... 10."""
    counts = [1, 7, 19, 27, 33, 57, 81, 81, 93, 123, 147]
    for R, want in enumerate(counts):
        n = basis.sphere(2.0 * math.pi, 16, R / 2.0, [0.0, 0.0, 0.0])
        assert n.shape[0] == want, R
        assert np.all(np.einsum("ij,ij->i", n, n) <= R)


def test_sphere_too_large_raises():
    with pytest.raises(ValueError):
        basis.sphere(5.0, 8, 40.0, [0, 0, 0])


# ---------------------------------------------------------------- Fourier conventions
def test_direct_dft_matches_library_fft():
    rng = np.random.default_rng(3)
    v = rng.standard_normal((8, 8, 8))
    ref = np.fft.fftn(v) / 8 ** 3
    assert np.abs(hamiltonian.direct_dft(v) - ref).max() < 1e-15 * 8 ** 3


def test_direct_dft_recovers_analytic_gaussian_coefficients():
    """The grid potential's DFT equals the analytic Gaussian Fourier coefficients
    (pins the sign of the exponent and the 1/N^3 and 1/Omega factors)."""
    w = synth.tiny_workload(a=6.0, N=12, natoms=2)
    vt = hamiltonian.direct_dft(w.vloc())
    a, N = w.a, w.N
    for n in [(0, 0, 0), (1, 0, 0), (0, -2, 1), (3, 2, -4), (-5, 5, 1)]:
        G = (2 * math.pi / a) * np.array(n, dtype=float)
        want = sum(d * (2 * math.pi * s * s) ** 1.5 / a ** 3 * math.exp(-0.5 * s * s * G @ G)
                   * np.exp(-1j * G @ R) for R, d, s in zip(w.pos, w.depth, w.width))
        got = vt[n[0] % N, n[1] % N, n[2] % N]
        assert abs(got - want) < 1e-13


def test_grid_potential_is_real_and_nyquist_free():
    w = synth.tiny_workload(a=6.0, N=12, natoms=3)
    vh = synth.gaussian_vhat(w.a, w.N, w.pos, w.depth, w.width)
    v = np.fft.ifftn(vh) * w.N ** 3
    assert np.abs(v.imag).max() < 1e-13
    assert np.all(vh[6] == 0) and np.all(vh[:, 6] == 0) and np.all(vh[:, :, 6] == 0)


# ---------------------------------------------------------------- Hamiltonian structure
def test_dense_H_is_hermitian_and_matches_fft_application():
    w = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=(0.25, 0.125, -0.375))
    H = _ham(w)
    Hd = H.dense()
    assert np.abs(Hd - Hd.conj().T).max() < 1e-14
    X = w.x0(H.npw, M=5)
    assert np.abs(Hd @ X - H.apply(X)).max() < 1e-12


def test_free_electron_closed_form():
    """V = 0, no projectors: eigenvalues are exactly the sorted 1/2 |k+G|^2."""
    a, N, k = 7.0, 16, np.array([0.1, 0.2, -0.3])
    miller = basis.sphere(a, N, synth.default_ecut(a, N), k)
    H = hamiltonian.Hamiltonian(a, N, k, miller, np.zeros((N, N, N)))
    ev = np.linalg.eigvalsh(H.dense())
    q = (2 * math.pi / a) * (miller + k)
    want = np.sort(0.5 * (q ** 2).sum(1))
    assert np.abs(ev - want).max() < 1e-12


def test_constant_potential_shifts_spectrum():
    """Adding a constant c to V(r) shifts every eigenvalue by exactly c."""
    w = synth.tiny_workload(a=6.0, N=12, natoms=2)
    H0 = _ham(w)
    H1 = _ham(w, v=w.vloc() + 0.37)
    e0 = np.linalg.eigvalsh(H0.dense())
    e1 = np.linalg.eigvalsh(H1.dense())
    assert np.abs(e1 - e0 - 0.37).max() < 1e-12


def test_translation_invariance():
    """Moving every atom (potential and projectors) by the same vector leaves the spectrum unchanged."""
    w = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=(0.25, 0.0, 0.125))
    e0 = np.linalg.eigvalsh(_ham(w).dense())[:30]
    w2 = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=(0.25, 0.0, 0.125))
    w2.pos = (w2.pos + np.array([1.234, -0.77, 2.5])) % w2.a
    w2._vloc = None
    e1 = np.linalg.eigvalsh(_ham(w2).dense())[:30]
    assert np.abs(e1 - e0).max() < 1e-11


def test_time_reversal():
    """Real V and beta(-q) = +-conj(beta(q)) give eps(k) = eps(-k)."""
    k = (0.375, -0.125, 0.25)
    w = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=k)
    wm = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=tuple(-x for x in k))
    e0 = np.linalg.eigvalsh(_ham(w).dense())[:30]
    e1 = np.linalg.eigvalsh(_ham(wm).dense())[:30]
    assert np.abs(e1 - e0).max() < 1e-11


def test_each_kpoint_of_a_multi_k_cell_has_its_own_hamiltonian():
    """The Hamiltonian of k-point j of a cell with several k-points is the one of the same cell
    with j as its only k-point: sphere, kinetic energies and projectors all follow k_j."""
    import dataclasses
    ks = np.array([[0.25, 0.125, -0.375], [0.0, 0.0, 0.0], [0.5, 0.25, 0.0]])
    w = dataclasses.replace(synth.tiny_workload(a=6.0, N=12, natoms=2), kpts=ks)
    for j in range(len(ks)):
        wj = dataclasses.replace(w, kpts=ks[j:j + 1])
        Hj, H1 = hamiltonian.for_workload(w, j), hamiltonian.for_workload(wj, 0)
        assert Hj.npw == H1.npw
        np.testing.assert_allclose(np.linalg.eigvalsh(Hj.dense()), np.linalg.eigvalsh(H1.dense()),
                                   rtol=0, atol=1e-11)
    e = [np.linalg.eigvalsh(hamiltonian.for_workload(w, j).dense())[:20] for j in range(len(ks))]
    assert np.abs(e[0] - e[1]).max() > 1e-3 and np.abs(e[0] - e[2]).max() > 1e-3


def test_kb_rank_one_secular_equation():
    """V = 0 and one projector of energy E: every eigenvalue below the lowest
    kinetic energy solves 1 = E sum_n |beta(n)|^2 / (eps - T_n)."""
    a, N, k = 6.0, 12, np.array([0.0, 0.0, 0.0])
    miller = basis.sphere(a, N, synth.default_ecut(a, N), k)
    pos = np.array([[1.1, 2.2, 0.7]])
    beta = synth.kb_beta(miller, k, a, pos)[:, :1]
    E = np.array([-0.8])
    H = hamiltonian.Hamiltonian(a, N, k, miller, np.zeros((N, N, N)), beta, E)
    ev = np.linalg.eigvalsh(H.dense())
    T = 0.5 * ((2 * math.pi / a) * miller).astype(float) ** 2
    T = T.sum(1)
    b2 = np.abs(beta[:, 0]) ** 2
    f = lambda e: 1.0 - E[0] * np.sum(b2 / (e - T))
    root = scipy.optimize.brentq(f, -50.0, T.min() - 1e-12, xtol=1e-15)
    assert abs(ev[0] - root) < 1e-11
    # with E = 0 the projector drops out and the free-electron spectrum returns
    H0 = hamiltonian.Hamiltonian(a, N, k, miller, np.zeros((N, N, N)), beta, np.array([0.0]))
    assert np.abs(np.linalg.eigvalsh(H0.dense()) - np.sort(T)).max() < 1e-12


def test_projector_normalisation():
    """The s projector is continuum-normalised: sum |beta_s(q)|^2 -> 1 for a large cutoff."""
    a, N = 8.0, 48
    miller = basis.sphere(a, N, synth.default_ecut(a, N), [0, 0, 0])
    beta = synth.kb_beta(miller, [0, 0, 0], a, np.array([[0.0, 0.0, 0.0]]))
    assert abs(np.sum(np.abs(beta[:, 0]) ** 2) - 1.0) < 1e-3


def test_free_electron_shells_of_the_cubic_lattice():
    """V = 0 in a cell of side 2 pi (reciprocal lattice = integers, Ha units): at Gamma the
    lowest levels are 0, 1/2, 1, 3/2, 2, 5/2 with the numbers of ways to write 0..5 as a sum of
    three squares, 1, 6, 12, 8, 6, 24; at k = (1/2, 0, 0) they are 1/8 (twice) and 5/8 (8 times)."""
    a, N = 2 * math.pi, 16
    H = hamiltonian.Hamiltonian(a, N, np.zeros(3), basis.sphere(a, N, 3.0, np.zeros(3)), np.zeros((N, N, N)))
    ev = np.linalg.eigvalsh(H.dense())
    levels, counts = np.unique(np.round(ev[ev < 2.75], 12), return_counts=True)
    assert np.allclose(levels, [0.0, 0.5, 1.0, 1.5, 2.0, 2.5], atol=1e-12)
    assert list(counts) == [1, 6, 12, 8, 6, 24]
    k = np.array([0.5, 0.0, 0.0])
    H = hamiltonian.Hamiltonian(a, N, k, basis.sphere(a, N, 3.0, k), np.zeros((N, N, N)))
    ev = np.linalg.eigvalsh(H.dense())
    assert np.allclose(ev[:2], 0.125, atol=1e-12) and np.allclose(ev[2:10], 0.625, atol=1e-12)
    assert ev[10] > 0.625 + 0.1
