"""Pins of the oracle parts for the next rows of the hot path: the density from
the bands (SC-loop step 1, Sec. 2.1), the Gamma-point real-wavefunction form,
and the band-by-band PCG the paper compares LOBPCG with (Sec. 3.3).  Closed
forms, invariants and brute force; no GPU."""
import numpy as np
import pytest

import synth
from oracle import basis, density, gamma, hamiltonian, pcg


# ------------------------------------------------------------------ density
def _orthonormal(npw, nb, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((npw, nb)) + 1j * rng.standard_normal((npw, nb)))
    return Q


def _sphere(a=6.0, N=12, kpt=(0.0, 0.0, 0.0)):
    return basis.sphere(a, N, synth.default_ecut(a, N), kpt)


def test_density_fft_route_matches_plain_sum():
    a, N = 5.0, 8
    mil = _sphere(a, N, (0.25, 0.0, -0.125))
    C = _orthonormal(len(mil), 3, 1)
    f = np.array([2.0, 1.5, 0.25])
    r1 = density.density(a, N, mil, C, f)
    r2 = density.density_direct(a, N, mil, C, f)
    assert np.abs(r1 - r2).max() < 1e-14 * np.abs(r2).max() * N ** 3


def test_density_integrates_to_the_occupations():
    """Parseval on the grid: (Omega/N^3) sum_j rho = sum_n f_n for orthonormal bands."""
    a, N = 6.0, 12
    mil = _sphere(a, N)
    C = _orthonormal(len(mil), 5, 2)
    f = np.array([2.0, 2.0, 1.0, 0.5, 0.0])
    rho = density.density(a, N, mil, C, f)
    assert density.electron_count(a, rho) == pytest.approx(f.sum(), rel=1e-13)
    assert rho.min() >= 0.0


def test_density_of_plane_waves_closed_form():
    """One plane wave: rho = f / Omega everywhere.  Two with equal weight:
    rho(r_j) = (1 + cos(2 pi (n1 - n2).j / N)) / Omega."""
    a, N = 6.0, 12
    mil = _sphere(a, N)
    i1 = int(np.flatnonzero((mil == [1, -1, 0]).all(1))[0])
    i2 = int(np.flatnonzero((mil == [0, 2, 1]).all(1))[0])
    c = np.zeros((len(mil), 1), complex)
    c[i1] = 1.0
    rho = density.density(a, N, mil, c, np.array([2.0]))
    assert np.abs(rho - 2.0 / a ** 3).max() < 1e-15
    c[i2] = 1j
    c /= np.sqrt(2.0)
    rho = density.density(a, N, mil, c, np.array([1.0]))
    g = np.arange(N)
    jx, jy, jz = np.meshgrid(g, g, g, indexing="ij")
    dn = np.array([1, -1, 0]) - np.array([0, 2, 1])
    # c(n2) = i c(n1): |e^{i a1} + i e^{i a2}|^2 / 2 = 1 + sin(a1 - a2)
    phase = 2 * np.pi * (dn[0] * jx + dn[1] * jy + dn[2] * jz) / N
    assert np.abs(rho - (1.0 + np.sin(phase)) / a ** 3).max() < 1e-14


def test_density_translation_and_rotation_invariance():
    """Multiplying c(G) by exp(-2 pi i n.t/N) moves the density by the grid vector t;
    a unitary mixing of equally occupied bands leaves it unchanged."""
    a, N = 6.0, 12
    mil = _sphere(a, N, (0.125, 0.25, 0.0))
    C = _orthonormal(len(mil), 4, 3)
    f = np.full(4, 2.0)
    rho = density.density(a, N, mil, C, f)
    t = np.array([3, -2, 5])
    Ct = C * np.exp(-2j * np.pi * (mil @ t) / N)[:, None]
    rho_t = density.density(a, N, mil, Ct, f)
    assert np.abs(rho_t - np.roll(rho, shift=tuple(t), axis=(0, 1, 2))).max() < 1e-14
    U = _orthonormal(4, 4, 4)
    assert np.abs(density.density(a, N, mil, C @ U, f) - rho).max() < 1e-14


# ------------------------------------------------------------------ Gamma-point real form
def _gamma_H(kb=True, seed=11):
    w = synth.tiny_workload(a=6.0, N=12, natoms=2, kb=kb, kpt=(0.0, 0.0, 0.0), seed=seed)
    return w, hamiltonian.for_workload(w)


def test_half_set_pairs_every_plane_wave_once():
    mil = _sphere()
    zero, plus, minus = gamma.half_set(mil)
    assert (mil[zero] == 0).all()
    assert np.array_equal(mil[minus], -mil[plus])
    allidx = np.sort(np.concatenate([[zero], plus, minus]))
    assert np.array_equal(allidx, np.arange(len(mil)))
    with pytest.raises(ValueError):
        gamma.half_set(_sphere(kpt=(0.25, 0.0, 0.0)))


def test_real_basis_is_unitary_and_gives_real_orbitals():
    a, N = 6.0, 12
    mil = _sphere(a, N)
    U = gamma.real_basis(mil)
    assert np.abs(U.conj().T @ U - np.eye(len(mil))).max() < 1e-15
    x = np.random.default_rng(5).standard_normal((len(mil), 3))
    c = gamma.to_sphere(mil, x)
    box = np.zeros((N, N, N, 3), complex)
    box[basis.box_index(mil, N)] = c
    psi = np.fft.ifftn(box, axes=(0, 1, 2))
    assert np.abs(psi.imag).max() < 1e-15 * np.abs(psi.real).max() * N ** 3


def test_real_form_of_H_is_real_with_the_same_spectrum():
    """At Gamma (real V, KB projectors real in r space) U^H H U is real symmetric and
    has the spectrum of the complex H."""
    _, H = _gamma_H()
    Hc = H.dense()
    Hr = gamma.RealHamiltonian(H).dense()
    scale = np.abs(Hc).max()
    assert np.abs(Hr.imag).max() < 1e-14 * scale
    assert np.abs(Hr.real - Hr.real.T).max() < 1e-14 * scale
    assert np.abs(np.linalg.eigvalsh(Hr.real) - np.linalg.eigvalsh(Hc)).max() < 1e-12 * scale


def test_real_basis_kinetic_energies_are_those_of_the_plane_waves():
    """u_G and v_G combine e_G and e_-G, which have the same kinetic energy at Gamma, so the
    kinetic diagonal in the real basis is the plane waves' 1/2 |G|^2, each value once per
    plane wave (the preconditioner of the real-form solve is built on it)."""
    _, H = _gamma_H()
    RH = gamma.RealHamiltonian(H)
    np.testing.assert_allclose(np.sort(RH.T), np.sort(H.T), rtol=1e-14, atol=1e-14)


def test_half_storage_inner_products_and_round_trip():
    mil = _sphere()
    rng = np.random.default_rng(6)
    A = gamma.to_sphere(mil, rng.standard_normal((len(mil), 3)))
    B = gamma.to_sphere(mil, rng.standard_normal((len(mil), 4)))
    hA, hB = gamma.to_half(mil, A), gamma.to_half(mil, B)
    assert hA.shape[0] == (len(mil) + 1) // 2
    assert np.abs(gamma.half_inner(hA, hB) - (A.conj().T @ B)).max() < 1e-13
    assert np.abs(gamma.from_half(mil, hA) - A).max() == 0.0


def test_real_H_application_keeps_orbitals_real():
    _, H = _gamma_H()
    rH = gamma.RealHamiltonian(H)
    x = np.random.default_rng(7).standard_normal((H.npw, 2))
    y_full = H.apply(rH.U @ x)
    # H maps real orbitals to real orbitals: c(-G) = conj(c(G)) holds for H psi
    zero, plus, minus = gamma.half_set(H.miller)
    assert np.abs(y_full[minus] - np.conj(y_full[plus])).max() < 1e-12 * np.abs(y_full).max()
    assert np.abs(y_full[zero].imag).max() < 1e-12 * np.abs(y_full).max()
    assert np.abs(rH.U @ rH.apply(x) - y_full).max() < 1e-12 * np.abs(y_full).max()


def test_real_mode_lobpcg_matches_complex_dense():
    w, H = _gamma_H()
    ref = np.linalg.eigvalsh(H.dense())[:8]
    x0 = np.random.default_rng(8).standard_normal((H.npw, 8))
    r = gamma.solve_real(H, x0, block=4, nline=4, tol=1e-10)
    assert r.converged and r.X.dtype == np.float64
    assert np.abs(r.eig - ref).max() < 1e-10
    c = gamma.to_sphere(H.miller, r.X)
    assert np.abs(H.apply(c) - c * r.eig[None, :]).max() < 1e-9


def test_real_form_rejects_a_general_k_point():
    w = synth.tiny_workload(a=6.0, N=12, natoms=1, kpt=(0.25, 0.0, 0.0))
    with pytest.raises(ValueError):
        gamma.RealHamiltonian(hamiltonian.for_workload(w))


# ------------------------------------------------------------------ band-by-band PCG
def test_line_minimum_against_brute_force():
    rng = np.random.default_rng(9)
    th = np.linspace(-np.pi / 2, np.pi / 2, 200001)
    for _ in range(20):
        A, B, C = rng.standard_normal(3) * 3
        theta, e = pcg.line_minimum(A, B, C)
        E = A * np.cos(th) ** 2 + B * np.sin(th) ** 2 + 2 * C * np.sin(th) * np.cos(th)
        assert e == pytest.approx(E.min(), abs=1e-9)
        assert -np.pi / 2 < theta <= np.pi / 2
    # a diagonal pencil already at its minimum does not move
    assert pcg.line_minimum(-1.0, 2.0, 0.0) == (0.0, -1.0)


class _Dense:
    def __init__(self, H, T):
        self.Hm, self.T = H, T

    def apply(self, X):
        return self.Hm @ X


def test_pcg_two_plane_waves_one_iteration_is_exact():
    """npw = 2: span[x, d] is the whole space, so one iteration (with a flat
    preconditioner) reaches the lowest eigenvalue (a+b)/2 - sqrt(((a-b)/2)^2 + |c|^2)."""
    a, b, c = 0.7, -0.4, 0.3 - 0.5j
    Hm = np.array([[a, c], [np.conj(c), b]])
    op = _Dense(Hm, np.array([1.0, 1.0]))
    x, eps = pcg.band_pcg(op, np.array([1.0, 0.2j]), op.T, None, nline=1)
    exact = (a + b) / 2 - np.sqrt(((a - b) / 2) ** 2 + abs(c) ** 2)
    assert eps == pytest.approx(exact, abs=1e-15)
    assert np.linalg.norm(Hm @ x - eps * x) < 1e-14


def test_pcg_rayleigh_quotient_never_increases_and_keeps_the_constraint():
    w, H = _gamma_H()
    X0 = w.x0(H.npw, M=4)
    Y, _ = np.linalg.qr(X0[:, :2])
    trace = []
    x, _ = pcg.band_pcg(H, X0[:, 2], H.T, Y, nline=6, trace=trace)
    assert all(t1 <= t0 + 1e-12 for t0, t1 in zip(trace[:-1], trace[1:]))
    assert np.abs(Y.conj().T @ x).max() < 1e-13
    assert np.linalg.norm(x) == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("kpt", [(0.0, 0.0, 0.0), (0.25, 0.125, -0.375)])
def test_pcg_matches_dense(kpt):
    w = synth.tiny_workload(a=6.0, N=12, natoms=2, kpt=kpt, seed=11)
    H = hamiltonian.for_workload(w)
    ref = np.linalg.eigvalsh(H.dense())[:6]
    r = pcg.solve_pcg(H, w.x0(H.npw, M=6), nline=4, tol=1e-10)
    assert r.converged
    assert np.abs(r.eig - ref).max() < 1e-10


def test_pcg_free_electrons_closed_form():
    a, N = 6.0, 12
    k = np.zeros(3)
    mil = basis.sphere(a, N, synth.default_ecut(a, N), k)
    H = hamiltonian.Hamiltonian(a, N, k, mil, np.zeros((N, N, N)))
    r = pcg.solve_pcg(H, synth.start_vectors(5, H.npw, 7), nline=4, tol=1e-10)
    assert r.converged
    assert np.abs(r.eig - np.sort(H.T)[:7]).max() < 1e-10
