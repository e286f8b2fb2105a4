"""Seeded synthetic inputs for the plane-wave LOBPCG eigensolver.

This module only *generates inputs*: cells, atom sites, a Gaussian local
potential sampled on the real-space grid, Kleinman-Bylander projector
coefficients evaluated at given Miller indices, KB energies, k-points and
random start vectors.  It holds none of the eigensolver's or the
Hamiltonian-application arithmetic, so that the CPU oracle (``oracle/``) and
the GPU library can both take their inputs from here without sharing any
method code.

The paper (Sec. 5) benchmarks fcc gold with 108 atoms, 648 bands and a 108^3
grid, and a 10 k-point variant; the pseudopotential data those systems need is
not available, so seeded synthetic cells of the same shape stand in for them:

* local potential: a sum of Gaussians ``d exp(-|r-R|^2/(2 w^2))`` with
  ``d ~ U(-3,-1)`` Ha and ``w ~ U(0.8,1.2)`` bohr, given by its analytic
  Fourier coefficients with the Nyquist planes set to zero, sampled on the
  grid ``r_j = a j / N`` (so the grid potential is real and band-limited);
* KB projectors: per atom one s and three p Gaussian projectors of radius
  ``r_p = 1`` bohr, continuum normalised, with energies ``E ~ U(-1,1)`` Ha
  (one for s, one shared by the three p);
* atom sites: jittered fcc (or rock-salt) lattices, jitter ``+-0.05 a/n_c``;
* k-points in reduced coordinates.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "default_ecut",
    "fcc_sites",
    "rocksalt_sites",
    "gaussian_vhat",
    "vloc_grid",
    "kb_beta",
    "start_vectors",
    "make_workload",
    "tiny_workload",
]


def default_ecut(a: float, N: int) -> float:
    """Cutoff whose sphere radius is a quarter of the FFT box edge.

    ``Ecut = 1/2 (pi N / (2 a))^2`` Ha, i.e. ``|G| <= (2 pi / a)(N/4)``; the
    zero-padded FFT then needs no aliasing guard (Sec. 5.1 notes the same
    half-box rule for the number of FFT planes).
    """
    return 0.5 * (math.pi * N / (2.0 * a)) ** 2


def fcc_sites(n_c: int, a: float) -> np.ndarray:
    """Sites of ``n_c^3`` conventional fcc cells filling a cube of side ``a``."""
    basis = np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])
    cells = np.array([[i, j, k] for i in range(n_c) for j in range(n_c) for k in range(n_c)], dtype=float)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    return sites * (a / n_c)


def rocksalt_sites(n_c: int, a: float) -> np.ndarray:
    """Two interpenetrating fcc lattices shifted by half a conventional cell."""
    s = fcc_sites(n_c, a)
    return np.concatenate([s, s + np.array([0.5, 0.0, 0.0]) * (a / n_c)], axis=0)


def _box_index(N: int) -> np.ndarray:
    """Signed frequency of each box index: 0..N/2-1, -N/2..-1."""
    n = np.arange(N)
    return np.where(n < N // 2, n, n - N)


def gaussian_vhat(a: float, N: int, pos: np.ndarray, depth: np.ndarray, width: np.ndarray) -> np.ndarray:
    """Analytic Fourier coefficients of the Gaussian local potential.

    ``Vhat(n) = sum_a d_a (2 pi w_a^2)^{3/2} / Omega exp(-w_a^2 |G_n|^2 / 2) exp(-i G_n.R_a)``
    on the N^3 box (index ``n mod N``), with every plane that contains a
    Nyquist index (``n_d = -N/2``) set to zero.
    """
    omega = a ** 3
    g = (2.0 * math.pi / a) * _box_index(N).astype(np.float64)
    vhat = np.zeros((N, N, N), dtype=np.complex128)
    for R, d, w in zip(pos, depth, width):
        pref = d * (2.0 * math.pi * w * w) ** 1.5 / omega
        fx = np.exp(-0.5 * w * w * g * g - 1j * g * R[0])
        fy = np.exp(-0.5 * w * w * g * g - 1j * g * R[1])
        fz = np.exp(-0.5 * w * w * g * g - 1j * g * R[2])
        vhat += pref * (fx[:, None, None] * fy[None, :, None]) * fz[None, None, :]
    if N % 2 == 0:
        h = N // 2
        vhat[h, :, :] = 0.0
        vhat[:, h, :] = 0.0
        vhat[:, :, h] = 0.0
    return vhat


def vloc_grid(vhat: np.ndarray) -> np.ndarray:
    """Real-space samples ``V(r_j) = sum_n Vhat(n) exp(2 pi i n.j/N)``, C-order [x][y][z]."""
    N = vhat.shape[0]
    v = np.fft.ifftn(vhat) * (N ** 3)
    return np.ascontiguousarray(v.real)


def kb_beta(miller: np.ndarray, kpt, a: float, pos: np.ndarray, rp: float = 1.0) -> np.ndarray:
    """KB projector coefficients at the plane waves ``q = 2 pi/a (n + k)``.

    Per atom (in order): ``beta_s(q) = c exp(-|q|^2 rp^2/2) exp(-i q.R)`` and
    ``beta_p_alpha(q) = c sqrt(2) rp q_alpha exp(-|q|^2 rp^2/2) exp(-i q.R)``
    for alpha = x, y, z, with ``c = (4 pi rp^2)^{3/4} / sqrt(Omega)``.

    Returns a complex128 array of shape (npw, 4 * natoms).
    """
    miller = np.asarray(miller, dtype=np.float64)
    q = (2.0 * math.pi / a) * (miller + np.asarray(kpt, dtype=np.float64)[None, :])
    omega = a ** 3
    c = (4.0 * math.pi * rp * rp) ** 0.75 / math.sqrt(omega)
    q2 = np.einsum("ij,ij->i", q, q)
    radial = c * np.exp(-0.5 * q2 * rp * rp)
    nat = len(pos)
    out = np.empty((q.shape[0], 4 * nat), dtype=np.complex128)
    for ia, R in enumerate(pos):
        ph = radial * np.exp(-1j * (q @ np.asarray(R, dtype=np.float64)))
        out[:, 4 * ia] = ph
        out[:, 4 * ia + 1] = math.sqrt(2.0) * rp * q[:, 0] * ph
        out[:, 4 * ia + 2] = math.sqrt(2.0) * rp * q[:, 1] * ph
        out[:, 4 * ia + 3] = math.sqrt(2.0) * rp * q[:, 2] * ph
    return out


def start_vectors(seed: int, npw: int, M: int, k_index: int = 0) -> np.ndarray:
    """Random complex normal start block ``(N(0,1) + i N(0,1))/sqrt(2)``, shape (npw, M)."""
    rng = np.random.default_rng([seed, 7, k_index])
    x = rng.standard_normal((npw, M)) + 1j * rng.standard_normal((npw, M))
    return x / math.sqrt(2.0)


@dataclass
class Workload:
    """A synthetic cell: everything both solvers need, in neutral form."""

    name: str
    a: float
    N: int
    ecut: float
    kpts: np.ndarray                 # (nk, 3) reduced coordinates
    pos: np.ndarray                  # (natoms, 3) bohr
    depth: np.ndarray                # (natoms,) Ha
    width: np.ndarray                # (natoms,) bohr
    proj_E: np.ndarray               # (nproj,) Ha; empty when there is no KB part
    nbands: int
    block: int
    nline: int = 4
    seed: int = 0
    kb: bool = True
    _vloc: np.ndarray | None = field(default=None, repr=False)

    @property
    def nk(self) -> int:
        return int(self.kpts.shape[0])

    @property
    def nproj(self) -> int:
        return int(self.proj_E.shape[0])

    def vloc(self) -> np.ndarray:
        """The real grid potential V(r_j), float64 [x][y][z]."""
        if self._vloc is None:
            self._vloc = vloc_grid(gaussian_vhat(self.a, self.N, self.pos, self.depth, self.width))
        return self._vloc

    def beta(self, miller: np.ndarray, k_index: int) -> np.ndarray:
        """Projectors (npw, nproj) at the given Miller indices of k-point ``k_index``."""
        if self.nproj == 0:
            return np.zeros((len(miller), 0), dtype=np.complex128)
        return kb_beta(miller, self.kpts[k_index], self.a, self.pos)

    def x0(self, npw: int, k_index: int = 0, M: int | None = None) -> np.ndarray:
        return start_vectors(self.seed, npw, self.nbands if M is None else M, k_index)


def _jitter(rng, sites, a, n_c):
    return (sites + rng.uniform(-0.05, 0.05, size=sites.shape) * (a / n_c)) % a


def _species(rng, nat, kb):
    depth = rng.uniform(-3.0, -1.0, size=nat)
    width = rng.uniform(0.8, 1.2, size=nat)
    if kb:
        es = rng.uniform(-1.0, 1.0, size=nat)
        ep = rng.uniform(-1.0, 1.0, size=nat)
        E = np.stack([es, ep, ep, ep], axis=1).reshape(-1)
    else:
        E = np.zeros(0)
    return depth, width, E


# Workload recipes (seed = 1000 + index, numpy default_rng):
#   gamma24     a=10 N=24  Gamma,      4 random atoms, local only,   M=16   m=16
#   k96         a=20 N=96  k=(1/4)^3, 64 rock-salt atoms + 256 KB,   M=256  m=64
#   gamma120    a=25 N=120 Gamma,    108 fcc atoms + 432 KB,         M=1024 m=128
#   mp72x10     a=16 N=72  10 MP k,   32 fcc atoms + 128 KB,         M=128  m=64 per k
#   large160    a=32 N=160 Gamma+(1/4)^3, 256 fcc atoms + 1024 KB,   M=2048 m=256 per k
WORKLOADS = ("gamma24", "k96", "gamma120", "mp72x10", "large160")


def make_workload(name: str) -> Workload:
    """Build one of the named synthetic cells (see ``WORKLOADS``)."""
    idx = WORKLOADS.index(name) + 1
    seed = 1000 + idx
    rng = np.random.default_rng(seed)
    if name == "gamma24":
        a, N = 10.0, 24
        pos = rng.uniform(0.0, a, size=(4, 3))
        depth, width, E = _species(rng, 4, kb=False)
        return Workload(name, a, N, default_ecut(a, N), np.zeros((1, 3)), pos, depth, width, E, 16, 16, seed=seed, kb=False)
    if name == "k96":
        a, N, n_c = 20.0, 96, 2
        pos = _jitter(rng, rocksalt_sites(n_c, a), a, n_c)
        depth, width, E = _species(rng, len(pos), kb=True)
        return Workload(name, a, N, default_ecut(a, N), np.full((1, 3), 0.25), pos, depth, width, E, 256, 64, seed=seed)
    if name == "gamma120":
        a, N, n_c = 25.0, 120, 3
        pos = _jitter(rng, fcc_sites(n_c, a), a, n_c)
        depth, width, E = _species(rng, len(pos), kb=True)
        return Workload(name, a, N, default_ecut(a, N), np.zeros((1, 3)), pos, depth, width, E, 1024, 128, seed=seed)
    if name == "mp72x10":
        a, N, n_c = 16.0, 72, 2
        pos = _jitter(rng, fcc_sites(n_c, a), a, n_c)
        depth, width, E = _species(rng, len(pos), kb=True)
        grid = np.array([(2 * r - 5) / 8.0 for r in range(1, 5)])
        mp = np.array([[x, y, z] for x in grid for y in grid for z in grid])
        pick = rng.choice(len(mp), size=10, replace=False)
        return Workload(name, a, N, default_ecut(a, N), mp[pick], pos, depth, width, E, 128, 64, seed=seed)
    if name == "large160":
        a, N, n_c = 32.0, 160, 4
        pos = _jitter(rng, fcc_sites(n_c, a), a, n_c)
        depth, width, E = _species(rng, len(pos), kb=True)
        kp = np.array([[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]])
        return Workload(name, a, N, default_ecut(a, N), kp, pos, depth, width, E, 2048, 256, seed=seed)
    raise KeyError(name)


def tiny_workload(a: float = 6.0, N: int = 12, natoms: int = 2, kb: bool = True, kpt=(0.0, 0.0, 0.0),
                  nbands: int = 8, block: int = 4, seed: int = 7, ecut: float | None = None) -> Workload:
    """A small random cell for unit tests (same recipe, free sizes)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, a, size=(natoms, 3))
    depth, width, E = _species(rng, natoms, kb=kb)
    return Workload(f"tiny_a{a:g}_N{N}", a, N, default_ecut(a, N) if ecut is None else ecut,
                    np.asarray([kpt], dtype=float), pos, depth, width, E, nbands, block, seed=seed, kb=kb)
