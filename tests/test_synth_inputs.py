"""The seeded synthetic inputs both sides take: reproducible, shaped as stated, and physical
(a real, Nyquist-free grid potential; KB projectors of the stated count; start blocks that
differ between k-points and are reproducible per seed)."""
import numpy as np
import pytest

import synth

SHAPES = {  # atoms, projectors, nk, bands, block
    "gamma24": (4, 0, 1, 16, 16),
    "k96": (64, 256, 1, 256, 64),
    "gamma120": (108, 432, 1, 1024, 128),
    "mp72x10": (32, 128, 10, 128, 64),
    "large160": (256, 1024, 2, 2048, 256),
}


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_workload_shapes(name):
    w = synth.make_workload(name)
    nat, nproj, nk, nb, m = SHAPES[name]
    assert (len(w.pos), w.nproj, w.nk, w.nbands, w.block) == (nat, nproj, nk, nb, m)
    assert np.all((w.pos >= 0) & (w.pos < w.a))
    assert np.all((w.depth >= -3) & (w.depth <= -1)) and np.all((w.width >= 0.8) & (w.width <= 1.2))
    if nproj:
        assert np.all(np.abs(w.proj_E) <= 1.0)


def test_workloads_are_reproducible_and_seeded_apart():
    a, b = synth.make_workload("gamma24"), synth.make_workload("gamma24")
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vloc(), b.vloc())
    assert np.array_equal(a.x0(500), b.x0(500))
    k = synth.make_workload("mp72x10")
    assert not np.array_equal(k.x0(100, 0, 4), k.x0(100, 1, 4))
    assert not np.array_equal(a.x0(100, 0, 4), k.x0(100, 0, 4))


def test_grid_potential_is_real_band_limited_and_attractive():
    w = synth.make_workload("gamma24")
    v = w.vloc()
    assert v.dtype == np.float64 and v.shape == (24, 24, 24)
    vh = np.fft.fftn(v) / v.size
    N = 24
    assert np.abs(vh[N // 2, :, :]).max() < 1e-14 * np.abs(vh).max()   # Nyquist planes zero
    assert np.abs(vh[:, N // 2, :]).max() < 1e-14 * np.abs(vh).max()
    assert np.abs(vh[:, :, N // 2]).max() < 1e-14 * np.abs(vh).max()
    assert vh[0, 0, 0].real < 0.0   # Gaussian wells: negative average


def test_start_vectors_statistics():
    x = synth.start_vectors(3, 20000, 4)
    assert x.dtype == np.complex128
    assert abs(np.mean(np.abs(x) ** 2) - 1.0) < 0.02
    assert abs(np.mean(x.real * x.imag)) < 0.02
