"""Pins of the oracle's grid, sphere and Fourier conventions (CPU only)."""
import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 10, 15), (8, 9, 5)])
def test_fft_matches_direct_dft(shape):
    rng = np.random.default_rng(3)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    inv = basis.dft_direct(f, +1)
    fwd = basis.dft_direct(f, -1) / np.prod(shape)
    assert np.allclose(basis.r_from_G(f), inv, rtol=0, atol=1e-12 * np.abs(inv).max())
    assert np.allclose(basis.G_from_r(f), fwd, rtol=0, atol=1e-12 * np.abs(fwd).max())


def test_round_trip_and_parseval():
    rng = np.random.default_rng(4)
    f = rng.standard_normal((12, 10, 9))
    g = basis.G_from_r(f)
    assert np.allclose(np.real(basis.r_from_G(g)), f, atol=1e-13)
    # (1/N) sum |f(r)|^2 = sum |f(G)|^2
    assert np.isclose(np.mean(f * f), np.sum(np.abs(g) ** 2), rtol=1e-13)


def test_plane_wave_grid_values():
    """A single coefficient at Miller m gives e^{iG.r} on the grid points."""
    lat = np.diag([3.0, 4.0, 5.0]) + np.array([[0, 0, 0], [0.5, 0, 0], [0, 0.3, 0]])
    grid = (6, 8, 10)
    m = np.array([[1, -2, 3]])
    u = basis.r_from_G(basis.to_grid(np.array([1.0]), m, grid))
    B = basis.reciprocal(lat)
    G = m[0] @ B
    r = basis.grid_points(lat, grid)
    assert np.allclose(u, np.exp(1j * r @ G), atol=1e-12)


def test_reciprocal_lattice():
    lat = np.array([[4.0, 0.2, 0.0], [0.1, 5.0, 0.3], [0.0, 0.4, 6.0]])
    B = basis.reciprocal(lat)
    assert np.allclose(lat @ B.T, 2 * np.pi * np.eye(3), atol=1e-13)


def test_axis_miller_and_nyquist():
    assert list(basis.axis_miller(6)) == [0, 1, 2, -3, -2, -1]
    assert list(basis.axis_miller(5)) == [0, 1, 2, -2, -1]
    mask = basis.nyquist_mask((4, 5, 6))
    assert mask[2].all() and mask[:, :, 3].all()
    assert mask.sum() == 5 * 6 + 4 * 5 - 5


@pytest.mark.parametrize("kfrac", [(0, 0, 0), (0.25, -0.25, 0.0), (0.1, 0.3, -0.2)])
def test_sphere_brute_force(kfrac):
    """Sphere equals brute-force enumeration over a much larger box, sorted order."""
    lat = np.diag([8.0, 9.0, 14.0])
    ecut = 5.0
    mil, kin = basis.sphere(lat, (24, 24, 40), kfrac, ecut)
    B = basis.reciprocal(lat)
    k = np.asarray(kfrac, dtype=np.float64) @ B
    want = []
    for a in range(-12, 13):
        for b in range(-12, 13):
            for c in range(-20, 21):
                q = k + a * B[0] + b * B[1] + c * B[2]
                if 0.5 * float(q @ q) <= ecut:
                    want.append((a, b, c))
    assert [tuple(x) for x in mil] == sorted(want)
    assert np.all(kin <= ecut)
    assert np.allclose(kin, 0.5 * np.sum((k + mil @ B) ** 2, axis=1), rtol=1e-14)


def test_gamma_sphere_inversion_symmetric():
    mil, _ = basis.sphere(np.diag([10.0] * 3), (32, 32, 32), (0, 0, 0), 15.0)
    s = {tuple(x) for x in mil}
    assert all((-a, -b, -c) in s for a, b, c in s)
    assert mil.shape[0] == 2777


def test_integrate_constant():
    lat = np.diag([3.0, 4.0, 5.0])
    assert np.isclose(basis.integrate(np.full((5, 6, 7), 2.0), lat), 120.0)
