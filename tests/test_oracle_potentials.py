"""Pins of the oracle's electrostatics and projectors against closed forms (CPU only)."""
import math

import numpy as np
import pytest
from scipy import integrate as sint
from scipy.special import erf, erfc

from oracle import basis, potentials

# Madelung constant of the simple-cubic lattice of charges in a neutralising background,
# E = -ALPHA_SC Q^2 / (2 L) per cell, and of rock salt per ion pair (nearest neighbour d).
ALPHA_SC = 2.8372974794806
ALPHA_NACL = 1.747564594633


def _gauss_density(lat, grid, centre, Q, alpha):
    """Periodic sum of Q (alpha/pi)^{3/2} exp(-alpha r^2) sampled on the grid."""
    r = basis.grid_points(lat, grid)
    out = np.zeros(grid)
    A = np.asarray(lat)
    for n1 in (-1, 0, 1):
        for n2 in (-1, 0, 1):
            for n3 in (-1, 0, 1):
                d = r - (centre + n1 * A[0] + n2 * A[1] + n3 * A[2])
                out += Q * (alpha / math.pi) ** 1.5 * np.exp(-alpha * np.sum(d * d, axis=-1))
    return out


def test_hartree_gaussian_closed_form():
    L, alpha, Q = 10.0, 1.5, 1.0
    lat = np.diag([L] * 3)
    rho = _gauss_density(lat, (48, 48, 48), np.array([3.1, 4.7, 6.2]), Q, alpha)
    _, EH = potentials.hartree(rho, lat)
    omega = L ** 3
    want = Q * Q * math.sqrt(alpha / (2 * math.pi)) - Q * Q * ALPHA_SC / (2 * L) \
        + math.pi * Q * Q / (alpha * omega)
    assert abs(EH - want) < 1e-10


def test_hartree_potential_solves_poisson():
    """-lap v_H = 4 pi (rho - mean rho) checked through second differences' FFT
    eigenvalues is circular; instead: v_H of a single cosine density is analytic."""
    lat = np.diag([6.0, 7.0, 8.0])
    grid = (12, 14, 16)
    r = basis.grid_points(lat, grid)
    G = 2 * math.pi * np.array([1 / 6.0, 2 / 7.0, 0.0])
    rho = 0.3 + 0.1 * np.cos(r @ G)
    v, _ = potentials.hartree(rho, lat)
    assert np.allclose(v, 4 * math.pi * 0.1 * np.cos(r @ G) / (G @ G), atol=1e-13)


def test_local_potential_gaussian_charge_closed_form():
    """int rho_e v_loc for an electron Gaussian centred on the ion (generic point, so the
    structure-factor phase sign matters): -QZ [2/(sqrt(pi) s) - a/L + pi s^2/Omega]
    + Q pi Z r_c^2/Omega with s^2 = sigma_e^2 + r_c^2 (Gaussians exp(-r^2/sigma^2))."""
    L, Z, rc, Q, alpha = 12.0, 2.0, 0.5, 1.0, 2.0
    lat = np.diag([L] * 3)
    grid = (60, 60, 60)
    R = np.array([3.1, 4.7, 6.2])
    rho = _gauss_density(lat, grid, R, Q, alpha)
    v = potentials.vloc_r(lat, grid, [R], [Z], rc)
    E = float(basis.integrate(v * rho, lat))
    s2 = 1.0 / alpha + rc * rc
    s = math.sqrt(s2)
    omega = L ** 3
    want = -Q * Z * (2.0 / (math.sqrt(math.pi) * s) - ALPHA_SC / L + math.pi * s2 / omega) \
        + Q * math.pi * Z * rc * rc / omega
    assert abs(E - want) < 1e-9


def test_local_potential_radial_transform():
    """The short-range part Z erfc(r/r_c)/r of -Z erf(r/r_c)/r + Z/r transforms to
    4 pi Z (1 - exp(-q^2 r_c^2/4))/q^2, and its q -> 0 limit is pi Z r_c^2 (the G = 0 term)."""
    Z, rc = 3.0, 0.5
    for q in (0.0, 0.7, 2.3, 5.0):
        if q == 0.0:
            val = sint.quad(lambda r: 4 * math.pi * r * r * Z * erfc(r / rc) / r, 0, 20)[0]
            want = math.pi * Z * rc * rc
        else:
            val = sint.quad(lambda r: 4 * math.pi * r * r * Z * erfc(r / rc) / r
                            * math.sin(q * r) / (q * r), 0, 20, limit=200)[0]
            want = 4 * math.pi * Z * (1 - math.exp(-q * q * rc * rc / 4)) / (q * q)
        assert abs(val - want) < 1e-9
    lat = np.diag([5.0] * 3)
    vG = potentials.vloc_G(lat, (8, 8, 8), [[0.0, 0.0, 0.0]], [Z], rc)
    assert np.isclose(vG[0, 0, 0].real, math.pi * Z * rc * rc / 125.0)
    g = 2 * math.pi / 5.0
    assert np.isclose(vG[1, 0, 0].real, -4 * math.pi * Z / (g * g) * math.exp(-g * g * rc * rc / 4) / 125.0)


def test_local_potential_real_space_shape():
    """Away from the ion, v_loc differences follow -Z erf(r/r_c)/r (differences remove the
    periodic constant; the images contribute smooth terms that cancel to 1e-3 at L=24)."""
    L, Z, rc = 24.0, 1.0, 0.5
    lat = np.diag([L] * 3)
    grid = (96, 96, 96)
    v = potentials.vloc_r(lat, grid, [[0.0, 0.0, 0.0]], [Z], rc)
    h = L / 96
    r1, r2 = 2 * h, 8 * h
    dv = v[8, 0, 0] - v[2, 0, 0]
    want = -Z * erf(r2 / rc) / r2 + Z * erf(r1 / rc) / r1
    # the neutralising background adds -Z (2 pi / 3 Omega) r^2 to the ion's potential
    want += -Z * 2 * math.pi / (3 * L ** 3) * (r2 * r2 - r1 * r1)
    assert abs(dv - want) < 2e-5


def test_ewald_simple_cubic_madelung():
    for L in (5.0, 7.3):
        E = potentials.ewald(np.diag([L] * 3), [[0.3, 0.2, 0.1]], [2.0])
        assert abs(E - (-4.0 * ALPHA_SC / (2 * L))) < 1e-11


def test_ewald_rock_salt_madelung():
    a = 6.0
    pos, Z = [], []
    for f in [(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)]:
        pos.append(np.array(f) * a)
        Z.append(1.0)
        pos.append((np.array(f) + [0.5, 0, 0]) * a)
        Z.append(-1.0)
    E = potentials.ewald(np.diag([a] * 3), pos, Z)
    assert abs(E - (-4 * ALPHA_NACL / (a / 2))) < 1e-10


def test_ewald_independent_of_splitting():
    lat = np.array([[7.0, 0.0, 0.0], [1.0, 8.0, 0.0], [0.5, 0.5, 9.0]])
    pos = [[0.1, 0.2, 0.3], [3.0, 4.1, 2.2], [5.5, 1.0, 7.0]]
    Z = [2.0, 3.0, 1.0]
    e1 = potentials.ewald(lat, pos, Z, eta=0.3)
    e2 = potentials.ewald(lat, pos, Z, eta=0.9)
    assert abs(e1 - e2) < 1e-10


def test_kb_projector_is_transform_of_unit_gaussian():
    """|<k+G|beta>|^2 summed over a complete-enough sphere equals the projector norm 1
    (Parseval for a unit-norm Gaussian), and the phase follows the atom position."""
    L = 9.0
    lat = np.diag([L] * 3)
    mil, _ = basis.sphere(lat, (64, 64, 64), (0.1, 0.2, 0.3), 60.0)
    for s in (0.5, 1.0):
        beta = potentials.kb_projectors(lat, (0.1, 0.2, 0.3), mil, [[1.0, 2.0, 3.0]], [s])
        assert np.isclose(np.sum(np.abs(beta) ** 2), 1.0, rtol=1e-10)
    # real-space check: sum_G beta(G) e^{i(k+G).r} / sqrt(Omega) at the atom centre
    beta = potentials.kb_projectors(lat, (0, 0, 0), mil, [[0.0, 0.0, 0.0]], [1.0])
    val = np.sum(beta) / math.sqrt(L ** 3)
    assert np.isclose(val.real, (math.pi ** 1.5) ** -0.5, rtol=1e-8)
