"""Pins of the oracle's density functionals and potentials (CPU only)."""
import math

import numpy as np
import pytest

from oracle import basis, functionals as fn

LAT = np.diag([7.0, 8.0, 9.0])
GRID = (28, 32, 36)


def _smooth_density(scale=1.0):
    """Two Gaussian lumps on a small uniform background: smooth and band-limited enough
    for FFT derivatives to be accurate."""
    r = basis.grid_points(LAT, GRID)
    rho = np.full(GRID, 0.01 * scale)
    A = np.asarray(LAT)
    for c, a, q in (((2.0, 3.0, 4.0), 1.2, 2.0), ((4.5, 5.0, 5.5), 0.8, 1.0)):
        for n1 in (-1, 0, 1):
            for n2 in (-1, 0, 1):
                for n3 in (-1, 0, 1):
                    d = r - (np.array(c) + n1 * A[0] + n2 * A[1] + n3 * A[2])
                    rho += scale * q * (a / math.pi) ** 1.5 * np.exp(-a * np.sum(d * d, -1))
    return rho


def _smooth_perturbation():
    r = basis.grid_points(LAT, GRID)
    G1 = 2 * math.pi * np.array([1 / 7.0, 0, 0])
    G2 = 2 * math.pi * np.array([0, 1 / 8.0, 2 / 9.0])
    return 0.002 * (np.cos(r @ G1 + 0.3) + np.sin(r @ G2))


def test_slater_exchange_constant():
    """eps_x = -(3/4)(9/(4 pi^2))^{1/3} / r_s = -0.4581652932831429 / r_s."""
    for rs in (0.5, 1.0, 3.0):
        rho = 3.0 / (4 * math.pi * rs ** 3)
        assert np.isclose(fn.e_x_lda(rho) / rho, -0.4581652932831429 / rs, rtol=1e-14)


def _eps_c_at(rs):
    return fn.eps_c_pw92(3.0 / (4 * math.pi * rs ** 3))


def test_pw92_high_density_limit():
    """High density (Gell-Mann-Brueckner): eps_c = c0 ln rs - c1 + O(rs ln rs) with
    c0 = (1 - ln 2)/pi^2 exactly and c1 = 0.046644.  PW92 builds its beta_1 from c0 and c1
    and beta_2 = 2 A beta_1^2 so that no rs^{1/2} term appears.  The slope pins A (5 digits),
    the intercept pins beta_1; a wrong fourth digit of either moves them past the bounds."""
    c0 = (1 - math.log(2)) / math.pi ** 2
    r1, r2 = 1e-10, 1e-12
    e1, e2 = _eps_c_at(r1), _eps_c_at(r2)
    slope = (e2 - e1) / (math.log(r2) - math.log(r1))
    assert abs(slope / c0 - 1) < 1.5e-5, slope
    assert abs((e1 - slope * math.log(r1)) - (-0.046644)) < 2e-6
    A = fn.PW_A
    b1, b2 = fn.PW_BETA[0], fn.PW_BETA[1]
    assert abs(b2 / (2 * A * b1 * b1) - 1) < 5e-5


def test_pw92_low_density_limit():
    """Low density: eps_c = -d0/rs + d1/rs^{3/2} + O(1/rs^2) with d0 = 0.4335 and
    d1 = 1.4408 (the Wigner-crystal expansion PW92 is built to).  A fit of rs eps_c over
    rs = 1e3..1e5 recovers both; a wrong fourth digit of alpha_1, beta_3 or beta_4 fails."""
    rs = np.geomspace(1e3, 1e5, 9)
    y = np.array([_eps_c_at(r) * r for r in rs])
    X = np.stack([np.ones_like(rs), rs ** -0.5, rs ** -1.0, rs ** -1.5], axis=1)
    coef = np.linalg.lstsq(X, y, rcond=None)[0]
    assert abs(-coef[0] / 0.4335 - 1) < 1.2e-4, coef
    assert abs(coef[1] / 1.4408 - 1) < 2e-4, coef
    # a mid-range value well inside the published fit range (r_s = 2: about -0.0448 Ha)
    assert -0.0452 < _eps_c_at(2.0) < -0.0443


def test_pbe_constants_from_exact_conditions():
    """PBE's constants come from exact conditions, not fits: F_x(s -> inf) = 1 + kappa is the
    local Lieb-Oxford bound 1.679 / (C_x 2^{1/3}) (C_x = (3/4)(3/pi)^{1/3}), beta is the
    Ma-Brueckner gradient coefficient (16/pi)(3 pi^2)^{1/3} 0.004235 and gamma = (1 - ln 2)/pi^2.
    Evaluated through the energy density where the constant shows up in its output."""
    rho = 0.3
    fx_inf = fn.e_xc_pbe(rho, 1e40) / fn.e_x_lda(rho)
    lo = 1.679 / (0.75 * (3 / math.pi) ** (1 / 3) * 2 ** (1 / 3))
    assert abs(fx_inf - lo) < 5e-4, (fx_inf, lo)
    assert abs(fn.PBE_BETA / ((16 / math.pi) * (3 * math.pi ** 2) ** (1 / 3) * 0.004235) - 1) < 1.5e-4
    assert abs(fn.PBE_GAMMA - (1 - math.log(2)) / math.pi ** 2) < 1e-17


def test_lc94_gradient_expansion():
    """LC94 is fitted to reproduce the second-order gradient expansion of the kinetic energy,
    T = T_TF + T_W/9, i.e. F(s) = 1 + (5/27) s^2 + O(s^4) (its c + d = 0.18512 against
    5/27 = 0.18519).  Pins the small-s curvature to 4e-4; the individual constants a, b,
    alpha, f and the split of c + d have no independent value here (parity unpinned)."""
    s = np.array([1e-4, 2e-4])
    F, _ = fn.kedf_F(s, fn.KEDF_LC94)
    curv = (F - 1.0) / s ** 2
    assert np.all(np.abs(curv / (5 / 27) - 1) < 4e-4), curv
    # revAPBEK: F = 1 + mu s^2 + ... with mu = 0.23889 (not the gradient expansion's 5/27);
    # its kappa and mu are the cited functional's published values (parity unpinned)
    F, _ = fn.kedf_F(s, fn.KEDF_REVAPBEK)
    assert np.allclose((F - 1.0) / s ** 2, fn.RAPBEK_MU, rtol=1e-6)


def test_pbe_reduces_to_lda_and_limits():
    rho = np.array([1e-3, 0.05, 0.3, 2.0])
    assert np.allclose(fn.e_xc_pbe(rho, np.zeros_like(rho)), fn.e_xc_lda(rho), rtol=1e-14)
    # exchange enhancement saturates at 1 + kappa for s -> infinity; correlation -> 0 for t -> inf
    sig = 1e30 * np.ones_like(rho)
    ex = fn.e_x_lda(rho) * (1 + fn.PBE_KAPPA)
    assert np.allclose(fn.e_xc_pbe(rho, sig), ex, rtol=1e-9)
    # PBE fixes mu = beta pi^2 / 3 so that the second-order gradient terms of exchange
    # (e_x mu s^2) and correlation (rho beta t^2) cancel for slowly varying densities
    assert abs(fn.PBE_MU - fn.PBE_BETA * math.pi ** 2 / 3) < 1e-15
    r0 = 0.2
    kf = (3 * math.pi ** 2 * r0) ** (1 / 3)
    s2 = 1e-7
    sig = s2 * 4 * kf * kf * r0 * r0
    diff = fn.e_xc_pbe(r0, sig) - fn.e_xc_pbe(r0, 0.0)
    assert abs(diff) < 1e-5 * abs(fn.e_x_lda(r0) * fn.PBE_MU * s2)


def test_kedf_enhancement_factors():
    s = np.array([0.0, 0.1, 1.0, 5.0])
    for kind in (fn.KEDF_REVAPBEK, fn.KEDF_LC94):
        F, dF = fn.kedf_F(s, kind)
        assert np.isclose(F[0], 1.0) and np.isclose(dF[0], 0.0)
        # derivative against complex step of F itself
        h = 1e-30
        cs = np.imag(fn.kedf_F(s[1:] + 1j * h, kind)[0]) / h
        assert np.allclose(dF[1:], cs, rtol=1e-12)
    F, _ = fn.kedf_F(np.array([1e8]), fn.KEDF_REVAPBEK)
    assert np.isclose(F[0], 1 + fn.RAPBEK_KAPPA, rtol=1e-9)


def test_complex_step_matches_finite_difference():
    rho = np.array([0.01, 0.2, 1.5])
    sig = np.array([0.001, 0.05, 0.4])
    e, er, es = fn._complex_step(fn.e_xc_pbe, rho, sig)
    h = 1e-6
    fd_r = (fn.e_xc_pbe(rho * (1 + h), sig) - fn.e_xc_pbe(rho * (1 - h), sig)) / (2 * h * rho)
    fd_s = (fn.e_xc_pbe(rho, sig * (1 + h)) - fn.e_xc_pbe(rho, sig * (1 - h))) / (2 * h * sig)
    assert np.allclose(er, fd_r, rtol=1e-7)
    assert np.allclose(es, fd_s, rtol=1e-6)


def test_thomas_fermi_nonadditive_uniform():
    """Two uniform densities: T^nad = C_TF Omega [(a+b)^{5/3} - a^{5/3} - b^{5/3}],
    v_A^nad = (5/3) C_TF [(a+b)^{2/3} - a^{2/3}]."""
    a, b = 0.013, 0.041
    ra = np.full(GRID, a)
    rb = np.full(GRID, b)
    omega = basis.volume(LAT)
    T, v = fn.kinetic(ra + rb, LAT, fn.KEDF_TF)
    Ta, va = fn.kinetic(ra, LAT, fn.KEDF_TF)
    Tb, _ = fn.kinetic(rb, LAT, fn.KEDF_TF)
    want = fn.C_TF * omega * ((a + b) ** (5 / 3) - a ** (5 / 3) - b ** (5 / 3))
    assert np.isclose(T - Ta - Tb, want, rtol=1e-13)
    assert np.allclose(v - va, 5 / 3 * fn.C_TF * ((a + b) ** (2 / 3) - a ** (2 / 3)), rtol=1e-13)
    assert np.isclose(fn.C_TF, 2.871234000188191, rtol=1e-14)


def test_gga_kinetic_reduces_to_tf_for_uniform_density():
    rho = np.full(GRID, 0.07)
    for kind in (fn.KEDF_REVAPBEK, fn.KEDF_LC94):
        T, v = fn.kinetic(rho, LAT, kind)
        Ttf, vtf = fn.kinetic(rho, LAT, fn.KEDF_TF)
        assert np.isclose(T, Ttf, rtol=1e-13) and np.allclose(v, vtf, rtol=1e-12)


def test_reduced_gradient_constant():
    """s = |grad rho| / (2 k_F rho) with k_F = (3 pi^2 rho)^{1/3}."""
    rho, g = 0.3, 0.7
    kf = (3 * math.pi ** 2 * rho) ** (1 / 3)
    assert np.isclose(fn.C_S * g / rho ** (4 / 3), g / (2 * kf * rho), rtol=1e-14)


@pytest.mark.parametrize("which,kind", [("kin", fn.KEDF_TF), ("kin", fn.KEDF_REVAPBEK),
                                        ("kin", fn.KEDF_LC94), ("xc", fn.XC_LDA),
                                        ("xc", fn.XC_PBE)])
def test_potential_is_functional_derivative(which, kind):
    """(E[rho + e d] - E[rho - e d]) / 2e = int v d for a smooth perturbation d (pins the
    divergence term of the GGA potential)."""
    f = fn.kinetic if which == "kin" else fn.xc
    rho = _smooth_density()
    d = _smooth_perturbation()
    _, v = f(rho, LAT, kind)
    eps = 1e-3
    Ep, _ = f(rho + eps * d, LAT, kind)
    Em, _ = f(rho - eps * d, LAT, kind)
    fd = (Ep - Em) / (2 * eps)
    an = float(basis.integrate(v * d, LAT))
    assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


def test_gradient_and_divergence_of_plane_waves():
    r = basis.grid_points(LAT, GRID)
    G = 2 * math.pi * np.array([2 / 7.0, -1 / 8.0, 3 / 9.0])
    f = np.sin(r @ G)
    g = fn.gradient(f, LAT)
    for c in range(3):
        assert np.allclose(g[c], G[c] * np.cos(r @ G), atol=1e-12)
    div = fn.divergence(g, LAT)
    assert np.allclose(div, -(G @ G) * f, atol=1e-11)


def test_low_density_cut():
    rho = _smooth_density()
    rho[:3] = 1e-12
    _, v = fn.xc(rho, LAT, fn.XC_LDA)
    assert np.all(v[:3] == 0.0)
    _, v = fn.kinetic(rho, LAT, fn.KEDF_TF)
    assert np.all(v[:3] == 0.0)
