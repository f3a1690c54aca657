"""Semilocal density functionals and their potentials on the periodic grid.

Test infrastructure only (see ``oracle/__init__.py``).

* Kinetic-energy density functionals of the GGA family (Appendix, kinetic energy
  functional and potential): T = C_TF int rho^{5/3} F(s), s = C_s |grad rho| / rho^{4/3},
  C_TF = (3/10)(3 pi^2)^{2/3}.  The paper prints C_s = 1/(2 (2 pi^2)^{1/3}); the reduced
  gradient the cited enhancement factors are parameterised in is
  s = |grad rho| / (2 (3 pi^2)^{1/3} rho^{4/3}), so C_s = 1/(2 (3 pi^2)^{1/3}) is used
  (reading: typo in the printed constant).
  Potential in the paper's order: dG/drho = rho^{2/3} [5/3 F - 4/3 s F'],
  dG/dgrad rho = C_s rho^{1/3} F' grad rho / |grad rho|, and
  v_kin = C_TF { dG/drho - div( dG/dgrad rho ) }.
  F: Thomas-Fermi (F = 1), revAPBEK, LC94 (Computational Details name the latter two).
* Exchange-correlation: LDA (Slater exchange + Perdew-Wang 1992 correlation) and PBE
  (Computational Details).  The paper prints neither; the published forms are written
  out below.  For a GGA energy density e(rho, sigma = |grad rho|^2) the potential is the
  functional derivative (Appendix, generic GGA derivative)
  v = de/drho - div(2 de/dsigma grad rho);
  de/drho and de/dsigma are taken by complex-step differentiation of e, which is exact
  to rounding (no truncation error).
* Gradients and divergences are taken through FFTs (i G multiplication), with the
  Nyquist planes zeroed.
* Low density (the paper is silent): where rho < rho_cut a functional contributes zero
  energy density and zero potential; |grad rho| is floored at 1e-30 where divided by.
"""
from __future__ import annotations

import math

import numpy as np

from . import basis

C_TF = 0.3 * (3.0 * math.pi ** 2) ** (2.0 / 3.0)
C_S = 1.0 / (2.0 * (3.0 * math.pi ** 2) ** (1.0 / 3.0))

# Perdew-Wang 1992, unpolarised correlation
PW_A, PW_ALPHA1 = 0.031091, 0.21370
PW_BETA = (7.5957, 3.5876, 1.6382, 0.49294)
# PBE
PBE_KAPPA, PBE_MU = 0.804, 0.2195149727645171
PBE_BETA = 0.06672455060314922
PBE_GAMMA = (1.0 - math.log(2.0)) / math.pi ** 2
# revAPBEK
RAPBEK_KAPPA, RAPBEK_MU = 1.245, 0.23889
# LC94 (PW91 form)
LC94 = dict(a=0.093907, b=76.32, c=0.26608, d=-0.0809615, alpha=100.0, f=0.000057767)

XC_LDA, XC_PBE = 0, 1
KEDF_TF, KEDF_REVAPBEK, KEDF_LC94 = 0, 1, 2

_H_STEP = 1e-30


# ---------------------------------------------------------------- energy densities
def e_x_lda(rho):
    """Slater exchange energy per volume, -(3/4)(3/pi)^{1/3} rho^{4/3}."""
    return -0.75 * (3.0 / math.pi) ** (1.0 / 3.0) * rho ** (4.0 / 3.0)


def eps_c_pw92(rho):
    """Perdew-Wang 1992 correlation energy per electron (unpolarised)."""
    rs = (3.0 / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    b1, b2, b3, b4 = PW_BETA
    den = 2.0 * PW_A * (b1 * rs ** 0.5 + b2 * rs + b3 * rs ** 1.5 + b4 * rs * rs)
    return -2.0 * PW_A * (1.0 + PW_ALPHA1 * rs) * np.log(1.0 + 1.0 / den)


def e_xc_lda(rho, sigma=None):
    return e_x_lda(rho) + rho * eps_c_pw92(rho)


def e_xc_pbe(rho, sigma):
    """PBE exchange-correlation energy per volume as a function of rho and
    sigma = |grad rho|^2 (unpolarised, phi = 1)."""
    kf = (3.0 * math.pi ** 2 * rho) ** (1.0 / 3.0)
    s2 = sigma / (4.0 * kf * kf * rho * rho)
    fx = 1.0 + PBE_KAPPA - PBE_KAPPA / (1.0 + PBE_MU * s2 / PBE_KAPPA)
    ex = e_x_lda(rho) * fx
    ec_unif = eps_c_pw92(rho)
    ks = np.sqrt(4.0 * kf / math.pi)
    t2 = sigma / (4.0 * ks * ks * rho * rho)
    bg = PBE_BETA / PBE_GAMMA
    A = bg / (np.exp(-ec_unif / PBE_GAMMA) - 1.0)
    At2 = A * t2
    H = PBE_GAMMA * np.log(1.0 + bg * t2 * (1.0 + At2) / (1.0 + At2 + At2 * At2))
    return ex + rho * (ec_unif + H)


def kedf_F(s, kind):
    """Enhancement factor F(s) and its derivative F'(s)."""
    if kind == KEDF_TF:
        return np.ones_like(s), np.zeros_like(s)
    if kind == KEDF_REVAPBEK:
        k, mu = RAPBEK_KAPPA, RAPBEK_MU
        d = 1.0 + mu * s * s / k
        return 1.0 + k - k / d, 2.0 * mu * s / (d * d)
    if kind == KEDF_LC94:
        a, b, c, dd, al, f = (LC94[x] for x in ("a", "b", "c", "d", "alpha", "f"))
        ash = np.arcsinh(b * s)
        ex = np.exp(-al * s * s)
        num = 1.0 + a * s * ash + (c + dd * ex) * s * s
        den = 1.0 + a * s * ash + f * s ** 4
        dash = a * ash + a * s * b / np.sqrt(1.0 + (b * s) ** 2)
        dnum = dash + 2.0 * s * (c + dd * ex) - 2.0 * al * dd * s ** 3 * ex
        dden = dash + 4.0 * f * s ** 3
        return num / den, (dnum * den - num * dden) / (den * den)
    raise ValueError(kind)


# ---------------------------------------------------------------- FFT derivatives
def gradient(f_r, lattice):
    """grad f through FFT: IFFT(i G f(G)), Nyquist planes zeroed; three real grids."""
    grid = f_r.shape
    (gx, gy, gz), _ = basis.grid_gvectors(lattice, grid)
    fG = basis.G_from_r(f_r)
    fG[basis.nyquist_mask(grid)] = 0.0
    return [np.real(basis.r_from_G(1j * g * fG)) for g in (gx, gy, gz)]


def divergence(h, lattice):
    """div h through FFT: IFFT(i G . h(G)), Nyquist planes zeroed."""
    grid = h[0].shape
    (gx, gy, gz), _ = basis.grid_gvectors(lattice, grid)
    acc = np.zeros(grid, dtype=np.complex128)
    for g, hc in zip((gx, gy, gz), h):
        acc += 1j * g * basis.G_from_r(hc)
    acc[basis.nyquist_mask(grid)] = 0.0
    return np.real(basis.r_from_G(acc))


# ---------------------------------------------------------------- potentials
def _complex_step(fun, rho, sigma):
    """Energy density and its partial derivatives d/drho, d/dsigma (complex step)."""
    e = np.real(fun(rho, sigma))
    e_r = np.imag(fun(rho + 1j * _H_STEP, sigma)) / _H_STEP
    e_s = np.imag(fun(rho, sigma + 1j * _H_STEP)) / _H_STEP
    return e, e_r, e_s


def xc(rho, lattice, kind, rho_cut=1e-10):
    """Exchange-correlation energy E_XC[rho] and potential v_XC[rho](r)."""
    act = rho >= rho_cut
    e = np.zeros_like(rho)
    v = np.zeros_like(rho)
    if kind == XC_LDA:
        r = rho[act]
        ee, er, _ = _complex_step(lambda a, b: e_xc_lda(a), r, np.zeros_like(r))
        e[act], v[act] = ee, er
        return float(basis.integrate(e, lattice)), v
    if kind != XC_PBE:
        raise ValueError(kind)
    g = gradient(rho, lattice)
    sigma = g[0] ** 2 + g[1] ** 2 + g[2] ** 2
    ee, er, es = _complex_step(e_xc_pbe, rho[act], sigma[act])
    e[act] = ee
    dedr = np.zeros_like(rho)
    deds = np.zeros_like(rho)
    dedr[act], deds[act] = er, es
    v = dedr - divergence([2.0 * deds * gc for gc in g], lattice)
    return float(basis.integrate(e, lattice)), v


def kinetic(rho, lattice, kind, rho_cut=1e-10):
    """Orbital-free kinetic energy T~[rho] = C_TF int rho^{5/3} F(s) and its potential
    v~_kin[rho](r), following the Appendix's derivation step by step."""
    act = rho >= rho_cut
    e = np.zeros_like(rho)
    dGdrho = np.zeros_like(rho)
    if kind == KEDF_TF:
        r = rho[act]
        e[act] = C_TF * r ** (5.0 / 3.0)
        dGdrho[act] = C_TF * (5.0 / 3.0) * r ** (2.0 / 3.0)
        return float(basis.integrate(e, lattice)), dGdrho
    g = gradient(rho, lattice)
    gnorm = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    r = rho[act]
    s = C_S * gnorm[act] / r ** (4.0 / 3.0)
    F, dF = kedf_F(s, kind)
    e[act] = C_TF * r ** (5.0 / 3.0) * F
    dGdrho[act] = C_TF * r ** (2.0 / 3.0) * (5.0 / 3.0 * F - 4.0 / 3.0 * s * dF)
    coef = np.zeros_like(rho)
    coef[act] = C_TF * C_S * r ** (1.0 / 3.0) * dF / np.maximum(gnorm[act], 1e-30)
    v = dGdrho - divergence([coef * gc for gc in g], lattice)
    return float(basis.integrate(e, lattice)), v
