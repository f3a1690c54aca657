"""Electron-nucleus, Hartree and nucleus-nucleus terms; Kleinman-Bylander projectors.

Test infrastructure only (see ``oracle/__init__.py``).

* Hartree potential by the Poisson equation in reciprocal space,
  v_H(G) = 4 pi rho(G) / |G|^2 (Sec. 2, FFT Poisson solve; Appendix, Eq. for V_H).
* Electron-nucleus attraction of all nuclei grouped in one potential (Appendix,
  recast effective potential: "V_eN" of every nucleus; Eq. for E_eN^J).  The nuclei are
  modelled by Gaussian-regularised local potentials -Z erf(r/r_c)/r.
* Nuclear repulsion V_NN (Eq. of E_FDE) by an Ewald sum.
* Subsystem-specific nonlocal projectors (Appendix, subsystem-specific PAW projectors:
  only projectors of atoms in I act on the orbitals of I); modelled by Gaussian
  s-type Kleinman-Bylander projectors.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

from . import basis


def vloc_G(lattice, grid, pos, Z, rc):
    """Fourier coefficients v_loc(G) of sum_alpha -Z_alpha erf(|r - R_alpha|/r_c)/|r - R_alpha|.

    For G != 0: (1/Omega) sum_alpha (-4 pi Z_alpha / G^2) exp(-G^2 r_c^2 / 4) exp(-i G.R_alpha).
    G = 0 (uniform-background convention): the divergent -Z/r part is dropped and the
    finite remainder (1/Omega) sum_alpha pi Z_alpha r_c^2 is kept.  Nyquist planes zero."""
    omega = basis.volume(lattice)
    (gx, gy, gz), g2 = basis.grid_gvectors(lattice, grid)
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    Z = np.asarray(Z, dtype=np.float64)
    nz = g2 > 0
    form = np.zeros_like(g2)
    form[nz] = -4.0 * np.pi / g2[nz] * np.exp(-g2[nz] * rc * rc / 4.0)
    # structure factor S(G) = sum_alpha Z_alpha exp(-i G.R_alpha); in an orthorhombic cell
    # G.R = G_x x + G_y y + G_z z with G_x depending on the first index only (and so on), so the
    # exponential is a product of three 1D factors and the sum over atoms is one matrix product
    A = np.asarray(lattice, dtype=np.float64)
    if np.count_nonzero(A - np.diag(np.diag(A))) == 0:
        n1, n2, n3 = grid
        ex = np.exp(-1j * np.outer(pos[:, 0], gx[:, 0, 0]))  # [natoms][n1]
        ey = np.exp(-1j * np.outer(pos[:, 1], gy[0, :, 0]))
        ez = np.exp(-1j * np.outer(pos[:, 2], gz[0, 0, :]))
        m = (Z[:, None, None] * ex[:, :, None] * ey[:, None, :]).reshape(len(Z), n1 * n2)
        S = (m.T @ ez).reshape(n1, n2, n3)
    else:
        S = np.zeros(tuple(grid), dtype=np.complex128)
        for p, z in zip(pos, Z):
            S += z * np.exp(-1j * (gx * p[0] + gy * p[1] + gz * p[2]))
    out = form * S / omega
    out[0, 0, 0] = np.pi * float(Z.sum()) * rc * rc / omega
    out[basis.nyquist_mask(grid)] = 0.0
    return out


def vloc_r(lattice, grid, pos, Z, rc):
    return np.real(basis.r_from_G(vloc_G(lattice, grid, pos, Z, rc)))


def hartree_G(rho_r, lattice):
    """v_H(G) = 4 pi rho(G) / |G|^2, G = 0 and Nyquist planes set to zero."""
    grid = rho_r.shape
    _, g2 = basis.grid_gvectors(lattice, grid)
    rhoG = basis.G_from_r(rho_r)
    v = np.zeros_like(rhoG)
    nz = g2 > 0
    v[nz] = 4.0 * np.pi * rhoG[nz] / g2[nz]
    v[basis.nyquist_mask(grid)] = 0.0
    return v


def hartree(rho_r, lattice):
    """Hartree potential on the grid and E_H = (1/2) int v_H rho."""
    v = np.real(basis.r_from_G(hartree_G(rho_r, lattice)))
    return v, 0.5 * float(basis.integrate(v * rho_r, lattice))


def ewald(lattice, pos, Z, eta=None, tol=1e-16):
    """Nuclear repulsion of point charges Z_alpha with a neutralising background:
    E = 1/2 sum' Z_a Z_b erfc(eta d)/d + (2 pi/Omega) sum_{G!=0} exp(-G^2/4eta^2)/G^2 |S(G)|^2
        - eta/sqrt(pi) sum Z^2 - pi (sum Z)^2 / (2 Omega eta^2)."""
    A = np.asarray(lattice, dtype=np.float64)
    pos = np.asarray(pos, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    omega = basis.volume(A)
    B = basis.reciprocal(A)
    if eta is None:
        eta = math.sqrt(math.pi) / omega ** (1.0 / 3.0)
    x = math.sqrt(-math.log(tol))
    rmax = x / eta + 1.0
    gmax = 2.0 * eta * x + 1.0
    # real space
    nl = [int(math.ceil(rmax * np.linalg.norm(B[j]) / (2 * math.pi))) + 1 for j in range(3)]
    e_real = 0.0
    for n1 in range(-nl[0], nl[0] + 1):
        for n2 in range(-nl[1], nl[1] + 1):
            for n3 in range(-nl[2], nl[2] + 1):
                L = n1 * A[0] + n2 * A[1] + n3 * A[2]
                d = pos[:, None, :] - pos[None, :, :] + L
                r = np.sqrt((d * d).sum(-1))
                if n1 == 0 and n2 == 0 and n3 == 0:
                    np.fill_diagonal(r, np.inf)
                m = r < rmax
                e_real += 0.5 * np.sum((Z[:, None] * Z[None, :] * erfc(eta * r) / r)[m])
    # reciprocal space
    ng = [int(math.ceil(gmax * np.linalg.norm(A[j]) / (2 * math.pi))) + 1 for j in range(3)]
    m1, m2, m3 = np.meshgrid(*(np.arange(-n, n + 1) for n in ng), indexing="ij")
    gx, gy, gz = basis.cart_from_miller(m1.ravel(), m2.ravel(), m3.ravel(), B)
    g2 = gx * gx + gy * gy + gz * gz
    keep = (g2 > 0) & (g2 < gmax * gmax)
    gx, gy, gz, g2 = gx[keep], gy[keep], gz[keep], g2[keep]
    S = np.zeros(g2.shape, dtype=np.complex128)
    for p, z in zip(pos, Z):
        S += z * np.exp(1j * (gx * p[0] + gy * p[1] + gz * p[2]))
    e_rec = 2.0 * math.pi / omega * float(np.sum(np.exp(-g2 / (4 * eta * eta)) / g2 * np.abs(S) ** 2))
    e_self = -eta / math.sqrt(math.pi) * float(np.sum(Z * Z))
    e_bg = -math.pi * float(np.sum(Z)) ** 2 / (2.0 * omega * eta * eta)
    return e_real + e_rec + e_self + e_bg


def kb_projectors(lattice, kfrac, miller, pos, sigma):
    """Gaussian KB projectors of a set of atoms in the plane-wave basis of one k-point.

    beta_{a,i}(k+G) = Omega^{-1/2} (pi^{3/2} sigma_i^3)^{-1/2} (2 pi sigma_i^2)^{3/2}
                      exp(-|k+G|^2 sigma_i^2 / 2) exp(-i (k+G).R_a),
    the plane-wave matrix elements <k+G|beta> of the unit-norm real-space Gaussian
    (pi^{3/2} sigma^3)^{-1/2} exp(-|r-R|^2 / (2 sigma^2)).
    Returns [natoms * nproj, npw] with the projector index fastest."""
    omega = basis.volume(lattice)
    B = basis.reciprocal(lattice)
    kc = basis.kcart(lattice, kfrac)
    gx, gy, gz = basis.cart_from_miller(miller[:, 0], miller[:, 1], miller[:, 2], B)
    qx, qy, qz = kc[0] + gx, kc[1] + gy, kc[2] + gz
    q2 = qx * qx + qy * qy + qz * qz
    rows = []
    for p in np.asarray(pos, dtype=np.float64):
        phase = np.exp(-1j * (qx * p[0] + qy * p[1] + qz * p[2]))
        for s in sigma:
            amp = (omega ** -0.5) * (math.pi ** 1.5 * s ** 3) ** -0.5 * (2 * math.pi * s * s) ** 1.5
            rows.append(amp * np.exp(-q2 * s * s / 2.0) * phase)
    if not rows:
        return np.zeros((0, miller.shape[0]), dtype=np.complex128)
    return np.array(rows)


def kb_coupling(natoms, D):
    """Block-diagonal coupling matrix over (atom, projector) for a per-atom matrix D."""
    D = np.asarray(D, dtype=np.float64)
    if D.size == 0:
        return np.zeros((0, 0))
    return np.kron(np.eye(natoms), D)


def augmentation_G(lattice, grid, pos, coef, sigma):
    """sum_a coef_a g_a(G) for the normalised Gaussians g_a(r) = (pi sigma^2)^{-3/2}
    exp(-|r - R_a|^2 / sigma^2) of the ultrasoft-like augmentation charges (Appendix,
    subsystem-specific projectors; the paper's PAW/ultrasoft data are replaced by this model):
    g_a(G) = (1/Omega) exp(-G^2 sigma^2 / 4) exp(-i G.R_a), Nyquist planes zero, so that
    int g_a = 1 on the grid."""
    omega = basis.volume(lattice)
    (gx, gy, gz), g2 = basis.grid_gvectors(lattice, grid)
    shape = np.exp(-g2 * sigma * sigma / 4.0) / omega
    out = np.zeros(tuple(grid), dtype=np.complex128)
    for p, c in zip(np.asarray(pos, dtype=np.float64).reshape(-1, 3), np.asarray(coef, dtype=np.float64)):
        out += c * shape * np.exp(-1j * (gx * p[0] + gy * p[1] + gz * p[2]))
    out[basis.nyquist_mask(grid)] = 0.0
    return out


def augmentation_overlaps(lattice, grid, pos, sigma, v_r):
    """int v(r) g_a(r) dr for every atom a, with g_a the grid augmentation shape above:
    Parseval, (Omega / N_r) sum_r v g_a = Omega sum_G v(G) conj(g_a(G))."""
    omega = basis.volume(lattice)
    (gx, gy, gz), g2 = basis.grid_gvectors(lattice, grid)
    vG = basis.G_from_r(v_r)
    vG[basis.nyquist_mask(grid)] = 0.0
    shape = np.exp(-g2 * sigma * sigma / 4.0)
    out = []
    for p in np.asarray(pos, dtype=np.float64).reshape(-1, 3):
        out.append(float(np.real(np.sum(vG * shape * np.exp(1j * (gx * p[0] + gy * p[1] + gz * p[2]))))))
    del omega
    return np.array(out)

