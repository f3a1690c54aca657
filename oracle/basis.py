"""Cell, real-space grid, plane-wave sphere and discrete Fourier conventions.

Test infrastructure only (see ``oracle/__init__.py``).

Conventions (the paper is silent on them; Sec. 2 only states that orbitals are Bloch
functions psi = e^{ik.r} u with u periodic, Eq. KS):

* lattice rows a_i; reciprocal rows b_j with a_i . b_j = 2 pi delta_ij; Omega = |det a|.
* grid point r(i) = sum_j (i_j / n_j) a_j, i_j in [0, n_j); N_r = n1 n2 n3.
* a Miller index m (signed) labels G = m_1 b_1 + m_2 b_2 + m_3 b_3; it sits at grid
  index i_j = m_j mod n_j.  A grid index maps back to the signed index of ``fftfreq``
  order; for even n_j the index n_j/2 is the Nyquist plane m_j = -n_j/2.
* u_{jk}(r) = Omega^{-1/2} sum_G c_G e^{iG.r} with sum_G |c_G|^2 = 1.
* forward transform f(G) = (1/N_r) sum_r f(r) e^{-iG.r}; inverse f(r) = sum_G f(G) e^{iG.r};
  integrals over the cell are (Omega/N_r) sum_r.
* the wavefunction sphere holds every G with 0.5 |k+G|^2 <= E_cut, evaluated in FP64
  from the integer Miller indices (computational details: a wavefunction cutoff),
  sorted lexicographically by signed (m1, m2, m3).
"""
from __future__ import annotations

import numpy as np
import scipy.fft

FFT_WORKERS = -1  # all host cores


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_j with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def volume(lattice: np.ndarray) -> float:
    return float(abs(np.linalg.det(np.asarray(lattice, dtype=np.float64))))


def axis_miller(n: int) -> np.ndarray:
    """Signed Miller index of each grid index along one axis (fftfreq order)."""
    m = np.arange(n, dtype=np.int64)
    m[m >= (n + 1) // 2] -= n
    return m


def grid_miller(grid):
    """Three [n1, n2, n3] integer arrays of signed Miller indices of the full grid."""
    return np.meshgrid(axis_miller(grid[0]), axis_miller(grid[1]), axis_miller(grid[2]),
                       indexing="ij")


def nyquist_mask(grid) -> np.ndarray:
    """True where any Miller index lies on an even axis's -n/2 plane.

    Reading adopted for every G-space filter (Poisson, local potential, gradient,
    divergence): those coefficients are set to zero so that each filtered field is
    real by construction (the paper is silent on Nyquist planes)."""
    m1, m2, m3 = grid_miller(grid)
    mask = np.zeros(tuple(grid), dtype=bool)
    for m, n in ((m1, grid[0]), (m2, grid[1]), (m3, grid[2])):
        if n % 2 == 0:
            mask |= (m == -(n // 2))
    return mask


def cart_from_miller(m1, m2, m3, B):
    """Cartesian G = m1 b1 + m2 b2 + m3 b3 evaluated component by component
    (no fused multiply-add), returned as a tuple of three arrays."""
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    m3 = np.asarray(m3, dtype=np.float64)
    return tuple(m1 * B[0, c] + m2 * B[1, c] + m3 * B[2, c] for c in range(3))


def grid_gvectors(lattice, grid):
    """Cartesian G of every grid index, as three [n1, n2, n3] arrays, and |G|^2."""
    B = reciprocal(lattice)
    gx, gy, gz = cart_from_miller(*grid_miller(grid), B)
    return (gx, gy, gz), gx * gx + gy * gy + gz * gz


def grid_points(lattice, grid):
    """Cartesian coordinates of every grid point, [n1, n2, n3, 3]."""
    A = np.asarray(lattice, dtype=np.float64)
    f = np.meshgrid(*(np.arange(n) / n for n in grid), indexing="ij")
    return f[0][..., None] * A[0] + f[1][..., None] * A[1] + f[2][..., None] * A[2]


def sphere(lattice, grid, kfrac, ecut):
    """Plane-wave sphere of one k-point: Miller indices [npw, 3] (int64) sorted
    lexicographically by (m1, m2, m3), and the kinetic energies 0.5 |k+G|^2."""
    B = reciprocal(lattice)
    A = np.asarray(lattice, dtype=np.float64)
    kc = tuple(float(kfrac[0]) * B[0, c] + float(kfrac[1]) * B[1, c] + float(kfrac[2]) * B[2, c]
               for c in range(3))
    qmax = np.sqrt(2.0 * ecut) + np.sqrt(kc[0] ** 2 + kc[1] ** 2 + kc[2] ** 2)
    lim = [int(np.ceil(qmax * np.linalg.norm(A[j]) / (2.0 * np.pi))) + 1 for j in range(3)]
    r = [np.arange(-l, l + 1) for l in lim]
    m1, m2, m3 = np.meshgrid(*r, indexing="ij")
    m1, m2, m3 = m1.ravel(), m2.ravel(), m3.ravel()
    gx, gy, gz = cart_from_miller(m1, m2, m3, B)
    qx, qy, qz = kc[0] + gx, kc[1] + gy, kc[2] + gz
    kin = 0.5 * (qx * qx + qy * qy + qz * qz)
    keep = kin <= ecut
    mil = np.stack([m1[keep], m2[keep], m3[keep]], axis=1).astype(np.int64)
    order = np.lexsort((mil[:, 2], mil[:, 1], mil[:, 0]))
    mil = mil[order]
    kin = kin[keep][order]
    for j in range(3):
        span = mil[:, j].max() - mil[:, j].min() + 1
        if span > grid[j]:
            raise ValueError(f"sphere does not fit the grid along axis {j}")
    return mil, kin


def kcart(lattice, kfrac):
    B = reciprocal(lattice)
    return np.array([float(kfrac[0]) * B[0, c] + float(kfrac[1]) * B[1, c]
                     + float(kfrac[2]) * B[2, c] for c in range(3)])


def to_grid(coef, miller, grid):
    """Place sphere coefficients [..., npw] at their grid indices (zero elsewhere)."""
    coef = np.asarray(coef)
    box = np.zeros(coef.shape[:-1] + tuple(grid), dtype=np.complex128)
    idx = tuple(miller[:, j] % grid[j] for j in range(3))
    box[(Ellipsis,) + idx] = coef
    return box


def from_grid(box, miller, grid):
    idx = tuple(miller[:, j] % grid[j] for j in range(3))
    return box[(Ellipsis,) + idx]


def r_from_G(fG):
    """f(r) = sum_G f(G) e^{iG.r} over the last three axes."""
    n = np.prod(fG.shape[-3:])
    return scipy.fft.ifftn(fG, axes=(-3, -2, -1), workers=FFT_WORKERS) * n


def G_from_r(fr):
    """f(G) = (1/N_r) sum_r f(r) e^{-iG.r} over the last three axes."""
    n = np.prod(fr.shape[-3:])
    return scipy.fft.fftn(fr, axes=(-3, -2, -1), workers=FFT_WORKERS) / n


def dft_direct(f, sign):
    """Brute-force 3D DFT  F(i') = sum_i f(i) exp(sign * 2 pi i sum_j i_j i'_j / n_j),
    used only to pin the FFT conventions on tiny grids."""
    n1, n2, n3 = f.shape
    out = np.zeros_like(f, dtype=np.complex128)
    i1, i2, i3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    for a in range(n1):
        for b in range(n2):
            for c in range(n3):
                ph = sign * 2j * np.pi * (a * i1 / n1 + b * i2 / n2 + c * i3 / n3)
                out[a, b, c] = np.sum(f * np.exp(ph))
    return out


def integrate(f_r, lattice):
    """Cell integral of a grid function, (Omega/N_r) sum_r f(r)."""
    return volume(lattice) / np.prod(f_r.shape[-3:]) * np.sum(f_r, axis=(-3, -2, -1))
