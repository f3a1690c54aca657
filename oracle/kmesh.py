"""Monkhorst-Pack meshes, their reduction by symmetry, and density symmetrisation.

Test infrastructure only (see ``oracle/__init__.py``).

Computational Details: the periodic systems are sampled with a 2 x 2 x 1 Monkhorst-Pack mesh.
The mesh points of axis j are (2 r - q_j - 1) / (2 q_j), r = 1..q_j (crystal coordinates).
Time reversal relates k and -k (e(k) = e(-k), u_-k = conj(u_k), so both give the same
density); a point-group operation R of the whole system relates k and R k, and the density
of the reduced set becomes the full-mesh density once averaged over the group.  Only the
sign-flip operations about the origin (mirrors, two-fold axes and inversion of an
orthorhombic cell) are considered.  Exact rational arithmetic decides which points coincide
(modulo integers).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def monkhorst_pack(q, shift=(0, 0, 0)):
    axes = [[Fraction(2 * r - qj - 1, 2 * qj) + Fraction(sj).limit_denominator(1000) / (2 * qj)
             for r in range(1, qj + 1)] for qj, sj in zip(q, shift)]
    return [(a, b, c) for a in axes[0] for b in axes[1] for c in axes[2]]


def _flip(k, mask, sign=1):
    return tuple(sign * (-x if (mask >> d) & 1 else x) for d, x in enumerate(k))


def _key(k):
    return tuple(x - (x.numerator // x.denominator) for x in k)  # the point modulo integers


def reduce_mesh(points, ops=(), time_reversal=True):
    """Irreducible points (first of each orbit, mesh order) and weights orbit/len(points)."""
    group = {0} | set(ops)
    signs = (1, -1) if time_reversal else (1,)
    index = {_key(k): i for i, k in enumerate(points)}
    seen = [False] * len(points)
    out, w = [], []
    for i, k in enumerate(points):
        if seen[i]:
            continue
        orbit = {index[_key(_flip(k, m, s))] for m in group for s in signs if _key(_flip(k, m, s)) in index}
        for j in orbit:
            seen[j] = True
        out.append(k)
        w.append(Fraction(len(orbit), len(points)))
    return np.array([[float(x) for x in k] for k in out]), np.array([float(x) for x in w])


def symmetry_ops(lattice, pos, Z, tol=1e-6):
    """Sign-flip masks (bit c flips coordinate c) mapping the atoms onto equal-charge atoms."""
    L = np.diag(np.asarray(lattice, dtype=np.float64))
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    out = []
    for m in range(8):
        s = np.array([-1.0 if (m >> d) & 1 else 1.0 for d in range(3)])
        img = pos * s
        d = img[:, None, :] - pos[None, :, :]
        d -= L * np.round(d / L)
        close = (np.sqrt((d * d).sum(-1)) <= tol) & (np.asarray(Z)[:, None] == np.asarray(Z)[None, :])
        if close.any(axis=1).all():
            out.append(m)
    return out


def symmetrize(rho, ops):
    """(1 / |G|) sum_R rho(R r) on the grid: r -> -r (mod n) along each flipped axis."""
    acc = np.zeros_like(rho)
    for m in ops:
        f = rho
        for ax in range(3):
            if (m >> ax) & 1:
                f = np.roll(np.flip(f, axis=ax), 1, axis=ax)
        acc += f
    return acc / len(ops)
