"""Pins of the symmetry-reduced Monkhorst-Pack sampling of the oracle (CPU only)."""
import numpy as np
import pytest

from oracle import fde as ofde, kmesh, scf
from paper_1406_7803_gb300 import workloads


def test_mesh_points_and_reductions():
    pts = kmesh.monkhorst_pack((2, 2, 1))
    assert sorted(tuple(float(x) for x in p) for p in pts) == [(-0.25, -0.25, 0.0), (-0.25, 0.25, 0.0),
                                                             (0.25, -0.25, 0.0), (0.25, 0.25, 0.0)]
    k, w = kmesh.reduce_mesh(pts, (), time_reversal=False)
    assert len(k) == 4 and np.allclose(w, 0.25)
    k, w = kmesh.reduce_mesh(pts, (), time_reversal=True)  # k and -k pair up
    assert len(k) == 2 and np.allclose(w, 0.5)
    k, w = kmesh.reduce_mesh(pts, (1, 2, 3), time_reversal=True)  # mirrors x, y: one star
    assert len(k) == 1 and np.allclose(w, 1.0)
    # an odd mesh holds Gamma, its own partner under time reversal
    k, w = kmesh.reduce_mesh(kmesh.monkhorst_pack((3, 3, 1)), (), time_reversal=True)
    assert len(k) == 5 and abs(w.sum() - 1) < 1e-15 and np.allclose(sorted(w), [1 / 9] + [2 / 9] * 4)


def test_symmetry_operations_of_the_cells():
    wl = workloads.two_layer_slab_small()
    for s in wl.subsystems:
        assert kmesh.symmetry_ops(wl.lattice, s.pos, s.Z) == [0, 1, 2, 3]
    mol = workloads.molecule_on_slab_small()
    allpos = np.concatenate([s.pos for s in mol.subsystems])
    allZ = np.concatenate([s.Z for s in mol.subsystems])
    assert kmesh.symmetry_ops(mol.lattice, allpos, allZ) == [0]  # the seeded molecule breaks them


def test_symmetrize_is_a_projector():
    rng = np.random.default_rng(2)
    f = rng.standard_normal((6, 8, 5))
    g = kmesh.symmetrize(f, [0, 1, 2, 3])
    assert np.allclose(kmesh.symmetrize(g, [0, 1, 2, 3]), g, atol=1e-15)
    assert np.allclose(g, g[(-np.arange(6)) % 6][:, (-np.arange(8)) % 8], atol=1e-15)
    assert abs(g.sum() - f.sum()) < 1e-12


def test_reduced_mesh_gives_the_full_mesh_density():
    """A layer of the two-layer slab in the (mirror-symmetric) potential of the starting
    densities: eigenpairs on the full 2 x 2 x 1 mesh, and on the single irreducible point with
    its density averaged over the mirror group, give the same Methfessel-Paxton occupations,
    chemical potential, entropy term and density."""
    wl = workloads.two_layer_slab_small()
    sy = ofde.System(wl)
    rhos = np.array([workloads.initial_density(wl, I) for I in range(wl.nsub)])
    v = sy.build_veff(rhos)["veff"][0]
    s = wl.subsystems[0]
    eig, vec = [], []
    for k in range(s.nk):
        w, c = scf.eig_dense(sy, 0, k, v, s.nbands)
        eig.append(w)
        vec.append(c)
    occ, mu, S = scf.occupations(eig, s.wk, s.nelec, s.smearing, s.smearing_kind)
    full = sy.density(0, vec, occ)
    kr, wr = kmesh.reduce_mesh(kmesh.monkhorst_pack((2, 2, 1)), (1, 2, 3))
    red = workloads.with_kpoints(wl, 0, kr, wr)
    sr = ofde.System(red)
    w0, c0 = scf.eig_dense(sr, 0, 0, v, s.nbands)
    occ_r, mu_r, S_r = scf.occupations([w0], wr, s.nelec, s.smearing, s.smearing_kind)
    for e in eig:  # every mesh point carries the same levels
        assert np.abs(e - w0).max() < 1e-11
    assert abs(mu - mu_r) < 1e-12 and abs(S - S_r) < 1e-12
    rho_r = kmesh.symmetrize(sr.density(0, [c0], occ_r), [0, 1, 2, 3])
    assert np.abs(rho_r - full).max() < 1e-10 * np.abs(full).max()
    # without the averaging the single point's density is not the full one
    assert np.abs(sr.density(0, [c0], occ_r) - full).max() > 1e-6 * np.abs(full).max()
