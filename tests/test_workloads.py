"""The synthetic cells are what the design notes say they are (CPU only): sizes, atom counts,
charges, band counts, k-point sets and weights, electron counts, and the placement rules of the
seeded atoms (minimum separations, molecules in the vacuum above the slab).  These inputs
stand in for the paper's molecule-on-metal systems (Table 1), so their recipe is checked here
rather than trusted."""
import numpy as np
import pytest

from paper_1406_7803_gb300 import workloads


def _min_sep(pos, L):
    d = pos[:, None, :] - pos[None, :, :]
    d -= np.round(d / L) * L
    r = np.sqrt((d ** 2).sum(-1))
    r[np.diag_indices(len(pos))] = np.inf
    return r.min()


def _check_common(wl):
    for s in wl.subsystems:
        assert abs(s.wk.sum() - 1.0) < 1e-14
        assert s.kpts.shape == (s.nk, 3)
        assert 2 * s.nbands >= s.nelec  # every electron fits the bands
        assert s.pos.shape == (s.natoms, 3) and np.all(np.isfinite(s.pos))


def test_plain_fde_cell():
    wl = workloads.plain_fde_32()
    _check_common(wl)
    assert wl.grid == (32, 32, 32) and wl.ecut == 15.0 and wl.nsub == 2
    allpos = np.concatenate([s.pos for s in wl.subsystems])
    assert _min_sep(allpos, np.diag(wl.lattice)) >= 1.5
    for s in wl.subsystems:
        assert s.natoms == 3 and np.all(s.Z == 2.0) and s.nbands == 4 and s.nelec == 8.0 and s.nk == 1


@pytest.mark.parametrize("make,layers,per,bands,mol_atoms,mol_bands",
                         [(workloads.molecule_on_slab, 4, 9, 64, 6, 12),
                          (workloads.molecule_on_slab_small, 2, 4, 16, 2, 4)])
def test_molecule_on_slab_cells(make, layers, per, bands, mol_atoms, mol_bands):
    wl = make()
    _check_common(wl)
    slab, mol = wl.subsystems
    assert slab.natoms == layers * per and np.all(slab.Z == 3.0) and slab.nbands == bands
    assert slab.nk == 4 and np.allclose(slab.wk, 0.25) and slab.smearing == 0.01
    assert slab.nelec == 3.0 * slab.natoms
    assert mol.natoms == mol_atoms and np.all(mol.Z == 4.0) and mol.nbands == mol_bands and mol.nk == 1
    assert mol.smearing == 0.0 and mol.nelec == 2 * mol.nbands  # closed shell, integer filling
    # the molecule sits in the vacuum above the slab's top layer, around 5 bohr up
    top = slab.pos[:, 2].max()
    assert np.all(mol.pos[:, 2] > top + 2.0)
    assert abs(mol.pos[:, 2].mean() - (top + 5.0)) < 2.5


def test_batched_uneven_cell():
    wl = workloads.batched_uneven()
    _check_common(wl)
    L = np.diag(wl.lattice)
    assert wl.grid == (96, 96, 96) and wl.ecut == 20.0 and wl.nsub == 17
    slab = wl.subsystems[0]
    assert slab.natoms == 54 and slab.nbands == 96 and slab.nk == 2
    bands = [s.nbands for s in wl.subsystems[1:]]
    assert min(bands) >= 8 and max(bands) <= 64
    top = slab.pos[:, 2].max()
    centres = np.array([s.pos.mean(axis=0) for s in wl.subsystems[1:]])
    assert np.all(centres[:, 2] > top)
    # positions are periodic: atoms of different subsystems never overlap under minimum image
    allpos = np.concatenate([s.pos for s in wl.subsystems])
    assert _min_sep(allpos, L) > 0.5
    for s in wl.subsystems[1:]:
        assert s.natoms == s.nbands // 2 and np.all(s.Z == 4.0) and s.nelec == 4.0 * s.natoms


def test_large_cell():
    wl = workloads.large_cell()
    _check_common(wl)
    L = np.diag(wl.lattice)
    assert wl.grid == (144, 144, 288) and wl.ecut == 25.0 and wl.nsub == 33
    slab = wl.subsystems[0]
    assert slab.natoms == 216 and slab.nbands == 512 and slab.nk == 8 and np.allclose(slab.wk, 1 / 8)
    bands = [s.nbands for s in wl.subsystems[1:]]
    assert min(bands) >= 16 and max(bands) <= 48
    assert wl.band_k_pairs() == 512 * 8 + sum(bands) == 5209
    centres = np.array([s.pos.mean(axis=0) for s in wl.subsystems[1:]])
    assert np.all(centres[:, 2] > slab.pos[:, 2].max())
    allpos = np.concatenate([s.pos for s in wl.subsystems])
    assert _min_sep(allpos, L) > 0.5


def test_two_layer_slab_and_ultrasoft_cells():
    wl = workloads.two_layer_slab_small()
    _check_common(wl)
    assert wl.nsub == 2 and all(s.smearing_kind == "mp" and s.nk == 4 for s in wl.subsystems)
    # each layer is mirror-symmetric in x and y about the origin (the symmetry reduction's premise)
    L = np.diag(wl.lattice)
    for s in wl.subsystems:
        for axis in (0, 1):
            m = s.pos.copy()
            m[:, axis] = (-m[:, axis]) % L[axis]
            d = np.abs(np.sort(m, axis=0) - np.sort(s.pos, axis=0))
            assert np.all(np.minimum(d, L - d) < 1e-12)
    us = workloads.uspp_small()
    for s in us.subsystems:
        assert s.aug_sigma == workloads.USPP_SIGMA and np.allclose(s.proj_Q, workloads.USPP_Q)
        assert np.all(np.linalg.eigvalsh(np.array(s.proj_Q)) > 0)  # S = 1 + positive


def test_supersystem_holds_every_atom_and_electron():
    wl = workloads.molecule_on_slab_small()
    sup = workloads.supersystem(wl, extra_bands=2)
    (s,) = sup.subsystems
    assert s.natoms == sum(t.natoms for t in wl.subsystems)
    assert s.nelec == sum(t.nelec for t in wl.subsystems)
    assert s.nbands == sum(t.nbands for t in wl.subsystems) + 2
    assert s.nk == wl.subsystems[0].nk and s.smearing == wl.subsystems[0].smearing


def test_seeded_draws_are_reproducible():
    a = workloads.raw_orbitals(5, 1, 0, 4, 100)
    b = workloads.raw_orbitals(5, 1, 0, 4, 100)
    c = workloads.raw_orbitals(5, 1, 1, 4, 100)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    wl = workloads.molecule_on_slab_small()
    rho = workloads.initial_density(wl, 0)
    omega = abs(np.linalg.det(wl.lattice))
    assert abs(rho.sum() * omega / rho.size - wl.subsystems[0].nelec) < 1e-9
    assert np.all(rho >= 0)
