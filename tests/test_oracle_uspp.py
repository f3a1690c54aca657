"""Pins of the oracle's ultrasoft-like subsystems (CPU only): overlap operator, generalised
eigenproblem, augmented density and the screened coupling (Appendix: subsystem-specific
PAW / ultrasoft projectors, with the model augmentation of workloads.uspp_small)."""
import dataclasses

import numpy as np
import pytest

from oracle import basis, fde as ofde, scf
from paper_1406_7803_gb300 import workloads


def _tiny_uspp():
    """The ultrasoft-like slab + molecule cell at a lower cutoff (dense eigensolves in seconds)."""
    return dataclasses.replace(workloads.uspp_small(), ecut=4.0, name="uspp-tiny")


@pytest.fixture(scope="module")
def cell():
    wl = _tiny_uspp()
    sy = ofde.System(wl)
    rhos = np.array([workloads.initial_density(wl, I) for I in range(wl.nsub)])
    pot = sy.build_veff(rhos)
    return wl, sy, rhos, pot


def test_overlap_is_hermitian_positive_and_inverted_exactly(cell):
    wl, sy, _, _ = cell
    for I in range(wl.nsub):
        S = sy.dense_s(I, 0)
        assert np.abs(S - S.conj().T).max() < 1e-14
        w = np.linalg.eigvalsh(S)
        assert w.min() > 1 - 1e-12 and w.max() > 1.05  # q > 0: S = 1 + positive
        # the Woodbury inverse the Lanczos solver uses
        B = sy.proj[I][0].conj()
        inner = np.linalg.inv(np.linalg.inv(sy.Qmat[I]) + B @ B.conj().T)
        Sinv = np.eye(S.shape[0]) - B.conj().T @ inner @ B
        assert np.abs(S @ Sinv - np.eye(S.shape[0])).max() < 1e-10


@pytest.mark.parametrize("I,k", [(0, 1), (1, 0)])
def test_generalised_eigenpairs_dense_equal_lanczos(cell, I, k):
    wl, sy, _, pot = cell
    nb = wl.subsystems[I].nbands
    wd, vd = scf.eig_dense(sy, I, k, pot["veff"][I], nb)
    wl_, vl = scf.eig_lanczos(sy, I, k, pot["veff"][I], nb)
    assert np.abs(wd - wl_).max() < 1e-9
    for v in (vd, vl):
        G = v.conj() @ sy.apply_s(I, k, v).T  # S-orthonormal
        assert np.abs(G - np.eye(nb)).max() < 1e-9
        r = sy.apply_h(I, k, v, pot["veff"][I]) - (wd[:, None] * sy.apply_s(I, k, v))
        assert np.abs(r).max() < 1e-8


def test_augmented_density_holds_every_electron(cell):
    wl, sy, _, pot = cell
    for I, s in enumerate(wl.subsystems):
        eigs, vecs = [], []
        for k in range(s.nk):
            w, v = scf.eig_dense(sy, I, k, pot["veff"][I], s.nbands)
            eigs.append(w)
            vecs.append(v)
        occ, _, _ = scf.occupations(eigs, s.wk, s.nelec, s.smearing, s.smearing_kind)
        rho = sy.density(I, vecs, occ)
        assert abs(basis.integrate(rho, sy.lattice) - s.nelec) < 1e-10
        # without the augmentation the smooth part alone falls short
        smooth = sum(2 * s.wk[k] * np.einsum("j,jxyz->xyz", occ[k], np.abs(sy.orbitals_r(I, k, vecs[k])) ** 2)
                     for k in range(s.nk))
        assert basis.integrate(smooth, sy.lattice) < s.nelec - 0.05


def test_band_energy_form_needs_the_screened_coupling(cell):
    """For eigenpairs of H built from v_eff, sum f e - int v_eff rho equals T + E_NL (bare D)
    only if the augmentation charges in rho and the screening q int v_eff g_a in H match: the
    band-energy form of the total energy then equals the direct form."""
    wl, sy, rhos, pot = cell
    coefs, occs, eigs = [], [], []
    for I, s in enumerate(wl.subsystems):
        ck, ek = [], []
        for k in range(s.nk):
            w, v = scf.eig_dense(sy, I, k, pot["veff"][I], s.nbands)
            ck.append(v)
            ek.append(w)
        oc, _, _ = scf.occupations(ek, s.wk, s.nelec, s.smearing, s.smearing_kind)
        coefs.append(ck)
        occs.append(oc)
        eigs.append(ek)
    new = np.array([sy.density(I, coefs[I], occs[I]) for I in range(wl.nsub)])
    en = sy.energies(coefs, occs, new, eigs_all=eigs, veff_used=pot["veff"])
    # E_fde_band uses the eigenvalues of H[v_eff(start)] and -int v_eff(start) rho(new):
    # equal to the direct form up to the change of the grid terms between the two densities
    grid_new = sy.energies(coefs, occs, new)
    band_part = sum(2 * s.wk[k] * float(np.sum(occs[I][k] * eigs[I][k]))
                    for I, s in enumerate(wl.subsystems) for k in range(s.nk))
    deband = -sum(float(basis.integrate(pot["veff"][I] * new[I], sy.lattice)) for I in range(wl.nsub))
    assert abs((band_part + deband) - (grid_new["E_kin"] + grid_new["E_nl"])) < 1e-9
    assert np.isfinite(en["E_fde_band"])


def test_zero_augmentation_is_the_norm_conserving_cell(cell):
    wl, sy, _, pot = cell
    q0 = dataclasses.replace(wl, subsystems=[dataclasses.replace(s, proj_Q=((0.0, 0.0), (0.0, 0.0)))
                                             for s in wl.subsystems])
    plain = dataclasses.replace(wl, subsystems=[dataclasses.replace(s, proj_Q=(), aug_sigma=0.0)
                                                for s in wl.subsystems])
    s0, sp = ofde.System(q0), ofde.System(plain)
    w0, _ = np.linalg.eigh(s0.dense_h(1, 0, pot["veff"][1]))[0][:4], None
    wp, _ = np.linalg.eigh(sp.dense_h(1, 0, pot["veff"][1]))[0][:4], None
    assert np.abs(w0 - wp).max() < 1e-12
