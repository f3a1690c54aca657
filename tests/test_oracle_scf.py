"""Pins of the oracle's occupations, eigensolver and self-consistency loops (CPU only)."""
import numpy as np
import pytest

from oracle import basis, fde, scf
from paper_1406_7803_gb300 import workloads


def test_fermi_occupations_count_and_entropy():
    rng = np.random.default_rng(0)
    eigs = [np.sort(rng.uniform(-1, 1, 20)) for _ in range(4)]
    wk = np.full(4, 0.25)
    occ, mu, S = scf.occupations(eigs, wk, 17.0, 0.01)
    N = sum(2 * w * o.sum() for w, o in zip(wk, occ))
    assert abs(N - 17.0) < 1e-12
    assert all(np.all((o >= 0) & (o <= 1)) for o in occ)
    # entropy by its definition, term by term
    Sd = 0.0
    for w, o in zip(wk, occ):
        for n in o:
            if 0 < n < 1:
                Sd -= 2 * w * (n * np.log(n) + (1 - n) * np.log(1 - n))
    assert np.isclose(S, Sd, rtol=1e-12, atol=1e-14)


def test_fermi_zero_width_limit_is_integer_filling():
    e = [np.array([-0.5, -0.2, 0.1, 0.4, 0.9])]
    occ, mu, S = scf.occupations(e, np.ones(1), 6.0, 1e-5)
    assert np.allclose(occ[0], [1, 1, 1, 0, 0], atol=1e-12)
    occ_i, _, S_i = scf.occupations(e, np.ones(1), 6.0, 0.0)
    assert np.allclose(occ_i[0], [1, 1, 1, 0, 0]) and S_i == 0.0


@pytest.fixture(scope="module")
def mini():
    return fde.System(workloads.molecule_on_slab_small())


def test_lanczos_matches_dense_eigh(mini):
    sy = mini
    st = scf.initial_state(sy)
    pot = sy.build_veff(st.rhos)
    for I, k in ((0, 1), (1, 0)):
        nb = sy.subs[I].nbands
        wd, vd = scf.eig_dense(sy, I, k, pot["veff"][I], nb)
        wl, vl = scf.eig_lanczos(sy, I, k, pot["veff"][I], nb)
        assert np.abs(wd - wl).max() < 1e-10
        # the spanned subspaces agree (projector comparison is phase- and degeneracy-safe)
        Pd = vd.T @ vd.conj()
        Pl = vl.T @ vl.conj()
        assert np.abs(Pd - Pl).max() < 1e-7
        # residuals of the dense pairs
        hv = sy.apply_h(I, k, vd, pot["veff"][I])
        assert np.abs(hv - wd[:, None] * vd).max() < 1e-10


def test_subsystem_scf_fixed_point(mini):
    """The molecule's SCF in the frozen slab density is self-consistent and, at
    self-consistency, the band-energy form of E_FDE equals the direct form."""
    sy = mini
    st = scf.initial_state(sy)
    r = scf.solve_subsystem(sy, 1, st.rhos, st.rhos[1], st.coefs[1], 1e-10, dense_max=2000,
                            others=(st.coefs, st.occ, st.entropy))
    assert r["converged"]
    rhos = st.rhos.copy()
    rhos[1] = r["rho"]
    pot = sy.build_veff(rhos)
    w, v = scf.eig_dense(sy, 1, 0, pot["veff"][1], sy.subs[1].nbands)
    assert np.abs(w - r["eigs"][0]).max() < 1e-5
    coefs = [st.coefs[0], [v]]
    occ = [st.occ[0], r["occ"]]
    rhos[1] = sy.density(1, [v], r["occ"])
    en = sy.energies(coefs, occ, rhos, eigs_all=[st.eigs[0], [w]], veff_used=[pot["veff"][0], pot["veff"][1]])
    # the slab's orbitals carry no eigenvalues here; compare the molecule's part only
    assert abs(en["E_fde"] - en["E_fde_fragments"]) < 1e-10
    rq = np.real(np.sum(v.conj() * sy.apply_h(1, 0, v, pot["veff"][1]), axis=1))
    assert np.allclose(rq, w, atol=1e-10)


@pytest.mark.slow
def test_freeze_thaw_cycle_plain_fde_32():
    """One Jacobi freeze-and-thaw cycle on the 2 x 3-atom LDA + TF cell converges every
    subsystem SCF and leaves the three energy forms in agreement."""
    sy = fde.System(workloads.plain_fde_32())
    st = scf.initial_state(sy)
    new, en = scf.freeze_thaw_cycle(sy, st)
    assert en["converged"]
    assert abs(en["E_fde"] - en["E_fde_fragments"]) < 1e-10
    for I, s in enumerate(sy.subs):
        assert np.isclose(basis.integrate(new.rhos[I], sy.lattice), s.nelec, rtol=1e-12)
    pot = sy.build_veff(new.rhos)
    # orbitals are eigenvectors of the potential built from the cycle-start densities of
    # the other subsystem, so only their own eigen-residual is small against that one
    assert np.isfinite(en["E_fde"])
