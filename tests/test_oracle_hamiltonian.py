"""Pins of the oracle's density, embedded Hamiltonian, potentials and energies (CPU only)."""
import math

import numpy as np
import pytest

from oracle import basis, fde, functionals, potentials, scf
from paper_1406_7803_gb300 import workloads


@pytest.fixture(scope="module")
def mini():
    return fde.System(workloads.molecule_on_slab_small())


def _smooth_potential(sy, seed=5):
    """A smooth real potential: a few random Fourier modes."""
    rng = np.random.default_rng(seed)
    r = basis.grid_points(sy.lattice, sy.grid)
    B = basis.reciprocal(sy.lattice)
    v = np.full(sy.grid, -0.3)
    for _ in range(6):
        m = rng.integers(-3, 4, size=3)
        v += 0.2 * rng.standard_normal() * np.cos(r @ (m @ B) + rng.uniform(0, 6.28))
    return v


def _random_orbitals(sy, I, k, nb, seed=1):
    npw = sy.basis[I][k][0].shape[0]
    return sy.initial_orbitals(I, k, workloads.raw_orbitals(seed, I, k, nb, npw))


def test_plane_waves_are_kinetic_eigenvectors(mini):
    """With v_eff = 0 and no projectors, e^{i(k+G0).r} is an exact eigenvector with
    eigenvalue |k+G0|^2/2 (Eq. KS)."""
    sy = mini
    saved = sy.proj[0][1]
    sy.proj[0][1] = np.zeros((0, saved.shape[1]))
    try:
        mil, kin = sy.basis[0][1]
        for j in (0, 17, mil.shape[0] - 1):
            c = np.zeros((1, mil.shape[0]), dtype=complex)
            c[0, j] = 1.0
            h = sy.apply_h(0, 1, c, np.zeros(sy.grid))
            assert np.allclose(h, kin[j] * c, atol=1e-14)
        B = basis.reciprocal(sy.lattice)
        k = basis.kcart(sy.lattice, sy.subs[0].kpts[1])
        assert np.allclose(kin, 0.5 * np.sum((k + mil @ B) ** 2, 1), rtol=1e-14)
    finally:
        sy.proj[0][1] = saved


def test_dense_equals_fft_apply(mini):
    """The FFT form reproduces the plain dense H_{GG'} (wrap-around included)."""
    sy = mini
    v = _smooth_potential(sy)
    for I, k in ((0, 2), (1, 0)):
        c = _random_orbitals(sy, I, k, 3)
        H = sy.dense_h(I, k, v)
        a = sy.apply_h(I, k, c, v)
        b = (H @ c.T).T
        assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_constant_potential_shifts(mini):
    sy = mini
    c = _random_orbitals(sy, 0, 0, 2)
    h0 = sy.apply_h(0, 0, c, np.zeros(sy.grid))
    h1 = sy.apply_h(0, 0, c, np.full(sy.grid, 0.37))
    assert np.allclose(h1 - h0, 0.37 * c, atol=1e-13)


def test_hermiticity(mini):
    sy = mini
    v = _smooth_potential(sy, 9)
    c = _random_orbitals(sy, 0, 3, 2, seed=4)
    hc = sy.apply_h(0, 3, c, v)
    lhs = np.vdot(c[0], hc[1])
    rhs = np.conj(np.vdot(c[1], hc[0]))
    assert abs(lhs - rhs) < 1e-13
    H = sy.dense_h(1, 0, v)
    assert np.abs(H - H.conj().T).max() < 1e-14


def test_projectors_are_subsystem_specific(mini):
    """H_I's nonlocal part holds only projectors of the atoms of I: moving an atom of J
    leaves H_I - V_loc unchanged."""
    sy = mini
    c = _random_orbitals(sy, 1, 0, 2)
    a = sy.apply_h(1, 0, c, np.zeros(sy.grid))
    wl2 = workloads.molecule_on_slab_small()
    wl2.subsystems[0].pos[0] += 0.3
    sy2 = fde.System(wl2)
    b = sy2.apply_h(1, 0, c, np.zeros(sy.grid))
    assert np.allclose(a, b, atol=1e-14)
    assert sy.proj[1][0].shape[0] == 2 * sy.subs[1].natoms


def test_density_brute_force(mini):
    """rho_I on grid points equals 2 sum_k w_k sum_j n_jk |Omega^{-1/2} sum_G c_G e^{iG.r}|^2
    summed directly, and integrates to N_I."""
    sy = mini
    I = 0
    s = sy.subs[I]
    coefs = [_random_orbitals(sy, I, k, s.nbands, seed=2) for k in range(s.nk)]
    occ = [np.linspace(1.0, 0.2, s.nbands) for _ in range(s.nk)]
    rho = sy.density(I, coefs, occ)
    r = basis.grid_points(sy.lattice, sy.grid)
    B = basis.reciprocal(sy.lattice)
    for idx in ((0, 0, 0), (3, 7, 11), (23, 5, 59)):
        val = 0.0
        for k in range(s.nk):
            mil, _ = sy.basis[I][k]
            G = mil @ B
            u = coefs[k] @ np.exp(1j * G @ r[idx]) / math.sqrt(sy.omega)
            val += 2 * s.wk[k] * np.sum(occ[k] * np.abs(u) ** 2)
        assert np.isclose(rho[idx], val, rtol=1e-12)
    N = 2 * sum(s.wk[k] * occ[k].sum() for k in range(s.nk))
    assert np.isclose(basis.integrate(rho, sy.lattice), N, rtol=1e-12)


def _state(sy, seed=3):
    return scf.initial_state(sy, seed, density="orbitals")


def test_veff_recast_equals_embedding_form(mini):
    """V_eN + V_H[rho] + V_XC[rho_I] + V_kin^nad + V_XC^nad (recast) equals
    V_eN^I + V_H[rho_I] + V_XC[rho_I] + V_emb^I (Eq. embedding), pointwise."""
    sy = mini
    st = _state(sy)
    a = sy.build_veff(st.rhos)["veff"]
    b = sy.build_veff_embedding_form(st.rhos)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-11


def test_energy_forms_agree(mini):
    """E_FDE direct (Eq. E_FDE) = fragment recast with E_H^nad restored = band energy +
    deband recast, for any orthonormal orbitals with eigenvalues taken as Rayleigh quotients;
    and the Hartree energy by the subsystem recast equals E_H[rho]."""
    sy = mini
    st = _state(sy)
    pot = sy.build_veff(st.rhos)
    eigs = []
    for I, s in enumerate(sy.subs):
        ek = []
        for k in range(s.nk):
            c = st.coefs[I][k]
            hc = sy.apply_h(I, k, c, pot["veff"][I])
            ek.append(np.real(np.sum(c.conj() * hc, axis=1)))
        eigs.append(ek)
    en = sy.energies(st.coefs, st.occ, st.rhos, pot=pot, eigs_all=eigs, veff_used=pot["veff"])
    assert abs(en["E_fde"] - en["E_fde_fragments"]) < 1e-10
    assert abs(en["E_fde"] - en["E_fde_band"]) < 1e-10
    # Hartree recast: 1/2 sum_I [int V_H[rho_I] rho_I + int V_H^{I,emb} rho_I] = E_H[rho]
    vH = [potentials.hartree(r, sy.lattice)[0] for r in st.rhos]
    tot = 0.0
    for I in range(len(vH)):
        emb = sum(vH[J] for J in range(len(vH)) if J != I)
        tot += 0.5 * float(basis.integrate((vH[I] + emb) * st.rhos[I], sy.lattice))
    assert abs(tot - en["E_H"]) < 1e-11


def test_single_subsystem_is_plain_ks():
    """N_S = 1: every nonadditive term vanishes and V_eff = V_eN + V_H + V_XC."""
    wl = workloads.plain_fde_32()
    one = workloads.Workload(name="one", lattice=wl.lattice, grid=wl.grid, ecut=wl.ecut,
                             subsystems=[workloads.Subsystem(
                                 "all", np.concatenate([s.pos for s in wl.subsystems]),
                                 np.concatenate([s.Z for s in wl.subsystems]), 0.5, 8,
                                 wl.subsystems[0].kpts, wl.subsystems[0].wk, 16.0, 0.0)],
                             xc=wl.xc, kedf=wl.kedf, seed=wl.seed, tol=wl.tol)
    sy = fde.System(one)
    st = scf.initial_state(sy, density="orbitals")
    pot = sy.build_veff(st.rhos)
    en = sy.energies(st.coefs, st.occ, st.rhos, pot=pot)
    assert en["T_nad"] == 0.0 and abs(en["E_xc_nad"]) < 1e-14 and abs(en["E_H_nad"]) < 1e-14
    vH, _ = potentials.hartree(st.rhos[0], sy.lattice)
    _, vxc = functionals.xc(st.rhos[0], sy.lattice, one.xc)
    assert np.abs(pot["veff"][0] - (sy.vloc + vH + vxc)).max() < 1e-12


def test_total_density_is_sum(mini):
    sy = mini
    st = _state(sy)
    pot = sy.build_veff(st.rhos)
    assert np.allclose(pot["rho"], st.rhos[0] + st.rhos[1], rtol=0, atol=1e-15)
    N = sum(s.nelec for s in sy.subs)
    assert np.isclose(basis.integrate(pot["rho"], sy.lattice), N, rtol=1e-12)


def _gauss_overlap(s1, s2, d2):
    """<g_s1(. - A)|g_s2(. - B)> of unit-norm Gaussians (pi^{3/2} s^3)^{-1/2} exp(-r^2/(2 s^2)),
    |A - B|^2 = d2 (Gaussian product theorem)."""
    w = s1 * s1 + s2 * s2
    return (2.0 * s1 * s2 / w) ** 1.5 * math.exp(-d2 / (2.0 * w))


def _gaussian_cell(**uspp):
    """One Bloch-summed unit-norm Gaussian orbital (width 0.8 bohr, centred on atom A) in a 9
    bohr cube at a general k-point, sampled in real space and transformed with numpy's FFT
    (not the oracle's), and the closed-form projections <beta_ai|psi> = sum_T e^{ik.T}
    <g_sigma_i(. - R_a)|g(. - R_A - T)> (Gaussian product theorem) on both atoms."""
    L, n, sig = 9.0, 64, 0.8
    lat = np.diag([L] * 3)
    kfrac = np.array([0.1, 0.2, 0.3])
    RA = np.array([1.0, 2.0, 3.0])
    RB = RA + np.array([4.5, 0.3, -0.2])
    sub = workloads.Subsystem("pair", np.array([RA, RB]), np.array([1.0, 1.0]), 0.5, 1,
                              kfrac[None, :], np.ones(1), 2.0, 0.0,
                              workloads.KB_SIGMA, workloads.KB_D, **uspp)
    wl = workloads.Workload(name="gauss", lattice=lat, grid=(n, n, n), ecut=40.0, subsystems=[sub],
                            xc=workloads.XC_LDA, kedf=workloads.KEDF_TF, seed=0, tol=1e-6)
    sy = fde.System(wl)
    kc = 2.0 * math.pi * kfrac / L
    x = np.arange(n) * (L / n)
    r = np.stack(np.meshgrid(x, x, x, indexing="ij"), axis=-1)
    psi = np.zeros((n, n, n), dtype=np.complex128)
    for t in np.ndindex(3, 3, 3):
        T = (np.array(t) - 1) * L
        d2 = ((r - RA - T) ** 2).sum(-1)
        psi += np.exp(1j * kc @ T) * (math.pi ** 1.5 * sig ** 3) ** -0.5 * np.exp(-d2 / (2 * sig * sig))
    u = np.exp(-1j * (r @ kc)) * psi  # the periodic part
    F = np.fft.fftn(u) * math.sqrt(L ** 3) / n ** 3  # c_G = Omega^{-1/2} int u e^{-iG.r}
    mil, _ = sy.basis[0][0]
    c = F[mil[:, 0] % n, mil[:, 1] % n, mil[:, 2] % n][None, :]
    P = np.zeros((2, len(workloads.KB_SIGMA)), dtype=np.complex128)
    for a, Ra in enumerate((RA, RB)):
        for i, si in enumerate(workloads.KB_SIGMA):
            for t in np.ndindex(5, 5, 5):
                T = (np.array(t) - 2) * L
                P[a, i] += np.exp(1j * kc @ T) * _gauss_overlap(si, sig, float(((RA + T - Ra) ** 2).sum()))
    return sy, c, P, sig


def test_kinetic_and_nonlocal_energy_of_an_atom_centred_gaussian():
    """<psi|H|psi> with v_eff = 0 for the Gaussian orbital of the cell above: the kinetic part
    is 3/(4 sigma^2) and the nonlocal part sum_a P_a^H D P_a.  The second atom, 4.5 bohr away,
    has two nearly equidistant images, so a wrong sign of the projector phase, a dropped atom,
    a transposed coupling or a missing 1/2 in the kinetic term fails here."""
    sy, c, P, sig = _gaussian_cell()
    n = sy.grid[0]
    assert abs(np.sum(np.abs(c) ** 2) - 1.0) < 1e-10  # the sphere holds the whole Gaussian
    hc = sy.apply_h(0, 0, c, np.zeros((n, n, n)))
    e = np.vdot(c, hc)
    assert abs(e.imag) < 1e-12
    want_kin = 3.0 / (4.0 * sig * sig)
    D = np.array(workloads.KB_D)
    want_nl = float(sum(np.real(np.vdot(Pa, D @ Pa)) for Pa in P))
    kin_only = np.vdot(c, sy.basis[0][0][1][None, :] * c).real
    assert abs(kin_only - want_kin) < 1e-10, (kin_only, want_kin)
    assert abs(e.real - (want_kin + want_nl)) < 1e-10, (e.real - want_kin, want_nl)


def test_overlap_of_an_atom_centred_gaussian():
    """<psi|S|psi> = 1 + sum_a P_a^H q P_a for the ultrasoft-like model (Appendix, subsystem-
    specific projectors) with the off-diagonal q of the synthetic cells, and with v_eff = 0 the
    screening vanishes so H keeps the bare coupling D."""
    q = np.array(workloads.USPP_Q)
    sy, c, P, sig = _gaussian_cell(proj_Q=workloads.USPP_Q, aug_sigma=workloads.USPP_SIGMA)
    n = sy.grid[0]
    sc = sy.apply_s(0, 0, c)
    want = 1.0 + float(sum(np.real(np.vdot(Pa, q @ Pa)) for Pa in P))
    got = np.vdot(c, sc)
    assert abs(got.imag) < 1e-12 and abs(got.real - want) < 1e-10, (got, want)
    D = np.array(workloads.KB_D)
    e = np.vdot(c, sy.apply_h(0, 0, c, np.zeros((n, n, n)))).real
    want_h = 3.0 / (4.0 * sig * sig) + float(sum(np.real(np.vdot(Pa, D @ Pa)) for Pa in P))
    assert abs(e - want_h) < 1e-10
