"""Subsystem densities, embedded Kohn-Sham Hamiltonian and FDE energy.

Test infrastructure only (see ``oracle/__init__.py``).

* rho = sum_I rho_I on one shared grid (Eq. int1 / meth:1).
* rho_I = 2 sum_k w_k sum_j n_jk |u_jk(r)|^2 (Sec. 2, subsystem density with a BZ
  integral and fractional occupations; the BZ integral is the weighted k-sum).
* V_eff^I = V_eN (all nuclei) + V_H[rho] + V_XC[rho_I] + V_kin^nad + V_XC^nad
  (Appendix, recast effective potential), with V_XC[rho_I] + V_XC^nad = V_XC[rho] and
  V_kin^nad = v~_kin[rho] - v~_kin[rho_I].  The equivalent V_KS^I + V_emb^I form
  (Eq. embedding) is also provided, for the pin that the two agree.
* H_I u = [-(1/2)(grad + ik)^2 + V_eff^I] u (Eq. KS) plus the nonlocal projectors of
  the atoms of I only (Appendix, subsystem-specific projectors).  Both the plain dense
  matrix H_{GG'} and the FFT form P_sphere FFT[v . IFFT psi] are given.
* E_FDE (Eq. for E_FDE): sum_I {T_J[rho_I] + E_NL^I} + int v_loc rho + E_H[rho]
  + E_XC[rho] + T^nad + V_NN, and the two recast forms of the Appendix (fragment
  energies E_K, and band energies plus "deband"), the latter with E_H^nad restored
  (reading: the printed recast omits it).
"""
from __future__ import annotations

import numpy as np

from . import basis, functionals, potentials


class System:
    """Everything that depends only on the geometry: grid, spheres, potentials."""

    def __init__(self, wl):
        self.wl = wl
        self.lattice = np.asarray(wl.lattice, dtype=np.float64)
        self.grid = tuple(int(n) for n in wl.grid)
        self.omega = basis.volume(self.lattice)
        self.nr = int(np.prod(self.grid))
        self.subs = wl.subsystems
        allpos = np.concatenate([s.pos for s in self.subs], axis=0)
        allZ = np.concatenate([s.Z for s in self.subs], axis=0)
        rcs = {s.rc for s in self.subs}
        if len(rcs) != 1:
            raise ValueError("one r_c per workload")
        self.rc = rcs.pop()
        self.vloc = potentials.vloc_r(self.lattice, self.grid, allpos, allZ, self.rc)
        self.vloc_sub = [potentials.vloc_r(self.lattice, self.grid, s.pos, s.Z, self.rc)
                         for s in self.subs]
        self.enn = potentials.ewald(self.lattice, allpos, allZ)
        self.basis = []  # [I][k] -> (miller, kin)
        self.proj = []  # [I][k] -> beta [nproj, npw]
        self.Dmat = []  # [I] -> block-diagonal coupling
        # [I] -> block-diagonal augmentation coefficients q of ultrasoft-like atoms (None: the
        # subsystem is norm-conserving)
        self.Qmat = [potentials.kb_coupling(s.natoms, s.proj_Q) if getattr(s, "aug_sigma", 0.0) > 0 else None
                     for s in self.subs]
        for s in self.subs:
            bk, pk = [], []
            for k in s.kpts:
                mil, kin = basis.sphere(self.lattice, self.grid, k, wl.ecut)
                bk.append((mil, kin))
                pk.append(potentials.kb_projectors(self.lattice, k, mil, s.pos, s.proj_sigma))
            self.basis.append(bk)
            self.proj.append(pk)
            self.Dmat.append(potentials.kb_coupling(s.natoms, s.proj_D))

    # ------------------------------------------------------------ orbitals
    def initial_orbitals(self, I, k, raw):
        """Initial guess from raw complex draws: c_G = raw_G / (1 + |k+G|^2/2), then
        orthonormalised (QR).  Only the spanned subspace matters downstream."""
        mil, kin = self.basis[I][k]
        c = raw / (1.0 + kin)[None, :]
        q, _ = np.linalg.qr(c.T)
        return q.T.copy()

    def orbitals_r(self, I, k, coef):
        """u_jk(r) on the grid, Omega^{-1/2} sum_G c_G e^{iG.r}."""
        mil, _ = self.basis[I][k]
        return basis.r_from_G(basis.to_grid(coef, mil, self.grid)) / np.sqrt(self.omega)

    def density(self, I, coefs, occ):
        """rho_I(r) = 2 sum_k w_k sum_j n_jk |u_jk(r)|^2, plus for ultrasoft-like atoms the
        augmentation sum_a g_a(r) sum_ij q_ij 2 sum_k w_k sum_j n_jk Re <u|beta_ai><beta_aj|u>
        (it makes int rho_I = N_I for S-normalised orbitals)."""
        s = self.subs[I]
        rho = np.zeros(self.grid)
        for k in range(s.nk):
            u = self.orbitals_r(I, k, coefs[k])
            rho += 2.0 * s.wk[k] * np.einsum("j,jxyz->xyz", occ[k], np.abs(u) ** 2)
        if self.uspp(I):
            npj = len(s.proj_sigma)
            q = np.asarray(s.proj_Q, dtype=np.float64)
            ca = np.zeros(s.natoms)
            for k in range(s.nk):
                P = self.proj[I][k].conj() @ np.atleast_2d(coefs[k]).T  # [natoms * npj, nb]
                for a in range(s.natoms):
                    Pa = P[a * npj:(a + 1) * npj]
                    B = np.real(Pa.conj() @ (occ[k][:, None] * Pa.T))  # sum_j n_j conj(P_i) P_i'
                    ca[a] += 2.0 * s.wk[k] * float(np.sum(q * B))
            rho += np.real(basis.r_from_G(potentials.augmentation_G(self.lattice, self.grid, s.pos, ca,
                                                                       s.aug_sigma)))
        return rho

    # ------------------------------------------------------------ potentials
    def build_veff(self, rhos):
        """Recast effective potentials V_eff^I for every subsystem, plus the pieces the
        energy needs."""
        wl = self.wl
        rho = np.sum(rhos, axis=0)
        vH, EH = potentials.hartree(rho, self.lattice)
        Exc, vxc = functionals.xc(rho, self.lattice, wl.xc, wl.rho_cut)
        Tk, vk = functionals.kinetic(rho, self.lattice, wl.kedf, wl.rho_cut)
        veff, TkI = [], []
        common = self.vloc + vH + vxc + vk
        for rI in rhos:
            t, v = functionals.kinetic(rI, self.lattice, wl.kedf, wl.rho_cut)
            TkI.append(t)
            veff.append(common - v)
        return dict(rho=rho, vH=vH, EH=EH, Exc=Exc, vxc=vxc, Tk=Tk, vk=vk, TkI=TkI, veff=veff)

    def build_veff_embedding_form(self, rhos):
        """V_eff^I = V_eN^I + V_H[rho_I] + V_XC[rho_I] + V_emb^I with V_emb^I of
        Eq. embedding (subsystem-resolved Hartree and nuclear terms)."""
        wl = self.wl
        rho = np.sum(rhos, axis=0)
        vH = [potentials.hartree(r, self.lattice)[0] for r in rhos]
        vxc_I = [functionals.xc(r, self.lattice, wl.xc, wl.rho_cut)[1] for r in rhos]
        vk_I = [functionals.kinetic(r, self.lattice, wl.kedf, wl.rho_cut)[1] for r in rhos]
        vxc_tot = functionals.xc(rho, self.lattice, wl.xc, wl.rho_cut)[1]
        vk_tot = functionals.kinetic(rho, self.lattice, wl.kedf, wl.rho_cut)[1]
        out = []
        for I in range(len(rhos)):
            vemb = np.zeros(self.grid)
            for J in range(len(rhos)):
                if J != I:
                    vemb += vH[J] + self.vloc_sub[J]
            vemb += vk_tot - vk_I[I] + vxc_tot - vxc_I[I]
            out.append(self.vloc_sub[I] + vH[I] + vxc_I[I] + vemb)
        return out

    # ------------------------------------------------------------ ultrasoft-like atoms
    def uspp(self, I):
        return self.Qmat[I] is not None and self.Qmat[I].size > 0

    def coupling(self, I, veff_I):
        """Nonlocal coupling of subsystem I: the bare D, plus for ultrasoft-like atoms the
        screening q_ij int v_eff^I g_a (the augmentation charges q_ij g_a sit in the density, so
        the energy's derivative by <psi|beta_i><beta_j|psi> picks up their potential energy)."""
        if not self.uspp(I):
            return self.Dmat[I]
        s = self.subs[I]
        ov = potentials.augmentation_overlaps(self.lattice, self.grid, s.pos, s.aug_sigma, veff_I)
        q = np.asarray(s.proj_Q, dtype=np.float64)
        return self.Dmat[I] + np.kron(np.diag(ov), q)

    def apply_s(self, I, k, coef):
        """S_I psi = psi + sum_{a in I} beta q <beta|psi> (identity for norm-conserving I)."""
        coef = np.atleast_2d(coef)
        if not self.uspp(I):
            return coef.copy()
        beta = self.proj[I][k]
        return coef + (beta.T @ (self.Qmat[I] @ (beta.conj() @ coef.T))).T

    def dense_s(self, I, k):
        npw = self.basis[I][k][0].shape[0]
        S = np.eye(npw, dtype=np.complex128)
        if self.uspp(I):
            beta = self.proj[I][k]
            S = S + beta.T @ self.Qmat[I] @ beta.conj()
        return S

    # ------------------------------------------------------------ Hamiltonian
    def apply_h(self, I, k, coef, veff_I, coupling=None):
        """H_I psi for a block of orbitals [nb, npw], FFT form:
        1/2|k+G|^2 c_G + P_sphere FFT[v_eff . IFFT c] + sum_{a in I} beta D <beta|psi>
        (D screened for ultrasoft-like atoms; ``coupling`` may pass it precomputed)."""
        mil, kin = self.basis[I][k]
        coef = np.atleast_2d(coef)
        psi_r = basis.r_from_G(basis.to_grid(coef, mil, self.grid))
        loc = basis.from_grid(basis.G_from_r(veff_I[None] * psi_r), mil, self.grid)
        out = kin[None, :] * coef + loc
        beta = self.proj[I][k]
        if beta.shape[0]:
            D = self.coupling(I, veff_I) if coupling is None else coupling
            P = beta.conj() @ coef.T
            out = out + (beta.T @ (D @ P)).T
        return out

    def dense_h(self, I, k, veff_I):
        """Plain definition H_{GG'} = 1/2|k+G|^2 delta_{GG'} + V~((m - m') mod n)
        + sum beta(G) D beta(G')^*, with V~ the grid transform of v_eff."""
        mil, kin = self.basis[I][k]
        vG = basis.G_from_r(veff_I)
        d = mil[:, None, :] - mil[None, :, :]
        H = vG[d[..., 0] % self.grid[0], d[..., 1] % self.grid[1], d[..., 2] % self.grid[2]]
        H = H + np.diag(kin)
        beta = self.proj[I][k]
        if beta.shape[0]:
            H = H + beta.T @ self.coupling(I, veff_I) @ beta.conj()
        return H

    # ------------------------------------------------------------ energies
    def band_terms(self, I, coefs, occ):
        """Janak kinetic energy T_J[rho_I] and nonlocal energy E_NL^I."""
        s = self.subs[I]
        T = 0.0
        Enl = 0.0
        for k in range(s.nk):
            mil, kin = self.basis[I][k]
            c = coefs[k]
            T += 2.0 * s.wk[k] * float(np.sum(occ[k][:, None] * kin[None, :] * np.abs(c) ** 2))
            beta = self.proj[I][k]
            if beta.shape[0]:
                P = beta.conj() @ c.T
                e = np.real(np.einsum("pj,pq,qj->j", P.conj(), self.Dmat[I], P))
                Enl += 2.0 * s.wk[k] * float(np.sum(occ[k] * e))
        return T, Enl

    def energies(self, coefs_all, occ_all, rhos, pot=None, eigs_all=None, veff_used=None,
                 entropy=None):
        """E_FDE and its terms for the given orbitals (per subsystem lists over k).

        If eigenvalues and the potentials they were computed with are given, also the
        band-energy ("deband") form.  ``entropy`` [nsub] gives sigma_I S_I of smeared
        subsystems for the Mermin free energy F = E - sum sigma S."""
        wl = self.wl
        if pot is None:
            pot = self.build_veff(rhos)
        rho = pot["rho"]
        nsub = len(rhos)
        T = np.zeros(nsub)
        Enl = np.zeros(nsub)
        for I in range(nsub):
            T[I], Enl[I] = self.band_terms(I, coefs_all[I], occ_all[I])
        Eloc = float(basis.integrate(self.vloc * rho, self.lattice))
        Tnad = pot["Tk"] - float(np.sum(pot["TkI"]))
        E = float(T.sum() + Enl.sum()) + Eloc + pot["EH"] + pot["Exc"] + Tnad + self.enn
        out = dict(E_fde=E, E_kin=float(T.sum()), E_nl=float(Enl.sum()), E_loc=Eloc,
                   E_H=pot["EH"], E_xc=pot["Exc"], T_nad=Tnad, E_nn=self.enn,
                   T_sub=T, Enl_sub=Enl)
        ts = 0.0 if entropy is None else float(np.sum(entropy))
        out["TS"] = ts
        out["F_fde"] = E - ts
        # fragment-energy recast (Appendix), E_H^nad restored
        EK, EHI, ExcI = [], [], []
        for I in range(nsub):
            eh = potentials.hartree(rhos[I], self.lattice)[1]
            ex = functionals.xc(rhos[I], self.lattice, wl.xc, wl.rho_cut)[0]
            el = float(basis.integrate(self.vloc * rhos[I], self.lattice))
            EHI.append(eh)
            ExcI.append(ex)
            EK.append(T[I] + Enl[I] + el + ex + eh + self.enn)
        Exc_nad = pot["Exc"] - float(np.sum(ExcI))
        EH_nad = pot["EH"] - float(np.sum(EHI))
        out["E_K"] = np.array(EK)
        out["E_xc_nad"] = Exc_nad
        out["E_H_nad"] = EH_nad
        out["E_fde_fragments"] = float(np.sum(EK)) + Tnad + Exc_nad + EH_nad - (nsub - 1) * self.enn
        # band-energy + deband form
        if eigs_all is not None and veff_used is not None:
            Eb = 0.0
            for I in range(nsub):
                s = self.subs[I]
                band = sum(2.0 * s.wk[k] * float(np.sum(occ_all[I][k] * eigs_all[I][k]))
                           for k in range(s.nk))
                deband = -float(basis.integrate(veff_used[I] * rhos[I], self.lattice))
                Eb += band + deband
            out["E_fde_band"] = Eb + Eloc + pot["EH"] + pot["Exc"] + Tnad + self.enn
        return out
