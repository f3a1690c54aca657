"""The paper's default density refresh and the misplaced-electron metric <Delta rho>.

Test infrastructure only (see ``oracle/__init__.py``).

* Default refresh (Sec. 2, text after Fig. 1; Fig. 1b caption): the subsystem SCF of
  Fig. 1b is executed once per refresh.  Every subsystem takes one SCF step (eigenpairs of
  its H_I in the current V_eff^I, occupations, output density) and then every rho_I is
  refreshed together, so the total density and with it the Hartree and embedding
  potentials are rebuilt at every step.  At convergence every subsystem density is
  self-consistent with every other one: the fixed point is that of freeze-and-thaw cycles
  repeated to convergence.
  Readings (the paper is silent on mixing and on the stopping rule): the densities of all
  subsystems are mixed together, one Pulay (DIIS) step on the stacked vector
  (rho_1, ..., rho_NS) with the history and weight of the inner SCF (8, 0.3), so that one set
  of coefficients serves every subsystem (independent histories per subsystem ignore the
  coupling through the shared potential and were seen to stall near 1e-2 electrons); the run
  has converged when the FDE free energy changes by less than tol between steps and every
  subsystem's int|rho_out - rho_in| is below 10 tol.
* <Delta rho> = 1/2 int |rho_FDE(r) - rho_KS(r)| dr (Computational Details, Eq. deltarho):
  rho_KS from a supersystem Kohn-Sham run on the same grid, which is the same SCF on the
  one-subsystem cell of ``workloads.supersystem`` (with N_S = 1 every nonadditive term
  vanishes and FDE is KS).
"""
from __future__ import annotations

import numpy as np

from . import scf


def delta_rho(system, rho_a, rho_b):
    """<Delta rho> = 1/2 int |rho_a - rho_b| dr on the grid of ``system``."""
    return 0.5 * float(np.sum(np.abs(np.asarray(rho_a) - np.asarray(rho_b)))) * system.omega / system.nr


def scf_default_refresh(system, state, tol=None, max_scf=200, dense_max=0, log=None):
    """SCF of all subsystems with the total density refreshed after every step; returns the
    final state and the energies of its output densities."""
    wl = system.wl
    tol = wl.tol if tol is None else tol
    ns = len(system.subs)
    mixer = scf.Pulay()  # one DIIS on the stacked subsystem densities
    rho_in = np.array(state.rhos, copy=True)
    coefs = state.coefs
    F_prev = None
    en = None
    for it in range(1, max_scf + 1):
        pot = system.build_veff(rho_in)
        new_coefs, new_occ, new_eigs = [], [], []
        rho_out = np.zeros_like(rho_in)
        ent = np.zeros(ns)
        for I, s in enumerate(system.subs):
            eigs, vecs = [], []
            for k in range(s.nk):
                w, v = scf.eigensolve(system, I, k, pot["veff"][I], s.nbands, coefs[I][k], dense_max)
                eigs.append(w)
                vecs.append(v)
            occ, _, S = scf.occupations(eigs, s.wk, s.nelec, s.smearing, s.smearing_kind)
            rho_out[I] = system.density(I, vecs, occ)
            ent[I] = s.smearing * S
            new_coefs.append(vecs)
            new_occ.append(occ)
            new_eigs.append(eigs)
        en = system.energies(new_coefs, new_occ, rho_out, entropy=ent)
        dres = [float(np.sum(np.abs(rho_out[I] - rho_in[I]))) * system.omega / system.nr for I in range(ns)]
        dF = None if F_prev is None else en["F_fde"] - F_prev
        if log is not None:
            log.append(dict(it=it, F=en["F_fde"], dF=dF, dres=dres))
        coefs = new_coefs
        if F_prev is not None and abs(dF) < tol and max(dres) < 10.0 * tol:
            en["converged"], en["iters"] = True, it
            return scf.State(system, new_coefs, new_occ, new_eigs, rho_out, ent), en
        F_prev = en["F_fde"]
        rho_in = mixer(rho_in, rho_out)
    en["converged"], en["iters"] = False, max_scf
    return scf.State(system, new_coefs, new_occ, new_eigs, rho_out, ent), en
