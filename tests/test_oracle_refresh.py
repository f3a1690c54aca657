"""Pins of the default density refresh and of the misplaced-electron metric (CPU only)."""
import math

import numpy as np
import pytest
from scipy.special import erf

from oracle import basis, fde as ofde, refresh, scf
from paper_1406_7803_gb300 import workloads


def test_delta_rho_of_two_displaced_gaussians():
    """Two unit charges (alpha/pi)^{3/2} exp(-alpha r^2) a distance d apart along x: their
    difference is positive on one side of the bisecting plane, so
    1/2 int |rho_a - rho_b| = erf(sqrt(alpha) d / 2) (the difference of two 1D normal CDFs at
    d / 2).  The |.| kink at that plane makes the grid sum second order in the x spacing, so x
    is sampled finely; y and z (smooth, periodic) need few points."""
    L = np.array([16.0, 8.0, 8.0])
    grid = (768, 32, 32)

    class _S:  # the grid geometry the metric needs
        omega = float(np.prod(L))
        nr = int(np.prod(grid))

    r = basis.grid_points(np.diag(L), grid)
    alpha = 1.7
    for d in (0.3, 1.0, 2.5):
        ca, cb = np.array([8.0, 4.0, 4.0]), np.array([8.0 + d, 4.0, 4.0])
        ga = (alpha / math.pi) ** 1.5 * np.exp(-alpha * np.sum((r - ca) ** 2, -1))
        gb = (alpha / math.pi) ** 1.5 * np.exp(-alpha * np.sum((r - cb) ** 2, -1))
        want = erf(math.sqrt(alpha) * d / 2)
        assert abs(refresh.delta_rho(_S, ga, gb) - want) < 1e-4 * want, (d, want)
    assert refresh.delta_rho(_S, ga, ga) == 0.0


def test_supersystem_input_holds_every_atom_and_electron():
    wl = workloads.molecule_on_slab_small()
    sup = workloads.supersystem(wl, extra_bands=2)
    (s,) = sup.subsystems
    assert s.natoms == sum(x.natoms for x in wl.subsystems)
    assert s.nelec == sum(x.nelec for x in wl.subsystems)
    assert s.nbands == sum(x.nbands for x in wl.subsystems) + 2
    assert s.smearing == wl.subsystems[0].smearing and s.nk == wl.subsystems[0].nk


def _tiny():
    """The 2 x 3-atom LDA + TF cell at a lower cutoff (24^3 grid, 6 Ha, ~700 plane waves), so
    that dense eigensolves keep these SCF pins to seconds."""
    import dataclasses
    return dataclasses.replace(workloads.plain_fde_32(), grid=(24, 24, 24), ecut=6.0, name="plain-fde-tiny")


DENSE = 4000  # dense LAPACK eigensolves below this many plane waves


@pytest.fixture(scope="module")
def plain():
    wl = _tiny()
    sy = ofde.System(wl)
    return wl, sy


def test_default_refresh_reaches_the_freeze_and_thaw_fixed_point(plain):
    """The refreshed SCF and freeze-and-thaw cycles solve the same coupled equations (Fig. 1b
    caption: run to self-consistency before the densities are exchanged, the SCF becomes
    freeze-and-thaw), so the refreshed SCF's converged state is a fixed point of the cycle:
    one freeze-and-thaw cycle started from it changes no density and no energy.  Cycles from
    the seeded start approach the same energy (linearly, with a ratio near 1/2 per cycle on
    this cell), while the refreshed SCF gets there in a few dozen single steps."""
    wl, sy = plain
    st_r, en_r = refresh.scf_default_refresh(sy, scf.initial_state(sy), tol=1e-10, dense_max=DENSE)
    assert en_r["converged"]
    st_f, en_f = scf.freeze_thaw_cycle(sy, st_r, tol=1e-10, dense_max=DENSE)
    assert en_f["converged"]
    assert abs(en_f["F_fde"] - en_r["F_fde"]) < 1e-8
    for I in range(wl.nsub):
        assert refresh.delta_rho(sy, st_r.rhos[I], st_f.rhos[I]) < 1e-7
    # three cycles from the seeded start: each one halves (or better) the distance to it
    st, gaps = scf.initial_state(sy), []
    for _ in range(3):
        st, en = scf.freeze_thaw_cycle(sy, st, tol=1e-8, dense_max=DENSE)
        gaps.append(en["F_fde"] - en_r["F_fde"])
    assert all(g > 0 for g in gaps) and gaps[1] < 0.5 * gaps[0] and gaps[2] < 0.5 * gaps[1], gaps


def test_single_subsystem_refresh_is_kohn_sham(plain):
    """With one subsystem holding every atom the nonadditive terms vanish and the refreshed SCF
    is the plain KS SCF: it equals the one-subsystem freeze-and-thaw cycle (an SCF to
    self-consistency), and <Delta rho> between the two runs is zero to the tolerance."""
    wl, _ = plain
    sup = workloads.supersystem(wl, extra_bands=2)
    sy = ofde.System(sup)
    st, en = refresh.scf_default_refresh(sy, scf.initial_state(sy), tol=1e-10, dense_max=DENSE)
    assert en["converged"]
    assert en["T_nad"] == 0.0 and en["E_xc_nad"] == 0.0 and en["E_H_nad"] == 0.0
    st_f, en_f = scf.freeze_thaw_cycle(sy, scf.initial_state(sy), tol=1e-10, dense_max=DENSE)
    assert abs(en["F_fde"] - en_f["F_fde"]) < 1e-8
    assert refresh.delta_rho(sy, st.rhos[0], st_f.rhos[0]) < 1e-7
