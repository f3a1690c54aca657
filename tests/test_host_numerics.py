"""The library's host-side numerics (no device work) against the oracle and closed forms, on
the CPU: the plane-wave sphere, the Ewald nuclear repulsion, occupations with the chemical
potential and the Mermin term, and the Pulay mixing coefficients.  The engine calls these
same routines (hostmath.cu)."""
import math

import numpy as np
import pytest

from oracle import basis, potentials, scf
from paper_1406_7803_gb300 import fde, workloads


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_7803_gb300 import build
    build.build()
    fde.load()


@pytest.mark.parametrize("make", [workloads.plain_fde_32, workloads.molecule_on_slab_small,
                                  workloads.molecule_on_slab])
def test_sphere_equals_oracle_sphere(make):
    wl = make()
    L = np.diag(wl.lattice)
    for s in wl.subsystems:
        for kf in s.kpts:
            mil, kin = fde.host_sphere(L, kf, wl.ecut)
            want_mil, want_kin = basis.sphere(wl.lattice, wl.grid, kf, wl.ecut)
            assert np.array_equal(mil.astype(np.int64), want_mil)
            assert np.abs(kin - want_kin).max() <= 1e-13 * want_kin.max()


def test_sphere_boundary_and_brute_force():
    """A cutoff exactly on a shell (|G|^2/2 = ecut for G = (1, 0, 0) 2 pi / L) includes it, and
    the count equals a brute-force count of integer triples."""
    L = np.array([2 * math.pi, 2 * math.pi, 2 * math.pi])  # |G_m|^2 = |m|^2
    mil, kin = fde.host_sphere(L, [0.0, 0.0, 0.0], 4.5)  # |m|^2 <= 9
    brute = [(a, b, c) for a in range(-4, 5) for b in range(-4, 5) for c in range(-4, 5)
             if a * a + b * b + c * c <= 9]
    assert len(mil) == len(brute)
    assert sorted(map(tuple, mil.tolist())) == sorted(brute)
    assert [3, 0, 0] in mil.tolist() and kin.max() == 4.5


def test_ewald_equals_oracle_and_madelung():
    rng = np.random.default_rng(3)
    L = np.array([9.0, 10.0, 11.0])
    pos = rng.uniform(0, 1, (5, 3)) * L
    Z = rng.uniform(1, 4, 5)
    e = fde.host_ewald(L, pos, Z)
    assert abs(e - potentials.ewald(np.diag(L), pos, Z)) < 1e-10 * abs(e)
    # simple cubic lattice of unit charges in a neutralising background: E = -a / (2 L)
    a_sc = 2.8372974794806
    for Lc in (1.0, 7.5):
        e1 = fde.host_ewald(np.full(3, Lc), np.zeros((1, 3)), np.ones(1))
        assert abs(e1 - (-a_sc / (2.0 * Lc))) < 1e-12 / Lc


def test_fermi_occupations_equal_oracle():
    rng = np.random.default_rng(5)
    eig = np.sort(rng.uniform(-1.0, 0.5, (4, 16)), axis=1)
    wk = np.full(4, 0.25)
    occ, mu, ts = fde.host_occupations(eig, wk, 18.0, 0.01)
    o_occ, o_mu, o_S = scf.occupations(list(eig), wk, 18.0, 0.01)
    assert np.abs(occ - np.array(o_occ)).max() < 1e-12
    assert abs(mu - o_mu) < 1e-12
    assert abs(ts - 0.01 * o_S) < 1e-14
    assert abs(2.0 * np.sum(wk[:, None] * occ) - 18.0) < 1e-12


@pytest.mark.parametrize("kind", ["mp", "gauss"])
def test_methfessel_paxton_and_gaussian_occupations_equal_oracle(kind):
    """The host's closed forms (first-order Methfessel-Paxton, Gaussian) against the oracle's
    general-order Hermite construction with its entropy term by quadrature."""
    rng = np.random.default_rng(6)
    eig = np.sort(rng.uniform(-1.0, 0.5, (4, 16)), axis=1)
    wk = np.full(4, 0.25)
    sigma = 0.005  # 1e-2 Ry (Computational Details)
    occ, mu, ts = fde.host_occupations(eig, wk, 18.0, sigma, kind)
    o_occ, o_mu, o_S = scf.occupations(list(eig), wk, 18.0, sigma, kind)
    assert np.abs(occ - np.array(o_occ)).max() < 1e-12
    assert abs(mu - o_mu) < 1e-12
    assert abs(ts - sigma * o_S) < 1e-13
    assert abs(2.0 * np.sum(wk[:, None] * occ) - 18.0) < 1e-12


def test_integer_occupations_and_argument_checks():
    eig = np.array([[0.3, -0.2, 0.1, -0.5, 0.9]])
    occ, mu, ts = fde.host_occupations(eig, [1.0], 6.0, 0.0)
    # the three lowest levels (-0.5, -0.2, 0.1) hold the 6 electrons; mu is the highest of them
    assert occ.tolist() == [[0.0, 1.0, 1.0, 1.0, 0.0]]
    assert mu == 0.1 and ts == 0.0
    o_occ, o_mu, _ = scf.occupations([eig[0]], [1.0], 6.0, 0.0)
    assert np.array_equal(occ[0], o_occ[0]) and mu == o_mu
    with pytest.raises(fde.FDEError):
        fde.host_occupations(eig, [1.0], 5.0, 0.0)   # odd electron count without smearing
    with pytest.raises(fde.FDEError):
        fde.host_occupations(np.zeros((2, 3)), [0.5, 0.5], 4.0, 0.0)  # integer filling needs one k


def test_pulay_coefficients_equal_oracle_step():
    """The coefficients minimise |sum c_i R_i| with sum c = 1: compare with the oracle's own
    mixing step (scf.Pulay) on the same residual history."""
    rng = np.random.default_rng(8)
    rin = [rng.standard_normal(50) for _ in range(4)]
    rout = [r + 0.1 * rng.standard_normal(50) for r in rin]
    mixer = scf.Pulay()
    for a, b in zip(rin, rout):
        want = mixer(a, b)
    res = np.array([b - a for a, b in zip(rin, rout)])
    c, ok = fde.host_pulay(res @ res.T)
    assert ok and abs(c.sum() - 1.0) < 1e-12
    got = sum(ci * (a + 0.3 * (b - a)) for ci, a, b in zip(c, rin, rout))
    assert np.abs(got - want).max() < 1e-10


def test_pulay_singular_history_keeps_the_newest_residual():
    r = np.ones((2, 3))
    c, ok = fde.host_pulay(r @ r.T)  # two identical residuals: singular bordered system
    assert not ok and c.tolist() == [0.0, 1.0]


def test_host_entry_points_reject_bad_arguments():
    lib = fde.load()
    n = fde.C.c_int()
    e = fde.C.c_double()
    L = np.ones(3)
    assert lib.fde_host_sphere(None, None, 1.0, fde.C.byref(n), None, None) == fde.FDE_EINVAL
    assert lib.fde_host_sphere(fde._hptr(L), fde._hptr(np.zeros(3)), -1.0, fde.C.byref(n), None, None) == fde.FDE_EINVAL
    assert lib.fde_host_sphere(fde._hptr(-L), fde._hptr(np.zeros(3)), 1.0, fde.C.byref(n), None, None) == fde.FDE_EINVAL
    assert lib.fde_host_ewald(fde._hptr(L), 0, None, None, fde.C.byref(e)) == fde.FDE_EINVAL
    assert lib.fde_host_occupations(0, 1, None, None, 2.0, 0.0, 0, None, None, None) == fde.FDE_EINVAL
    assert lib.fde_host_pulay(0, None, None) == fde.FDE_EINVAL


@pytest.mark.parametrize("q,shift,ops,tr", [((2, 2, 1), (0, 0, 0), (), True), ((2, 2, 1), (0, 0, 0), (1, 2, 3), True),
                                            ((3, 3, 1), (0, 0, 0), (), True), ((4, 2, 2), (1, 0, 0), (1,), False),
                                            ((4, 4, 1), (0, 0, 0), (1, 2, 3), True), ((1, 1, 1), (0, 0, 0), (), True)])
def test_kmesh_equals_oracle(q, shift, ops, tr):
    from oracle import kmesh
    k, w = fde.host_kmesh(q, shift, tr, ops)
    ko, wo = kmesh.reduce_mesh(kmesh.monkhorst_pack(q, shift), ops, tr)
    assert np.array_equal(k, ko) and np.allclose(w, wo, rtol=0, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-14


def test_symmetry_ops_equal_oracle():
    from oracle import kmesh
    for wl in (workloads.two_layer_slab_small(), workloads.molecule_on_slab_small(), workloads.molecule_on_slab()):
        L = np.diag(wl.lattice)
        for s in wl.subsystems + workloads.supersystem(wl).subsystems:
            assert fde.host_symmetry_ops(L, s.pos, s.Z) == kmesh.symmetry_ops(wl.lattice, s.pos, s.Z)
