"""Seeded synthetic workloads shaped like the paper's molecule-on-metal-surface cells.

This module only builds *inputs*: cells, grids, cutoffs, atom positions and charges,
k-point sets, band counts, electron counts, functional choices and raw random draws.
It holds none of the method's arithmetic (no basis sets, no transforms, no potentials),
so that both the CUDA path and the CPU oracle can take their inputs from it without
sharing any computation.

The systems of the paper (Table 1; Computational Details) are a metal slab sampled with
a 2x2x1 Monkhorst-Pack mesh and smeared occupations, plus one or more molecules treated
at Gamma with integer occupations.  Their geometries and pseudopotentials are not
available, so the cells below are synthetic stand-ins of the same structure: a layered
slab of charge-Z model atoms under a vacuum region that holds the molecules.

Units are Hartree atomic units (bohr, Hartree).  All positions are Cartesian bohr;
k-points are in crystal coordinates (fractions of the reciprocal vectors).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

# Gaussian Kleinman-Bylander projector set shared by every atom that carries projectors:
# two s-type Gaussians of widths sigma (bohr) with a diagonal coupling matrix D (Ha).
KB_SIGMA = (0.5, 1.0)
KB_D = ((0.5, 0.0), (0.0, -0.25))

XC_LDA = 0  # Slater exchange + Perdew-Wang 1992 correlation
XC_PBE = 1
KEDF_TF = 0  # Thomas-Fermi, F(s) = 1
KEDF_REVAPBEK = 1
KEDF_LC94 = 2


@dataclass
class Subsystem:
    name: str
    pos: np.ndarray  # [natoms, 3] bohr
    Z: np.ndarray  # [natoms]
    rc: float  # width of the erf-regularised local potential
    nbands: int
    kpts: np.ndarray  # [nk, 3] crystal coordinates
    wk: np.ndarray  # [nk], sums to 1
    nelec: float
    smearing: float  # smearing width in Ha; 0 means integer occupations
    proj_sigma: Tuple[float, ...] = ()
    proj_D: Tuple[Tuple[float, ...], ...] = ()
    smearing_kind: str = "fermi"  # "fermi", "mp" (first-order Methfessel-Paxton) or "gauss"
    # ultrasoft augmentation of the atoms of this subsystem (empty: norm-conserving): the overlap
    # S = 1 + sum_a |beta_a> q <beta_a| and augmentation charges q_ij g_a(r), g_a a normalised
    # Gaussian of width aug_sigma on the atom
    proj_Q: Tuple[Tuple[float, ...], ...] = ()
    aug_sigma: float = 0.0

    @property
    def natoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def nk(self) -> int:
        return int(self.kpts.shape[0])


@dataclass
class Workload:
    name: str
    lattice: np.ndarray  # rows are the lattice vectors a_1, a_2, a_3 (bohr)
    grid: Tuple[int, int, int]
    ecut: float  # Ha, wavefunction cutoff: 0.5|k+G|^2 <= ecut
    subsystems: List[Subsystem]
    xc: int
    kedf: int
    seed: int
    tol: float  # energy convergence threshold (Ha)
    rho_cut: float = 1e-10
    description: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nsub(self) -> int:
        return len(self.subsystems)

    def band_k_pairs(self) -> int:
        return sum(s.nbands * s.nk for s in self.subsystems)


def _min_image_dist(a, b, lengths):
    d = a - b
    d -= lengths * np.round(d / lengths)
    return float(np.sqrt((d * d).sum()))


def _place_uniform(rng, n, lengths, min_sep, existing=(), max_tries=200000):
    """Uniform positions in an orthorhombic box with a minimum periodic separation."""
    out = list(existing)
    placed = []
    tries = 0
    while len(placed) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place atoms with the requested separation")
        p = rng.uniform(0.0, 1.0, 3) * lengths
        if all(_min_image_dist(p, q, lengths) >= min_sep for q in out):
            out.append(p)
            placed.append(p)
    return np.array(placed)


def _place_in_sphere(rng, n, centre, radius, min_sep, lengths, max_tries=200000):
    placed = []
    tries = 0
    while len(placed) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place molecule atoms")
        d = rng.uniform(-1.0, 1.0, 3)
        if (d * d).sum() > 1.0:
            continue
        p = centre + radius * d
        if all(_min_image_dist(p, q, lengths) >= min_sep for q in placed):
            placed.append(p)
    return np.array(placed)


def _mp_mesh(q1, q2, q3):
    """Unreduced Monkhorst-Pack mesh, crystal coordinates, equal weights."""
    def axis(q):
        return [(2 * r - q - 1) / (2.0 * q) for r in range(1, q + 1)]
    pts = [(a, b, c) for a in axis(q1) for b in axis(q2) for c in axis(q3)]
    k = np.array(pts, dtype=np.float64)
    return k, np.full(len(pts), 1.0 / len(pts))


def _slab(nx, ny, nlayers, lengths, interlayer, z0, Z):
    sx, sy = lengths[0] / nx, lengths[1] / ny
    pos = []
    for l in range(nlayers):
        off = 0.5 if (l % 2) else 0.0
        for i in range(nx):
            for j in range(ny):
                pos.append(((i + 0.5 + off) * sx, (j + 0.5 + off) * sy, z0 + l * interlayer))
    pos = np.array(pos)
    pos[:, 0] %= lengths[0]
    pos[:, 1] %= lengths[1]
    return pos, np.full(len(pos), float(Z))


GAMMA = (np.zeros((1, 3)), np.ones(1))


def plain_fde_32(seed: int = 1001, natoms: int = 3) -> Workload:
    """Two 3-atom subsystems (Z=2, 4 doubly occupied bands each) in a 10 bohr cube,
    32^3 grid, 15 Ha cutoff, Gamma only, LDA + Thomas-Fermi, local potentials only."""
    rng = np.random.default_rng(seed)
    L = np.array([10.0, 10.0, 10.0])
    allpos = _place_uniform(rng, 2 * natoms, L, 1.5)
    subs = []
    for i in range(2):
        subs.append(Subsystem(
            name=f"frag{i}", pos=allpos[i * natoms:(i + 1) * natoms].copy(),
            Z=np.full(natoms, 2.0), rc=0.5, nbands=4, kpts=GAMMA[0].copy(), wk=GAMMA[1].copy(),
            nelec=8.0, smearing=0.0))
    return Workload(name="plain-fde-10bohr-32cubed" + ("" if natoms == 3 else f"-{natoms}atoms"),
                    lattice=np.diag(L), grid=(32, 32, 32), ecut=15.0,
                    subsystems=subs, xc=XC_LDA, kedf=KEDF_TF, seed=seed, tol=1e-8,
                    description="2 subsystems x 3 atoms (Z=2), 4 bands each, LDA + TF, FP64")


def molecule_on_slab(seed: int = 1002, lengths=(16.0, 16.0, 40.0), grid=(72, 72, 180),
                     ecut=20.0, slab_xy=3, slab_layers=4, interlayer=3.7, slab_bands=64,
                     mp=(2, 2, 1), mol_atoms=6, mol_bands=12, name=None) -> Workload:
    """A Z=3 slab (Fermi smearing 0.01 Ha, Monkhorst-Pack k-mesh) under a Z=4 molecule
    placed 5 bohr above its top layer at Gamma; PBE + revAPBEK; 2 KB projectors per atom."""
    rng = np.random.default_rng(seed)
    L = np.array(lengths, dtype=np.float64)
    spos, sZ = _slab(slab_xy, slab_xy, slab_layers, L, interlayer, 2.0, 3)
    kp, wk = _mp_mesh(*mp)
    top = 2.0 + (slab_layers - 1) * interlayer
    centre = np.array([L[0] / 2, L[1] / 2, top + 5.0])
    mpos = _place_in_sphere(rng, mol_atoms, centre, 2.5, 1.4, L)
    slab = Subsystem("slab", spos, sZ, 0.5, slab_bands, kp, wk, float(sZ.sum()), 0.01,
                     KB_SIGMA, KB_D)
    mol = Subsystem("molecule", mpos, np.full(mol_atoms, 4.0), 0.5, mol_bands,
                    GAMMA[0].copy(), GAMMA[1].copy(), 4.0 * mol_atoms, 0.0, KB_SIGMA, KB_D)
    return Workload(name=name or "molecule-on-slab-16x16x40-72x72x180",
                    lattice=np.diag(L), grid=tuple(grid), ecut=ecut, subsystems=[slab, mol],
                    xc=XC_PBE, kedf=KEDF_REVAPBEK, seed=seed, tol=1e-6,
                    description="slab (36 atoms Z=3, 64 bands x 4 k) + molecule (6 atoms Z=4, 12 bands, Gamma)")


def molecule_on_slab_small(seed: int = 1012) -> Workload:
    """Same structure as molecule_on_slab at a size the oracle solves in seconds:
    8x8x20 bohr, 24x24x60 grid, 6 Ha; 2 layers of 2x2 atoms with 16 bands x 4 k-points,
    plus a 2-atom molecule with 4 bands."""
    return molecule_on_slab(seed=seed, lengths=(8.0, 8.0, 20.0), grid=(24, 24, 60), ecut=6.0,
                            slab_xy=2, slab_layers=2, interlayer=3.0, slab_bands=16,
                            mol_atoms=2, mol_bands=4, name="molecule-on-slab-8x8x20-24x24x60")


def two_layer_slab_small(mp=(2, 2, 1), smearing_kind: str = "mp") -> Workload:
    """The 2-layer slab of molecule_on_slab_small split into its two layers as subsystems (each
    layer is mirror-symmetric in x and y about the origin, so the whole cell is too): 4 Z=3
    atoms and 8 bands per layer on a Monkhorst-Pack mesh with Methfessel-Paxton smearing of
    1e-2 Ry (Computational Details), PBE + revAPBEK, 2 KB projectors per atom."""
    L = np.array([8.0, 8.0, 20.0])
    pos, Z = _slab(2, 2, 2, L, 3.0, 2.0, 3)
    kp, wk = _mp_mesh(*mp)
    subs = [Subsystem(f"layer{l}", pos[4 * l:4 * l + 4].copy(), Z[4 * l:4 * l + 4].copy(), 0.5, 8, kp.copy(),
                      wk.copy(), 12.0, 0.005, KB_SIGMA, KB_D, smearing_kind) for l in range(2)]
    return Workload(name="two-layer-slab-8x8x20-24x24x60", lattice=np.diag(L), grid=(24, 24, 60), ecut=6.0,
                    subsystems=subs, xc=XC_PBE, kedf=KEDF_REVAPBEK, seed=1013, tol=1e-6,
                    description="two slab layers (4 atoms Z=3, 8 bands each) on a 2x2x1 mesh, MP smearing")


USPP_Q = ((0.25, 0.05), (0.05, 0.10))
USPP_SIGMA = 0.7


def uspp_small(q=USPP_Q, sigma: float = USPP_SIGMA) -> Workload:
    """The small slab + molecule cell with ultrasoft-like atoms: every atom's two Gaussian
    projectors also define the overlap S = 1 + sum_a |beta_a> q <beta_a| and augmentation
    charges q_ij g_a(r) (g_a a normalised Gaussian of width sigma), subsystem by subsystem
    (Appendix: subsystem-specific PAW / ultrasoft projectors)."""
    import dataclasses
    wl = molecule_on_slab_small()
    subs = [dataclasses.replace(s, proj_Q=q, aug_sigma=sigma) for s in wl.subsystems]
    return dataclasses.replace(wl, subsystems=subs, name=wl.name + "-uspp")


def with_kpoints(wl: Workload, isub: int, kpts, wk) -> Workload:
    """The same workload with the k-points and weights of one subsystem replaced."""
    import dataclasses
    subs = list(wl.subsystems)
    subs[isub] = dataclasses.replace(subs[isub], kpts=np.asarray(kpts, dtype=np.float64).reshape(-1, 3),
                                     wk=np.asarray(wk, dtype=np.float64))
    return dataclasses.replace(wl, subsystems=subs)


def batched_uneven(seed: int = 1003, nmol: int = 16) -> Workload:
    """A 54-atom slab (96 bands x 2 k-points) plus molecules with 8..64 bands at Gamma in a
    24 bohr cube on a 96^3 grid at 20 Ha."""
    rng = np.random.default_rng(seed)
    L = np.array([24.0, 24.0, 24.0])
    spos, sZ = _slab(3, 3, 6, L, 2.5, 2.0, 3)
    kp = np.array([[0.25, 0.0, 0.0], [-0.25, 0.0, 0.0]])
    subs = [Subsystem("slab", spos, sZ, 0.5, 96, kp, np.array([0.5, 0.5]), float(sZ.sum()),
                      0.01, KB_SIGMA, KB_D)]
    bands = rng.integers(8, 65, size=nmol)
    centres = []
    for m in range(nmol):
        for _ in range(100000):
            c = np.array([rng.uniform(0, L[0]), rng.uniform(0, L[1]), rng.uniform(17.0, 23.0)])
            if all(_min_image_dist(c, q, L) >= 5.0 for q in centres):
                break
        centres.append(c)
        na = int(bands[m]) // 2
        pos = _place_in_sphere(rng, na, c, 3.0, 0.8, L)
        subs.append(Subsystem(f"mol{m}", pos, np.full(na, 4.0), 0.5, int(bands[m]),
                              GAMMA[0].copy(), GAMMA[1].copy(), 4.0 * na, 0.0, KB_SIGMA, KB_D))
    return Workload(name="batched-uneven-24cubed-96cubed", lattice=np.diag(L),
                    grid=(96, 96, 96), ecut=20.0, subsystems=subs, xc=XC_PBE,
                    kedf=KEDF_REVAPBEK, seed=seed, tol=1e-6,
                    description="slab 54 atoms (96 bands x 2 k) + 16 molecules of 8..64 bands")


def supersystem(wl: Workload, extra_bands: int = 0) -> Workload:
    """The same cell as one subsystem holding every atom and every electron: the input of the
    supersystem Kohn-Sham reference run (Computational Details: FDE densities are compared
    with KS-DFT of the whole system on the same grid).  Bands add up (plus extra_bands); the
    k-points and smearing are those of the first smeared subsystem if there is one (the metal
    sets the sampling of the whole cell), else Gamma with integer occupations.  Every
    subsystem must carry the same projector set."""
    sm = [s for s in wl.subsystems if s.smearing > 0]
    ref = sm[0] if sm else wl.subsystems[0]
    sig = {(tuple(s.proj_sigma), tuple(s.proj_Q), s.aug_sigma) for s in wl.subsystems}
    if len(sig) != 1 or len({s.rc for s in wl.subsystems}) != 1:
        raise ValueError("the supersystem needs one projector set and one r_c")
    whole = Subsystem(name="supersystem",
                      pos=np.concatenate([s.pos for s in wl.subsystems], axis=0),
                      Z=np.concatenate([s.Z for s in wl.subsystems]), rc=ref.rc,
                      nbands=sum(s.nbands for s in wl.subsystems) + extra_bands,
                      kpts=ref.kpts.copy(), wk=ref.wk.copy(),
                      nelec=float(sum(s.nelec for s in wl.subsystems)), smearing=ref.smearing,
                      proj_sigma=tuple(ref.proj_sigma), proj_D=tuple(ref.proj_D),
                      smearing_kind=ref.smearing_kind, proj_Q=tuple(ref.proj_Q), aug_sigma=ref.aug_sigma)
    return Workload(name=wl.name + "-supersystem", lattice=wl.lattice.copy(), grid=wl.grid, ecut=wl.ecut,
                    subsystems=[whole], xc=wl.xc, kedf=wl.kedf, seed=wl.seed, tol=wl.tol, rho_cut=wl.rho_cut,
                    description="supersystem KS reference of " + wl.name)


def large_cell(seed: int = 1005, nmol: int = 32, slab_bands: int = 512, mp=(4, 2, 1)) -> Workload:
    """A 30 x 30 x 60 bohr cell on a 144 x 144 x 288 grid at 25 Ha: a 216-atom Z=3 slab (6 layers
    of 6 x 6 at 5 bohr, 2.5 bohr apart, alternate layers shifted) with 512 bands on an unreduced
    4 x 2 x 1 Monkhorst-Pack mesh (8 k-points, Fermi smearing 0.01 Ha), plus 32 molecules of
    16..48 bands (U{16..48}) at Gamma, floor(b/2) atoms of Z=4 each, centred in the vacuum above
    the slab at least 5 bohr apart; PBE + revAPBEK, 2 KB projectors per atom."""
    rng = np.random.default_rng(seed)
    L = np.array([30.0, 30.0, 60.0])
    spos, sZ = _slab(6, 6, 6, L, 2.5, 2.0, 3)
    kp, wk = _mp_mesh(*mp)
    subs = [Subsystem("slab", spos, sZ, 0.5, slab_bands, kp, wk, float(sZ.sum()), 0.01, KB_SIGMA, KB_D)]
    bands = rng.integers(16, 49, size=nmol)
    centres = []
    for m in range(nmol):
        for _ in range(100000):
            c = np.array([rng.uniform(0, L[0]), rng.uniform(0, L[1]), rng.uniform(20.0, 52.0)])
            if all(_min_image_dist(c, q, L) >= 5.0 for q in centres):
                break
        centres.append(c)
        na = int(bands[m]) // 2
        pos = _place_in_sphere(rng, na, c, 3.0, 0.8, L)
        subs.append(Subsystem(f"mol{m}", pos, np.full(na, 4.0), 0.5, int(bands[m]),
                              GAMMA[0].copy(), GAMMA[1].copy(), 4.0 * na, 0.0, KB_SIGMA, KB_D))
    return Workload(name="large-30x30x60-144x144x288", lattice=np.diag(L), grid=(144, 144, 288), ecut=25.0,
                    subsystems=subs, xc=XC_PBE, kedf=KEDF_REVAPBEK, seed=seed, tol=1e-6,
                    description="slab 216 atoms (512 bands x 8 k) + 32 molecules of 16..48 bands")


def raw_orbitals(seed: int, isub: int, ik: int, nbands: int, npw: int) -> np.ndarray:
    """Raw complex normal draws (N(0,1) + i N(0,1)) for the initial orbitals of one
    (subsystem, k-point).  Shaping and orthonormalisation are done by the solver."""
    rng = np.random.default_rng([seed, isub, ik])
    re = rng.standard_normal((nbands, npw))
    im = rng.standard_normal((nbands, npw))
    return re + 1j * im


def initial_density(wl: Workload, isub: int, alpha: float = 2.0) -> np.ndarray:
    """Starting density of one subsystem on the shared grid: a superposition of
    normalised Gaussians (alpha/pi)^{3/2} exp(-alpha |r - R_a|^2) on its atoms (periodic
    images included), weighted by Z_a and scaled to hold N_I electrons.  Grid layout
    [n1][n2][n3], point (i1, i2, i3) at sum_j (i_j / n_j) a_j."""
    s = wl.subsystems[isub]
    A = np.asarray(wl.lattice, dtype=np.float64)
    n1, n2, n3 = wl.grid
    rho = np.zeros(wl.grid)
    if np.count_nonzero(A - np.diag(np.diag(A))) == 0:
        # orthorhombic cell: the Gaussian factorises over the axes, and so does the sum over
        # the 27 images (i, j, k), one axis at a time
        L = np.diag(A)
        x = [np.arange(n) / n * L[c] for c, n in enumerate(wl.grid)]
        for p, z in zip(s.pos, s.Z):
            g = [sum(np.exp(-alpha * (x[c] - (p[c] + i * L[c])) ** 2) for i in (-1, 0, 1)) for c in range(3)]
            rho += z * (alpha / np.pi) ** 1.5 * (g[0][:, None, None] * g[1][None, :, None] * g[2][None, None, :])
    else:
        f = np.meshgrid(np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3, indexing="ij")
        r = f[0][..., None] * A[0] + f[1][..., None] * A[1] + f[2][..., None] * A[2]
        for p, z in zip(s.pos, s.Z):
            for i in (-1, 0, 1):
                for j in (-1, 0, 1):
                    for k in (-1, 0, 1):
                        d = r - (p + i * A[0] + j * A[1] + k * A[2])
                        rho += z * (alpha / np.pi) ** 1.5 * np.exp(-alpha * np.sum(d * d, axis=-1))
    omega = abs(np.linalg.det(A))
    total = rho.sum() * omega / rho.size
    return rho * (s.nelec / total)


def raw_field(seed: int, shape, tag: int = 0) -> np.ndarray:
    """Raw uniform draws in [0, 1) used by tests that need a seeded real field."""
    rng = np.random.default_rng([seed, 7919, tag])
    return rng.uniform(0.0, 1.0, size=shape)


WORKLOADS = {
    "plain-fde-10bohr-32cubed": plain_fde_32,
    "molecule-on-slab-16x16x40-72x72x180": molecule_on_slab,
    "molecule-on-slab-8x8x20-24x24x60": molecule_on_slab_small,
    "batched-uneven-24cubed-96cubed": batched_uneven,
    "large-30x30x60-144x144x288": large_cell,
}
