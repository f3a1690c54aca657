"""Thin ctypes binding of the C ABI in ``include/fde.h`` (argument marshalling only).

Every computation happens inside ``libfde.so``; this module converts Python/NumPy/torch
arguments into the plain pointers and sizes the ABI takes.  Device buffers are passed as
torch CUDA tensors (``data_ptr()``), the stream as ``torch.cuda.current_stream()``.
There is no fallback: if the library is missing or fails to load, importing the entry
points raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfde.so")

FDE_OK, FDE_EINVAL, FDE_ENOMEM, FDE_ECUDA, FDE_ENOCONV, FDE_ENONFINITE, FDE_ETIMEOUT, FDE_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
FDE_PREC_FP64, FDE_PREC_MIXED = 0, 1
FDE_PRECOND_TPA, FDE_PRECOND_LEARNED = 0, 1
FDE_PRECOND_PARAMS = 8641
FDE_SMEAR_FERMI, FDE_SMEAR_MP, FDE_SMEAR_GAUSS = 0, 1, 2
SMEAR_KINDS = {"fermi": FDE_SMEAR_FERMI, "mp": FDE_SMEAR_MP, "gauss": FDE_SMEAR_GAUSS}
STATUS_NAMES = {0: "FDE_OK", -1: "FDE_EINVAL", -2: "FDE_ENOMEM", -3: "FDE_ECUDA", -4: "FDE_ENOCONV",
                -5: "FDE_ENONFINITE", -6: "FDE_ETIMEOUT", -7: "FDE_EUNSUPPORTED"}


class CellDesc(C.Structure):
    _fields_ = [("lattice", (C.c_double * 3) * 3), ("grid", C.c_int * 3), ("ecut_ha", C.c_double)]


class FuncDesc(C.Structure):
    _fields_ = [("xc", C.c_int), ("kedf", C.c_int), ("rho_cut", C.c_double)]


class SubsysDesc(C.Structure):
    _fields_ = [("natoms", C.c_int), ("pos", C.POINTER(C.c_double)), ("Z", C.POINTER(C.c_double)),
                ("rc", C.c_double), ("nproj_per_atom", C.c_int), ("proj_sigma", C.POINTER(C.c_double)),
                ("proj_D", C.POINTER(C.c_double)), ("nbands", C.c_int), ("nk", C.c_int),
                ("kpts", C.POINTER(C.c_double)), ("wk", C.POINTER(C.c_double)), ("nelec", C.c_double),
                ("smearing_ha", C.c_double), ("smearing_kind", C.c_int), ("proj_Q", C.POINTER(C.c_double)),
                ("aug_sigma", C.c_double)]


class Energies(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E_fde", "F_fde", "TS", "E_kin", "E_nl", "E_loc", "E_H", "E_xc",
                                          "T_nad", "E_xc_nad", "E_H_nad", "E_nn", "E_band_form")] + \
               [("iters", C.c_int), ("dE", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


EXPORTS = {
    "fde_create": (C.c_int, [C.POINTER(CellDesc), C.POINTER(FuncDesc), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "fde_add_subsystem": (C.c_int, [C.c_void_p, C.POINTER(SubsysDesc), C.POINTER(C.c_int)]),
    "fde_get_basis": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_void_p]),
    "fde_set_density": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "fde_get_density": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fde_build_vemb": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Energies)]),
    "fde_set_veff": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fde_apply_h": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "fde_apply_h_host": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "fde_apply_s": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "fde_apply_h_all": (C.c_int, [C.c_void_p]),
    "fde_init_orbitals": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "fde_set_orbitals": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "fde_get_orbitals": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fde_subspace_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                                     C.POINTER(C.c_int)]),
    "fde_update_density": (C.c_int, [C.c_void_p, C.c_int]),
    "fde_energy": (C.c_int, [C.c_void_p, C.POINTER(Energies)]),
    "fde_scf_subsystem": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.POINTER(Energies)]),
    "fde_freeze_thaw_cycle": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(Energies)]),
    "fde_scf_refresh": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(Energies)]),
    "fde_delta_rho": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "fde_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "fde_profile_get": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "fde_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "fde_apply_h_local_static": (C.c_int, [C.POINTER(CellDesc), C.POINTER(C.c_double), C.c_int, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "fde_fft3d": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "fde_fft3d_f64": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "fde_hot_step": (C.c_int, [C.c_void_p, C.c_int]),
    "fde_get_hpsi": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "fde_gemm_hn_f32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.c_void_p, C.c_int, C.c_int]),
    "fde_set_gemm_path": (C.c_int, [C.c_int]),
    "fde_set_tc_wait_limit": (C.c_int, [C.c_longlong]),
    "fde_set_precond_path": (C.c_int, [C.c_int]),
    "fde_hot_step_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fde_host_sphere": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fde_host_ewald": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fde_host_occupations": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int,
                                       C.c_void_p, C.c_void_p, C.c_void_p]),
    "fde_host_pulay": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p]),
    "fde_host_kmesh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "fde_host_symmetry_ops": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                        C.c_void_p]),
    "fde_set_symmetry": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fde_tuned_plane_variant": (C.c_int, [C.c_int, C.c_int]),
    "fde_pin_plane_variant": (C.c_int, [C.c_int]),
    "fde_gemm_rot_f32": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int]),
    "fde_dense_eigh": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "fde_set_precond": (C.c_int, [C.c_void_p, C.c_int]),
    "fde_precond_set_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fde_precond_get_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "fde_precond_harvest": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "fde_precond_add_pairs": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_void_p]),
    "fde_precond_clear": (C.c_int, [C.c_void_p]),
    "fde_precond_record": (C.c_int, [C.c_void_p, C.c_int]),
    "fde_precond_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "fde_precond_train": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "fde_precond_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "fde_get_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "fde_sync": (C.c_int, [C.c_void_p]),
    "fde_last_error": (C.c_char_p, [C.c_void_p]),
    "fde_destroy": (C.c_int, [C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libfde.so and declare every exported entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_1406_7803_gb300/build.py)")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def precond_initial_weights(seed: int = 0) -> np.ndarray:
    """Starting parameters of the learned preconditioner in the library's flat layout
    (W1 b1 W2 b2 W3 b3 W4 b4): hidden weights N(0, 1/fan_in) from a seeded generator, zero
    biases and a zero output layer, so that training starts from the kinetic preconditioner."""
    rng = np.random.default_rng([seed, 4099])
    width, layers, out = 64, ((3, 64), (64, 64), (64, 64), (64, 1)), []
    for i, (fi, fo) in enumerate(layers):
        W = np.zeros((fo, fi)) if i == len(layers) - 1 else rng.standard_normal((fo, fi)) / np.sqrt(fi)
        out += [W.ravel(), np.zeros(fo)]
    del width
    return np.concatenate(out).astype(np.float32)


def tuned_plane_variant(n1: int, n3: int) -> int:
    """Variant of the FP32 plane pass the tuner chose for this grid shape (-1: none yet)."""
    return int(load().fde_tuned_plane_variant(int(n1), int(n3)))


def pin_plane_variant(variant: int) -> None:
    """Pin the FP32 plane-pass variant (0..7) for this process, or -1 to return to tuning."""
    if load().fde_pin_plane_variant(int(variant)) != FDE_OK:
        raise FDEError(FDE_EINVAL, "fde_pin_plane_variant: variant must be -1..7")


def host_sphere(lengths, kfrac, ecut):
    """Miller indices [npw, 3] and kinetic energies [npw] of the plane-wave sphere (host code)."""
    lib = load()
    L = np.ascontiguousarray(lengths, dtype=np.float64)
    kf = np.ascontiguousarray(kfrac, dtype=np.float64)
    n = C.c_int()
    s = lib.fde_host_sphere(_hptr(L), _hptr(kf), float(ecut), C.byref(n), None, None)
    if s != FDE_OK:
        raise FDEError(s, "fde_host_sphere")
    mil = np.zeros((n.value, 3), dtype=np.int32)
    kin = np.zeros(n.value)
    s = lib.fde_host_sphere(_hptr(L), _hptr(kf), float(ecut), C.byref(n), _hptr(mil), _hptr(kin))
    if s != FDE_OK or n.value != kin.size:
        raise FDEError(s, "fde_host_sphere")
    return mil, kin


def host_ewald(lengths, pos, Z):
    """Ewald nuclear repulsion (Ha) of point charges in an orthorhombic cell (host code)."""
    L = np.ascontiguousarray(lengths, dtype=np.float64)
    p = np.ascontiguousarray(pos, dtype=np.float64)
    z = np.ascontiguousarray(Z, dtype=np.float64)
    e = C.c_double()
    s = load().fde_host_ewald(_hptr(L), int(z.size), _hptr(p), _hptr(z), C.byref(e))
    if s != FDE_OK:
        raise FDEError(s, "fde_host_ewald")
    return e.value


def host_occupations(eig, wk, nelec, sigma, kind="fermi"):
    """(occ [nk, nb], mu, sigma S) of the eigenvalues eig [nk, nb] (host code); kind is the
    smearing ("fermi", "mp" first-order Methfessel-Paxton, "gauss")."""
    ev = np.ascontiguousarray(eig, dtype=np.float64)
    w = np.ascontiguousarray(wk, dtype=np.float64)
    occ = np.zeros_like(ev)
    mu, ts = C.c_double(), C.c_double()
    s = load().fde_host_occupations(int(ev.shape[0]), int(ev.shape[1]), _hptr(ev), _hptr(w), float(nelec),
                                    float(sigma), int(SMEAR_KINDS[kind]), _hptr(occ), C.byref(mu), C.byref(ts))
    if s != FDE_OK:
        raise FDEError(s, "fde_host_occupations")
    return occ, mu.value, ts.value


def host_pulay(overlap):
    """Pulay coefficients from the residual overlaps [m, m] (host code); (coef, solved)."""
    ov = np.ascontiguousarray(overlap, dtype=np.float64)
    c = np.zeros(ov.shape[0])
    s = load().fde_host_pulay(int(ov.shape[0]), _hptr(ov), _hptr(c))
    return c, s == FDE_OK


def host_kmesh(q, shift=(0, 0, 0), time_reversal=True, ops=()):
    """Irreducible Monkhorst-Pack points [nk, 3] (crystal) and weights [nk] (host code)."""
    lib = load()
    qa = np.ascontiguousarray(q, dtype=np.int32)
    sh = np.ascontiguousarray(shift, dtype=np.float64)
    oa = np.ascontiguousarray(ops if len(ops) else [0], dtype=np.int32)
    n = C.c_int(0)
    s = lib.fde_host_kmesh(_hptr(qa), _hptr(sh), int(bool(time_reversal)), int(len(ops)), _hptr(oa), C.byref(n),
                           None, None)
    if s != FDE_OK:
        raise FDEError(s, "fde_host_kmesh")
    k = np.zeros((n.value, 3))
    w = np.zeros(n.value)
    s = lib.fde_host_kmesh(_hptr(qa), _hptr(sh), int(bool(time_reversal)), int(len(ops)), _hptr(oa), C.byref(n),
                           _hptr(k), _hptr(w))
    if s != FDE_OK:
        raise FDEError(s, "fde_host_kmesh")
    return k, w


def host_symmetry_ops(lengths, pos, Z, tol=1e-6):
    """Sign-flip masks (identity first) that map the atoms onto themselves (host code)."""
    L = np.ascontiguousarray(lengths, dtype=np.float64)
    p = np.ascontiguousarray(np.asarray(pos).reshape(-1, 3), dtype=np.float64)
    z = np.ascontiguousarray(Z, dtype=np.float64)
    ops = np.zeros(8, dtype=np.int32)
    n = C.c_int()
    s = load().fde_host_symmetry_ops(_hptr(L), int(z.size), _hptr(p), _hptr(z), float(tol), C.byref(n), _hptr(ops))
    if s != FDE_OK:
        raise FDEError(s, "fde_host_symmetry_ops")
    return ops[:n.value].tolist()


def set_gemm_path(path: int) -> None:
    """Path of the library's FP32 band-block products: 0 CUDA cores, 1 tensor cores (TF32),
    3 tensor cores with split-TF32 operands.  Process-wide (default 3)."""
    s = load().fde_set_gemm_path(int(path))
    if s != FDE_OK:
        raise FDEError(s, "fde_set_gemm_path: path must be 0, 1 or 3")


def set_tc_wait_limit(polls: int) -> None:
    """Poll limit of the tensor-core products' stage waits (0: run out at once; -1: default)."""
    s = load().fde_set_tc_wait_limit(int(polls))
    if s != FDE_OK:
        raise FDEError(s, "fde_set_tc_wait_limit")


def set_precond_path(path: int) -> None:
    """Where the learned preconditioner's inference and training run: 1 tensor cores (default),
    0 CUDA cores.  Process-wide."""
    s = load().fde_set_precond_path(int(path))
    if s != FDE_OK:
        raise FDEError(s, "fde_set_precond_path: path must be 0 or 1")


class FDEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _dptr(t):
    """Device pointer of a torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _dbl(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


class Context:
    """One library context (cell, grid, functionals, subsystems) on the current device."""

    def __init__(self, lattice, grid, ecut, xc, kedf, rho_cut=1e-10, prec="fp64", stream=None):
        self.lib = load()
        cell = CellDesc()
        for i in range(3):
            for j in range(3):
                cell.lattice[i][j] = float(lattice[i][j])
            cell.grid[i] = int(grid[i])
        cell.ecut_ha = float(ecut)
        func = FuncDesc(int(xc), int(kedf), float(rho_cut))
        self.prec = FDE_PREC_MIXED if prec == "mixed" else FDE_PREC_FP64
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        s = self.lib.fde_create(C.byref(cell), C.byref(func), self.prec, st, C.byref(h))
        if s != FDE_OK:
            raise FDEError(s, "fde_create failed (see stderr)")
        self.h = h
        self.grid = tuple(int(n) for n in grid)
        self.nsub = 0
        self._keep = []

    def _check(self, s, what):
        if s != FDE_OK and s != FDE_ENOCONV:
            raise FDEError(s, f"{what}: {self.lib.fde_last_error(self.h).decode()}")
        return s

    def close(self):
        if getattr(self, "h", None):
            self.lib.fde_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- setup --------------------------------------------------------------------------
    def add_subsystem(self, pos, Z, rc, nbands, kpts, wk, nelec, smearing, proj_sigma=(), proj_D=(),
                      smearing_kind="fermi", proj_Q=(), aug_sigma=0.0):
        pos, ppos = _dbl(np.asarray(pos).reshape(-1, 3))
        Z, pZ = _dbl(Z)
        kpts, pk = _dbl(np.asarray(kpts).reshape(-1, 3))
        wk, pw = _dbl(wk)
        sig, psig = _dbl(proj_sigma if len(proj_sigma) else [0.0])
        D, pD = _dbl(np.asarray(proj_D).reshape(-1) if len(proj_sigma) else [0.0])
        Q, pQ = _dbl(np.asarray(proj_Q).reshape(-1) if len(proj_Q) else [0.0])
        d = SubsysDesc(int(Z.size), ppos, pZ, float(rc), int(len(proj_sigma)), psig, pD, int(nbands),
                       int(kpts.shape[0]), pk, pw, float(nelec), float(smearing), int(SMEAR_KINDS[smearing_kind]),
                       pQ if len(proj_Q) else None, float(aug_sigma))
        sid = C.c_int()
        self._check(self.lib.fde_add_subsystem(self.h, C.byref(d), C.byref(sid)), "fde_add_subsystem")
        self.nsub += 1
        return sid.value

    def basis(self, sub, k):
        n = C.c_int()
        self._check(self.lib.fde_get_basis(self.h, sub, k, C.byref(n), None), "fde_get_basis")
        mil = np.zeros((n.value, 3), dtype=np.int32)
        self._check(self.lib.fde_get_basis(self.h, sub, k, C.byref(n), _hptr(mil)), "fde_get_basis")
        return mil

    # ---- data path ----------------------------------------------------------------------
    def set_density(self, sub, rho):
        if hasattr(rho, "is_cuda"):
            return self._check(self.lib.fde_set_density(self.h, sub, _dptr(rho), 1), "fde_set_density")
        a = np.ascontiguousarray(rho, dtype=np.float64)
        return self._check(self.lib.fde_set_density(self.h, sub, _hptr(a), 0), "fde_set_density")

    def get_density(self, sub, out):
        return self._check(self.lib.fde_get_density(self.h, sub, _dptr(out)), "fde_get_density")

    def build_vemb(self, out=None, energies=False):
        e = Energies() if energies else None
        self._check(self.lib.fde_build_vemb(self.h, _dptr(out), C.byref(e) if e is not None else None),
                    "fde_build_vemb")
        return e.as_dict() if e is not None else None

    def set_veff(self, sub, v):
        return self._check(self.lib.fde_set_veff(self.h, sub, _dptr(v)), "fde_set_veff")

    def apply_h(self, sub, k, psi, hpsi, nb):
        return self._check(self.lib.fde_apply_h(self.h, sub, k, _dptr(psi), _dptr(hpsi), int(nb)), "fde_apply_h")

    def apply_s(self, sub, k, psi, spsi, nb):
        return self._check(self.lib.fde_apply_s(self.h, sub, k, _dptr(psi), _dptr(spsi), int(nb)), "fde_apply_s")

    def apply_h_host(self, sub, k, psi, hpsi, nb):
        return self._check(self.lib.fde_apply_h_host(self.h, sub, k, _hptr(psi), _hptr(hpsi), int(nb)),
                           "fde_apply_h_host")

    def apply_h_all(self):
        return self._check(self.lib.fde_apply_h_all(self.h), "fde_apply_h_all")

    def init_orbitals(self, sub, k, raw):
        a = np.ascontiguousarray(raw, dtype=np.complex128)
        return self._check(self.lib.fde_init_orbitals(self.h, sub, k, _hptr(a)), "fde_init_orbitals")

    def set_orbitals(self, sub, k, psi):
        return self._check(self.lib.fde_set_orbitals(self.h, sub, k, _dptr(psi)), "fde_set_orbitals")

    def get_orbitals(self, sub, k, out, nbands):
        eig = np.zeros(nbands)
        occ = np.zeros(nbands)
        self._check(self.lib.fde_get_orbitals(self.h, sub, k, _dptr(out), _hptr(eig), _hptr(occ)),
                    "fde_get_orbitals")
        return eig, occ

    def subspace_solve(self, sub, k, tol, max_iter=100, precond=FDE_PRECOND_TPA):
        it = C.c_int()
        s = self._check(self.lib.fde_subspace_solve(self.h, sub, k, float(tol), int(max_iter), int(precond),
                                                    C.byref(it)), "fde_subspace_solve")
        return s, it.value

    def update_density(self, sub):
        return self._check(self.lib.fde_update_density(self.h, sub), "fde_update_density")

    def energy(self):
        e = Energies()
        self._check(self.lib.fde_energy(self.h, C.byref(e)), "fde_energy")
        return e.as_dict()

    def scf_subsystem(self, sub, tol, max_scf=100):
        e = Energies()
        s = self._check(self.lib.fde_scf_subsystem(self.h, sub, float(tol), int(max_scf), C.byref(e)),
                        "fde_scf_subsystem")
        return s, e.as_dict()

    def freeze_thaw_cycle(self, tol, max_scf=100):
        e = Energies()
        s = self._check(self.lib.fde_freeze_thaw_cycle(self.h, float(tol), int(max_scf), C.byref(e)),
                        "fde_freeze_thaw_cycle")
        return s, e.as_dict()

    def scf_refresh(self, tol, max_scf=200):
        """SCF of every subsystem with the total density refreshed after every step."""
        e = Energies()
        s = self._check(self.lib.fde_scf_refresh(self.h, float(tol), int(max_scf), C.byref(e)), "fde_scf_refresh")
        return s, e.as_dict()

    def set_symmetry(self, ops):
        """Symmetrise the densities built from orbitals over the sign-flip masks ops."""
        a = np.ascontiguousarray(ops, dtype=np.int32)
        return self._check(self.lib.fde_set_symmetry(self.h, int(a.size), _hptr(a)), "fde_set_symmetry")

    def delta_rho(self, rho_ref):
        """1/2 int |rho - rho_ref| against a device grid rho_ref (torch float64, CUDA)."""
        out = C.c_double()
        self._check(self.lib.fde_delta_rho(self.h, _dptr(rho_ref), C.byref(out)), "fde_delta_rho")
        return out.value

    def sync(self):
        return self._check(self.lib.fde_sync(self.h), "fde_sync")

    def profile_enable(self, on=True):
        return self._check(self.lib.fde_profile_enable(self.h, int(on)), "fde_profile_enable")

    def dense_eigh(self, A, nvec, w, V):
        return self._check(self.lib.fde_dense_eigh(self.h, int(A.shape[0]), _dptr(A), int(nvec), _dptr(w), _dptr(V)),
                           "fde_dense_eigh")

    def gemm_hn_f32(self, A, B, K, C, path):
        """C = A^H B over the first K columns of the rows of A (m x lda) and B (n x ldb),
        complex64 device tensors; C complex128 (m x ldc)."""
        return self._check(self.lib.fde_gemm_hn_f32(self.h, _dptr(A), int(A.shape[1]), _dptr(B), int(B.shape[1]),
                                                    int(A.shape[0]), int(B.shape[0]), int(K), _dptr(C),
                                                    int(C.shape[1]), int(path)), "fde_gemm_hn_f32")

    def gemm_rot_f32(self, X, U, K, Y, alpha, beta, path):
        """Y = alpha sum_i U[i][j] X_i + beta Y over the first K columns: X complex64 (m x ldx),
        U complex128 (m x ldu, n = Y rows used), Y complex64 (n x ldy), device tensors."""
        return self._check(self.lib.fde_gemm_rot_f32(self.h, _dptr(X), int(X.shape[1]), _dptr(U), int(U.shape[1]),
                                                     int(X.shape[0]), int(Y.shape[0]), int(K), _dptr(Y),
                                                     int(Y.shape[1]), float(alpha), float(beta), int(path)),
                           "fde_gemm_rot_f32")

    def get_hpsi(self, sub, k, out):
        return self._check(self.lib.fde_get_hpsi(self.h, sub, k, _dptr(out)), "fde_get_hpsi")

    def hot_step_host(self, rhos, psis, hpsis):
        """The hot path end to end with host arrays: rhos[nsub] (float64 grids), psis and hpsis
        one complex128 [nbands][npw] array per (subsystem, k), subsystem-major.  The arrays stay
        owned by the caller; page-locked ones (e.g. numpy views of pinned torch tensors) are
        copied without staging."""
        if len(psis) != len(hpsis) or len(rhos) == 0:
            raise ValueError("one density per subsystem and one output per orbital block")
        arrs = [np.ascontiguousarray(r, dtype=np.float64) for r in rhos]
        ins = [np.ascontiguousarray(p, dtype=np.complex128) for p in psis]
        for o in hpsis:
            if o.dtype != np.complex128 or not o.flags["C_CONTIGUOUS"]:
                raise ValueError("H psi outputs must be C-contiguous complex128 arrays")
        tr = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        tp = (C.c_void_p * len(ins))(*[a.ctypes.data for a in ins])
        to = (C.c_void_p * len(hpsis))(*[o.ctypes.data for o in hpsis])
        return self._check(self.lib.fde_hot_step_host(self.h, tr, tp, to), "fde_hot_step_host")

    def hot_step(self, use_graph=False):
        return self._check(self.lib.fde_hot_step(self.h, int(bool(use_graph))), "fde_hot_step")

    # ---- learned preconditioner ----------------------------------------------------------
    def set_precond(self, mode):
        return self._check(self.lib.fde_set_precond(self.h, int(mode)), "fde_set_precond")

    def precond_set_weights(self, w):
        a = np.ascontiguousarray(w, dtype=np.float32)
        assert a.size == FDE_PRECOND_PARAMS
        return self._check(self.lib.fde_precond_set_weights(self.h, _hptr(a)), "fde_precond_set_weights")

    def precond_get_weights(self):
        w = np.zeros(FDE_PRECOND_PARAMS, dtype=np.float32)
        wb = np.zeros(FDE_PRECOND_PARAMS, dtype=np.float32)
        self._check(self.lib.fde_precond_get_weights(self.h, _hptr(w), _hptr(wb)), "fde_precond_get_weights")
        return w, wb

    def precond_harvest(self, sub, k, raw):
        a = np.ascontiguousarray(raw, dtype=np.complex128)
        return self._check(self.lib.fde_precond_harvest(self.h, sub, k, _hptr(a), int(a.shape[0])),
                           "fde_precond_harvest")

    def precond_add_pairs(self, sub, k, r, d, tband):
        r = np.ascontiguousarray(r, dtype=np.complex128)
        d = np.ascontiguousarray(d, dtype=np.complex128)
        tb = np.ascontiguousarray(tband, dtype=np.float64)
        return self._check(self.lib.fde_precond_add_pairs(self.h, sub, k, int(r.shape[0]), _hptr(r), _hptr(d),
                                                          _hptr(tb)), "fde_precond_add_pairs")

    def precond_record(self, iterations):
        return self._check(self.lib.fde_precond_record(self.h, int(iterations)), "fde_precond_record")

    def precond_clear(self):
        return self._check(self.lib.fde_precond_clear(self.h), "fde_precond_clear")

    def precond_loss_grad(self):
        g = np.zeros(FDE_PRECOND_PARAMS)
        loss = C.c_double()
        self._check(self.lib.fde_precond_loss_grad(self.h, _hptr(g), C.byref(loss)), "fde_precond_loss_grad")
        return loss.value, g

    def precond_train(self, steps, lr):
        l0, l1 = C.c_double(), C.c_double()
        self._check(self.lib.fde_precond_train(self.h, int(steps), float(lr), C.byref(l0), C.byref(l1)),
                    "fde_precond_train")
        return l0.value, l1.value

    def precond_apply(self, sub, k, r, w, nb, tband):
        tb = np.ascontiguousarray(tband, dtype=np.float64)
        return self._check(self.lib.fde_precond_apply(self.h, sub, k, _dptr(r), _dptr(w), int(nb), _hptr(tb)),
                           "fde_precond_apply")

    def stats(self):
        a, b = C.c_longlong(), C.c_longlong()
        self._check(self.lib.fde_get_stats(self.h, C.byref(a), C.byref(b)), "fde_get_stats")
        return a.value, b.value

    def fft3d(self, data, sign):
        return self._check(self.lib.fde_fft3d(self.h, _dptr(data), int(sign)), "fde_fft3d")

    def fft3d_f64(self, data, sign, arith):
        """The potential build's transform of a complex128 grid: arith 0 FP64, 1 double-float."""
        return self._check(self.lib.fde_fft3d_f64(self.h, _dptr(data), int(sign), int(arith)), "fde_fft3d_f64")

    def launch_count(self):
        n = C.c_longlong()
        self._check(self.lib.fde_launch_count(self.h, C.byref(n)), "fde_launch_count")
        return n.value

    def profile_get(self, kernel):
        n = C.c_int()
        ms = C.c_double()
        self._check(self.lib.fde_profile_get(self.h, kernel.encode(), C.byref(n), C.byref(ms)), "fde_profile_get")
        return n.value, ms.value


def apply_h_local_static(lattice, grid, kfrac, miller, veff, psi, hpsi, nb, stream=None):
    """fde_apply_h_local_static: local H psi with no device allocation (no context).
    miller, veff, psi, hpsi are torch CUDA tensors (int32 [npw][3], float64 grid, complex128
    [nb][npw])."""
    lib = load()
    cell = CellDesc()
    for i in range(3):
        for j in range(3):
            cell.lattice[i][j] = float(lattice[i][j])
        cell.grid[i] = int(grid[i])
    cell.ecut_ha = 0.0
    k = (C.c_double * 3)(*[float(x) for x in kfrac])
    s = lib.fde_apply_h_local_static(C.byref(cell), k, int(miller.shape[0]), _dptr(miller), _dptr(veff),
                                     _dptr(psi), _dptr(hpsi), int(nb), C.c_void_p(stream) if stream else None)
    if s != FDE_OK:
        raise FDEError(s, "fde_apply_h_local_static failed")
    return s


def context_from_workload(wl: workloads.Workload, prec="fp64", stream=None) -> Context:
    """Create a context and add every subsystem of a synthetic workload (marshalling only)."""
    ctx = Context(wl.lattice, wl.grid, wl.ecut, wl.xc, wl.kedf, wl.rho_cut, prec, stream)
    for s in wl.subsystems:
        ctx.add_subsystem(s.pos, s.Z, s.rc, s.nbands, s.kpts, s.wk, s.nelec, s.smearing,
                          s.proj_sigma, s.proj_D, s.smearing_kind, s.proj_Q, s.aug_sigma)
    return ctx


def seed_workload(ctx: Context, wl: workloads.Workload, seed=None):
    """Give every (subsystem, k) its seeded initial orbitals and every subsystem its seeded
    starting density (both generated by ``workloads``)."""
    seed = wl.seed if seed is None else seed
    for I, s in enumerate(wl.subsystems):
        for k in range(s.nk):
            npw = ctx.basis(I, k).shape[0]
            ctx.init_orbitals(I, k, workloads.raw_orbitals(seed, I, k, s.nbands, npw))
        ctx.set_density(I, workloads.initial_density(wl, I))
