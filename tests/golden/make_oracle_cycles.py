"""Write the oracle's one-cycle freeze-and-thaw energies of the slab + molecule cell.

The FP64 oracle needs about ten minutes of CPU time for this cycle (Lanczos to 1e-13 in
every inner SCF iteration of the smeared 4-k-point slab), too long to repeat inside the
GPU parity run, so its result is stored here.  This script calls only ``oracle/`` and the
seeded input generators; ``oracle_sha256`` records the oracle sources it ran, and a CPU
test fails when they change without the file being written again.

Usage: python tests/golden/make_oracle_cycles.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "ft_cycle_molecule_on_slab_small.json")
OUT_REFRESH = os.path.join(HERE, "refresh_two_layer_slab_small.json")
KEYS = ("F_fde", "E_fde", "E_kin", "E_nl", "E_loc", "E_H", "E_xc", "T_nad", "TS")


# The oracle modules the runs use (the learned-preconditioner oracle is not among them).
CYCLE_MODULES = ("__init__.py", "basis.py", "fde.py", "functionals.py", "kmesh.py", "potentials.py", "refresh.py",
                 "scf.py", "smearing.py")


def oracle_digest() -> str:
    """SHA-256 over the oracle sources of the cycle and the workload generator, in name order."""
    h = hashlib.sha256()
    for f in CYCLE_MODULES:
        with open(os.path.join(ROOT, "oracle", f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    with open(os.path.join(ROOT, "paper_1406_7803_gb300", "workloads.py"), "rb") as fh:
        h.update(b"workloads.py\0" + fh.read())
    return h.hexdigest()


def _write(path, rec):
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


def main() -> int:
    from oracle import fde as ofde, refresh, scf as oscf
    from paper_1406_7803_gb300 import workloads
    digest = oracle_digest()
    ok = True
    if "--refresh-only" not in sys.argv:
        # one Jacobi freeze-and-thaw cycle of the slab + molecule cell (Fermi-Dirac slab)
        wl = workloads.molecule_on_slab_small()
        sy = ofde.System(wl)
        st = oscf.initial_state(sy)
        t0 = time.perf_counter()
        _, en = oscf.freeze_thaw_cycle(sy, st, tol=1e-10)
        rec = {"workload": wl.name, "seed": wl.seed, "tol": 1e-10, "converged": bool(en["converged"]),
               "inner_iters": [int(i) for i in en["iters"]], "seconds": time.perf_counter() - t0,
               "energies": {k: float(en[k]) for k in KEYS}, "oracle_sha256": digest}
        _write(OUT, rec)
        ok &= rec["converged"]
    # the refreshed SCF of the two-layer slab on the full 2 x 2 x 1 mesh with Methfessel-Paxton
    # smearing; its total density and the <Delta rho> against the supersystem KS run
    wl = workloads.two_layer_slab_small()
    sy = ofde.System(wl)
    t0 = time.perf_counter()
    # a few hundred plane waves per k-point: dense LAPACK eigensolves (the same eigenpairs as
    # the Lanczos ones to rounding) keep the run to minutes
    st, en = refresh.scf_default_refresh(sy, oscf.initial_state(sy), tol=1e-10, dense_max=4000)
    sup = workloads.supersystem(wl, extra_bands=4)
    sk = ofde.System(sup)
    st_ks, en_ks = refresh.scf_default_refresh(sk, oscf.initial_state(sk), tol=1e-10, dense_max=4000)
    rec = {"workload": wl.name, "seed": wl.seed, "tol": 1e-10, "converged": bool(en["converged"] and en_ks["converged"]),
           "steps": int(en["iters"]), "ks_steps": int(en_ks["iters"]), "seconds": time.perf_counter() - t0,
           "energies": {k: float(en[k]) for k in KEYS}, "ks_energies": {k: float(en_ks[k]) for k in KEYS},
           "delta_rho": refresh.delta_rho(sy, st.rhos.sum(axis=0), st_ks.rhos[0]), "oracle_sha256": digest}
    _write(OUT_REFRESH, rec)
    ok &= rec["converged"]
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
