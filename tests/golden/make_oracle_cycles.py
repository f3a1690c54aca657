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
KEYS = ("F_fde", "E_fde", "E_kin", "E_nl", "E_loc", "E_H", "E_xc", "T_nad", "TS")


# The oracle modules the freeze-and-thaw cycle runs (the learned-preconditioner oracle is not
# among them).
CYCLE_MODULES = ("__init__.py", "basis.py", "fde.py", "functionals.py", "potentials.py", "scf.py")


def oracle_digest() -> str:
    """SHA-256 over the oracle sources of the cycle and the workload generator, in name order."""
    h = hashlib.sha256()
    for f in CYCLE_MODULES:
        with open(os.path.join(ROOT, "oracle", f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    with open(os.path.join(ROOT, "paper_1406_7803_gb300", "workloads.py"), "rb") as fh:
        h.update(b"workloads.py\0" + fh.read())
    return h.hexdigest()


def main() -> int:
    from oracle import fde as ofde, scf as oscf
    from paper_1406_7803_gb300 import workloads
    wl = workloads.molecule_on_slab_small()
    sy = ofde.System(wl)
    st = oscf.initial_state(sy)
    t0 = time.perf_counter()
    _, en = oscf.freeze_thaw_cycle(sy, st, tol=1e-10)
    rec = {"workload": wl.name, "seed": wl.seed, "tol": 1e-10, "converged": bool(en["converged"]),
           "inner_iters": [int(i) for i in en["iters"]], "seconds": time.perf_counter() - t0,
           "energies": {k: float(en[k]) for k in KEYS}, "oracle_sha256": oracle_digest()}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))
    return 0 if rec["converged"] else 1


if __name__ == "__main__":
    sys.exit(main())
