"""GPU parity of Methfessel-Paxton smearing and of symmetry-reduced Monkhorst-Pack sampling
(Computational Details: 2 x 2 x 1 Monkhorst-Pack mesh for the periodic systems, Methfessel-Paxton
smearing of 1e-2 Ry for the metallic subsystems).

Cell: the two layers of the small slab as two subsystems (each layer is mirror-symmetric in x
and y about the origin).  The oracle's refreshed SCF on the full 4-point mesh (stored golden
energies, tests/golden/refresh_two_layer_slab_small.json) is matched by the library on the full
mesh, on the 2-point mesh that time reversal leaves, and on the single point that the mirrors
leave with the densities averaged over the mirror group: every energy term within 1e-8 Ha in
FP64, the free energy within 1e-6 Ha in the mixed path, and <Delta rho> against the
supersystem KS run within 1e-8 electrons."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1406_7803_gb300 import fde, workloads  # noqa: E402

KEYS = ("F_fde", "E_fde", "E_kin", "E_nl", "E_loc", "E_H", "E_xc", "T_nad", "TS")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_7803_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(os.path.dirname(__file__), "golden", "refresh_two_layer_slab_small.json")) as f:
        rec = json.load(f)
    wl = workloads.two_layer_slab_small()
    assert rec["workload"] == wl.name and rec["converged"]
    return wl, rec


def _mesh(wl, ops, tr):
    k, w = fde.host_kmesh((2, 2, 1), (0, 0, 0), tr, ops)
    out = wl
    for I in range(wl.nsub):
        out = workloads.with_kpoints(out, I, k, w)
    return out


def _run(wl, prec, tol, ops=None):
    ctx = fde.context_from_workload(wl, prec=prec)
    if ops:
        ctx.set_symmetry(ops)
    fde.seed_workload(ctx, wl)
    s, e = ctx.scf_refresh(tol, 600)
    assert s == fde.FDE_OK
    return ctx, e


@pytest.mark.parametrize("mesh", ["full", "time_reversal", "mirrors"])
def test_refresh_with_methfessel_paxton_matches_oracle(golden, mesh):
    wl, rec = golden
    L = np.diag(wl.lattice)
    ops = [o for o in fde.host_symmetry_ops(L, wl.subsystems[0].pos, wl.subsystems[0].Z)]
    assert ops == [0, 1, 2, 3]
    if mesh == "full":
        run, sym = wl, None
    elif mesh == "time_reversal":
        run, sym = _mesh(wl, (), True), None
        assert run.subsystems[0].nk == 2
    else:
        run, sym = _mesh(wl, (1, 2, 3), True), ops
        assert run.subsystems[0].nk == 1
    ctx, got = _run(run, "fp64", 1e-10, sym)
    diffs = {k: got[k] - rec["energies"][k] for k in KEYS}
    assert all(abs(d) < 1e-8 for d in diffs.values()), (mesh, diffs)
    if mesh == "mirrors":
        # <Delta rho> against the supersystem KS run, itself on the reduced mesh
        sup = workloads.supersystem(run, extra_bands=4)
        ks, got_ks = _run(sup, "fp64", 1e-10, sym)
        assert abs(got_ks["F_fde"] - rec["ks_energies"]["F_fde"]) < 1e-8
        rho_ks = torch.zeros(tuple(wl.grid), dtype=torch.float64, device="cuda")
        ks.get_density(-1, rho_ks)
        assert abs(ctx.delta_rho(rho_ks) - rec["delta_rho"]) < 1e-8


def test_refresh_mixed_on_the_reduced_mesh(golden):
    wl, rec = golden
    run = _mesh(wl, (1, 2, 3), True)
    _, got = _run(run, "mixed", 1e-8, [0, 1, 2, 3])
    assert abs(got["F_fde"] - rec["energies"]["F_fde"]) < 1e-6


def test_symmetry_must_hold_for_every_subsystem():
    wl = workloads.molecule_on_slab_small()
    ctx = fde.context_from_workload(wl)
    for bad in ([0, 1], [0, 1, 2], [1, 2, 3]):  # breaks the molecule / not a group / no identity
        with pytest.raises(fde.FDEError) as e:
            ctx.set_symmetry(bad)
        assert e.value.status == fde.FDE_EINVAL
    ctx.set_symmetry([0])  # the identity alone is always accepted
