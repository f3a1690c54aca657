"""GPU parity of the paper's default density refresh (the subsystem SCF run once per exchange
of the densities) and of the misplaced-electron metric <Delta rho> against a supersystem
Kohn-Sham run on the same grid, on the 2 x 3-atom LDA + TF cell.

The oracle runs the same refreshed SCF (oracle.refresh) from the same seeded start to 1e-10 Ha;
the GPU FP64 path matches every energy term to 1e-8 Ha and <Delta rho> to 1e-8 electrons, the
mixed path (FP32 stage refined in FP64) the free energy to 1e-6 Ha."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import fde as ofde, refresh, scf as oscf  # noqa: E402
from paper_1406_7803_gb300 import fde, workloads  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_7803_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _tiny():
    import dataclasses
    return dataclasses.replace(workloads.plain_fde_32(), grid=(24, 24, 24), ecut=6.0, name="plain-fde-tiny")


@pytest.fixture(scope="module")
def oracle_runs():
    wl = _tiny()
    sy = ofde.System(wl)
    st, en = refresh.scf_default_refresh(sy, oscf.initial_state(sy), tol=1e-10, dense_max=4000)
    assert en["converged"]
    sup = workloads.supersystem(wl, extra_bands=2)
    sys_ks = ofde.System(sup)
    st_ks, en_ks = refresh.scf_default_refresh(sys_ks, oscf.initial_state(sys_ks), tol=1e-10, dense_max=4000)
    assert en_ks["converged"]
    drho = refresh.delta_rho(sy, st.rhos.sum(axis=0), st_ks.rhos[0])
    return wl, sup, en, en_ks, drho


def _run(wl, prec, tol):
    ctx = fde.context_from_workload(wl, prec=prec)
    fde.seed_workload(ctx, wl)
    s, e = ctx.scf_refresh(tol, 300)
    assert s == fde.FDE_OK
    return ctx, e


def test_refresh_scf_matches_oracle(oracle_runs):
    wl, sup, en, en_ks, drho = oracle_runs
    ctx, got = _run(wl, "fp64", 1e-10)
    diffs = {k: got[k] - en[k] for k in ("F_fde", "E_fde", "E_kin", "E_loc", "E_H", "E_xc", "T_nad", "E_nn")}
    assert all(abs(d) < 1e-8 for d in diffs.values()), diffs
    ks, got_ks = _run(sup, "fp64", 1e-10)
    assert abs(got_ks["F_fde"] - en_ks["F_fde"]) < 1e-8
    assert got_ks["T_nad"] == 0.0 or abs(got_ks["T_nad"]) < 1e-14
    rho_ks = torch.zeros(tuple(wl.grid), dtype=torch.float64, device="cuda")
    ks.get_density(-1, rho_ks)
    d = ctx.delta_rho(rho_ks)
    assert abs(d - drho) < 1e-8, (d, drho)
    assert 1e-4 < d < 0.5 * sum(s.nelec for s in wl.subsystems)
    # a single-subsystem context measured against its own density misplaces nothing
    assert ks.delta_rho(rho_ks) < 1e-15


def test_refresh_scf_mixed_matches_oracle(oracle_runs):
    wl, sup, en, en_ks, drho = oracle_runs
    ctx, got = _run(wl, "mixed", 1e-8)
    assert abs(got["F_fde"] - en["F_fde"]) < 1e-6, (got["F_fde"], en["F_fde"])
