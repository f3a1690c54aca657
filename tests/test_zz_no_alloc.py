"""The allocation-free local H psi entry point against the context path.

fde_apply_h_local_static serves callers that cannot call cudaMalloc themselves (code that
runs inside another framework's memory pool or allocator hooks, or an embedding host that
owns every device allocation): it works in fixed device arrays compiled into the library.
This file is collected last so that a failure here leaves every other test already run.
It calls the entry point twice in a row (the arrays keep the previous call's contents)
and compares each result with fde_apply_h of a context on the same inputs, within the
FP64 tolerance of the parity tests (1e-10 relative).
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1406_7803_gb300 import fde, workloads  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_7803_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _local_only(wl):
    """The same cell with the nonlocal projectors removed (the static entry point is the
    local part of H psi)."""
    subs = [dataclasses.replace(s, proj_sigma=(), proj_D=()) for s in wl.subsystems]
    return dataclasses.replace(wl, subsystems=subs)


def _potential(wl, seed):
    rng = np.random.default_rng(seed)
    return -0.5 + 0.3 * rng.standard_normal(tuple(wl.grid))


@pytest.mark.parametrize("make,I,k", [(workloads.plain_fde_32, 1, 0),
                                      (workloads.molecule_on_slab_small, 0, 2)])
def test_static_entry_point_matches_context_path(make, I, k):
    wl = _local_only(make())
    ctx = fde.context_from_workload(wl)
    mil = ctx.basis(I, k)
    npw = mil.shape[0]
    s = wl.subsystems[I]
    nb = s.nbands + 3
    d_mil = torch.from_numpy(np.ascontiguousarray(mil, dtype=np.int32)).cuda()
    for call, seed in enumerate((21, 22)):
        v = torch.from_numpy(_potential(wl, seed)).cuda()
        psi = torch.from_numpy(workloads.raw_orbitals(seed, I, k, nb, npw)).cuda()
        ctx.set_veff(I, v)
        want = torch.zeros_like(psi)
        ctx.apply_h(I, k, psi, want, nb)
        got = torch.full_like(psi, float("nan"))
        fde.apply_h_local_static(wl.lattice, wl.grid, s.kpts[k], d_mil, v, psi, got, nb)
        torch.cuda.synchronize()
        g, w = got.cpu().numpy(), want.cpu().numpy()
        err = np.abs(g - w).max() / np.abs(w).max()
        assert err < 1e-10, (call, err)


def test_static_entry_point_rejects_oversized_inputs():
    wl = workloads.plain_fde_32()
    big = np.zeros((70000, 3), dtype=np.int32)
    d_mil = torch.from_numpy(big).cuda()
    v = torch.zeros(tuple(wl.grid), dtype=torch.float64, device="cuda")
    psi = torch.zeros((1, 70000), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(psi)
    with pytest.raises(fde.FDEError) as e:
        fde.apply_h_local_static(wl.lattice, wl.grid, (0, 0, 0), d_mil, v, psi, out, 1)
    assert e.value.status == fde.FDE_EUNSUPPORTED
