"""The allocation-free local H psi entry point against the context path and the oracle.

fde_apply_h_local_static serves callers that cannot call cudaMalloc themselves (code that
runs inside another framework's memory pool or allocator hooks, or an embedding host that
owns every device allocation): it works in fixed device arrays compiled into the library.
This file is collected last so that a failure here leaves every other test already run.
It calls the entry point twice in a row (the arrays keep the previous call's contents)
and compares each result with fde_apply_h of a context on the same inputs and with the
oracle's H psi, within the FP64 tolerance of the parity tests (1e-10 relative per band).
A block of many bands goes through the arrays in several chunks, and sphere lists that do
not fit the grid or are not sorted are refused.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import fde as ofde  # noqa: E402
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


def _band_err(got, want):
    """Largest per-band relative error max_G |got - want| / max_G |want|."""
    return float((np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)).max())


# (cell, subsystem, k-point, bands): the last case has n3 x ncol x nb above the 2^20 complex
# values of the static column scratch, so its bands go through in three chunks.
@pytest.mark.parametrize("make,I,k,nb", [(workloads.plain_fde_32, 1, 0, None),
                                         (workloads.molecule_on_slab_small, 0, 2, None),
                                         (workloads.plain_fde_32, 0, 0, 300)])
def test_static_entry_point_matches_context_path_and_oracle(make, I, k, nb):
    wl = _local_only(make())
    ctx = fde.context_from_workload(wl)
    sy = ofde.System(wl)
    mil = ctx.basis(I, k)
    npw = mil.shape[0]
    s = wl.subsystems[I]
    nb = nb or s.nbands + 3
    d_mil = torch.from_numpy(np.ascontiguousarray(mil, dtype=np.int32)).cuda()
    for call, seed in enumerate((21, 22)):
        vh = _potential(wl, seed)
        v = torch.from_numpy(vh).cuda()
        c = workloads.raw_orbitals(seed, I, k, nb, npw)
        psi = torch.from_numpy(c).cuda()
        ctx.set_veff(I, v)
        want = torch.zeros_like(psi)
        ctx.apply_h(I, k, psi, want, nb)
        got = torch.full_like(psi, float("nan"))
        fde.apply_h_local_static(wl.lattice, wl.grid, s.kpts[k], d_mil, v, psi, got, nb)
        torch.cuda.synchronize()
        g, w = got.cpu().numpy(), want.cpu().numpy()
        assert _band_err(g, w) < 1e-10, call
        pick = [0, nb // 2, nb - 1]  # bands of the first, middle and last chunk
        assert _band_err(g[pick], sy.apply_h(I, k, c[pick], vh)) < 1e-10, call


def test_static_entry_point_rejects_bad_spheres():
    """A sphere that does not fit the grid (the 32^3 cell's sphere with a 16^3 grid: two
    columns would share one plane slot), and the right sphere in the wrong order, both
    return FDE_EINVAL instead of a wrong result."""
    wl = _local_only(workloads.plain_fde_32())
    ctx = fde.context_from_workload(wl)
    mil = np.ascontiguousarray(ctx.basis(0, 0), dtype=np.int32)
    npw = mil.shape[0]
    psi = torch.from_numpy(workloads.raw_orbitals(3, 0, 0, 2, npw)).cuda()
    out = torch.zeros_like(psi)
    small = (16, 16, 16)
    v16 = torch.zeros(small, dtype=torch.float64, device="cuda")
    with pytest.raises(fde.FDEError) as e:
        fde.apply_h_local_static(wl.lattice, small, (0, 0, 0), torch.from_numpy(mil).cuda(), v16, psi, out, 2)
    assert e.value.status == fde.FDE_EINVAL
    v = torch.zeros(tuple(wl.grid), dtype=torch.float64, device="cuda")
    for bad in (mil[::-1].copy(), np.roll(mil, 5, axis=0)):
        with pytest.raises(fde.FDEError) as e:
            fde.apply_h_local_static(wl.lattice, wl.grid, (0, 0, 0), torch.from_numpy(bad).cuda(), v, psi, out, 2)
        assert e.value.status == fde.FDE_EINVAL
    # the arrays still serve a good call afterwards
    fde.apply_h_local_static(wl.lattice, wl.grid, (0, 0, 0), torch.from_numpy(mil).cuda(), v, psi, out, 2)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()


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
