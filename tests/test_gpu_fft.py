"""GPU parity of the library's 3D transforms against the oracle's conventions.

Every grid shape below goes through the compile-time-length kernels (24, 32, 60, 72, 96,
144, 180, 288) or the runtime-length fallback (30, 40, 50), in both precisions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import basis  # noqa: E402
from paper_1406_7803_gb300 import fde, workloads  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_7803_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


SHAPES = [(24, 24, 60), (32, 32, 32), (72, 72, 180), (96, 96, 96), (96, 96, 144), (32, 32, 288), (30, 40, 50),
          (72, 72, 24)]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
@pytest.mark.parametrize("shape", SHAPES)
def test_fft3d_matches_oracle(shape, prec, tol):
    lat = np.diag([10.0, 11.0, 12.0])
    ctx = fde.Context(lat, shape, 1.0, workloads.XC_LDA, workloads.KEDF_TF, prec=prec)
    rng = np.random.default_rng(sum(shape))
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    for sign, want in ((-1, basis.G_from_r(f)), (+1, basis.r_from_G(f))):
        d = torch.from_numpy(f).to(device="cuda", dtype=dt)
        ctx.fft3d(d, sign)
        torch.cuda.synchronize()
        got = d.to(torch.complex128).cpu().numpy()
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < tol, (shape, prec, sign, err)


DD_SHAPES = [(24, 24, 60), (72, 72, 180), (96, 96, 96), (32, 32, 288), (144, 96, 32)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", DD_SHAPES)
def test_potential_build_transforms_match_oracle(shape, prec):
    """The potential build's transforms of FP64 grids: native FP64 to 1e-13 of the largest
    output, double-float (two floats per value on the FP32 pipes, as the mixed path transforms
    the densities and their gradients) to 2e-13 -- far below FP32's ~1e-6 (above), near FP64.
    The input spans 30 orders of magnitude, like densities between the atoms and the vacuum."""
    lat = np.diag([10.0, 11.0, 12.0])
    ctx = fde.Context(lat, shape, 1.0, workloads.XC_LDA, workloads.KEDF_TF, prec=prec)
    rng = np.random.default_rng(sum(shape) + 1)
    f = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 10.0 ** rng.uniform(-30, 0, shape)
    for arith, tol in ((0, 1e-13), (1, 2e-13)):
        for sign, want in ((-1, basis.G_from_r(f)), (+1, basis.r_from_G(f))):
            d = torch.from_numpy(f).to("cuda")
            ctx.fft3d_f64(d, sign, arith)
            torch.cuda.synchronize()
            got = d.cpu().numpy()
            err = np.abs(got - want).max() / np.abs(want).max()
            assert err < tol, (shape, prec, arith, sign, err)
