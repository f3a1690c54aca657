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
