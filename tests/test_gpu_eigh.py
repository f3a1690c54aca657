"""GPU parity of the FP64 Rayleigh-Ritz eigensolver (tridiagonalisation, bisection, inverse
iteration) against LAPACK, including exactly degenerate spectra."""
import numpy as np
import pytest
import scipy.linalg

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1406_7803_gb300 import fde, workloads  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1406_7803_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return fde.Context(np.diag([5.0] * 3), (8, 8, 8), 1.0, workloads.XC_LDA, workloads.KEDF_TF)


def _hermitian(n, seed, degenerate=False):
    rng = np.random.default_rng(seed)
    if not degenerate:
        a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        return (a + a.conj().T) / 2
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(-5, 5, n))
    lam[3:7] = lam[3]  # a four-fold degenerate level
    lam[10:12] = lam[10] + 1e-12  # a nearly degenerate pair
    return (q * lam) @ q.conj().T


@pytest.mark.parametrize("n,nvec,deg", [(1, 1, False), (2, 1, False), (7, 7, False), (64, 20, False),
                                         (128, 64, True), (192, 64, True), (192, 192, False)])
def test_dense_eigh_matches_lapack(ctx, n, nvec, deg):
    A = _hermitian(n, n + nvec, deg and n > 12)
    w_ref, v_ref = scipy.linalg.eigh(A)
    dA = torch.from_numpy(A).cuda()
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    V = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    ctx.dense_eigh(dA, nvec, w, V)
    w = w.cpu().numpy()
    V = V.cpu().numpy()[:, :nvec]
    scale = max(1.0, np.abs(w_ref).max())
    assert np.abs(w - w_ref).max() < 1e-12 * scale
    # eigen-residuals and orthonormality of the computed vectors
    assert np.abs(A @ V - V * w[:nvec]).max() < 1e-11 * scale
    assert np.abs(V.conj().T @ V - np.eye(nvec)).max() < 1e-12
