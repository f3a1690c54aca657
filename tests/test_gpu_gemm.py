"""Band-block inner products C = A^H B (Gram, subspace Hamiltonian, projector contraction)
on the three FP32 paths -- CUDA cores, tensor cores with TF32 operands, tensor cores with
split-TF32 operands -- against the FP64 product of the same FP32 inputs.

Error measure: max |C - C_ref| / max_i |a_i| max_j |b_j| (the scale of one inner product).
FP32 products summed in FP32 over a K-chunk carry ~sqrt(chunk) 6e-8 of that scale; TF32
operands (10 explicit mantissa bits) ~2^-11 per product."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1406_7803_gb300 import fde, workloads  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1406_7803_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return fde.Context(np.diag([5.0] * 3), (8, 8, 8), 1.0, workloads.XC_LDA, workloads.KEDF_TF, prec="mixed")


def _draw(rng, rows, ld, K):
    a = np.zeros((rows, ld), dtype=np.complex64)
    a[:, :K] = (rng.standard_normal((rows, K)) + 1j * rng.standard_normal((rows, K))).astype(np.complex64)
    # a spread of row scales, as in residual blocks
    a[:, :K] *= np.exp(rng.uniform(-3, 3, size=(rows, 1))).astype(np.float32)
    return a


SHAPES = [
    # m, n, K, lda, ldb
    (72, 64, 2777, 2777, 2777),      # projectors x bands of the 10-bohr cell (odd K and ld)
    (192, 192, 5003, 5003, 5003),    # Gram of a 3 x 64 search space: 2 x 3 tiles, ragged K tail
    (130, 65, 1000, 1003, 1001),     # ragged m and n tiles, padded rows
    (1, 1, 1, 1, 1),                 # degenerate
    (7, 3, 17, 18, 17),              # one partial k-tile
    (64, 12, 43613, 43613, 43613),   # molecule bands x slab-size sphere: many K-splits
]


@pytest.mark.parametrize("m,n,K,lda,ldb", SHAPES)
def test_products_match_fp64(ctx, m, n, K, lda, ldb):
    rng = np.random.default_rng([m, n, K])
    a = _draw(rng, m, lda, K)
    b = _draw(rng, n, ldb, K)
    ref = a[:, :K].astype(np.complex128).conj() @ b[:, :K].astype(np.complex128).T
    scale = np.linalg.norm(a, axis=1).max() * np.linalg.norm(b, axis=1).max()
    dA, dB = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    err = {}
    for path in (0, 1, 3):
        out = torch.full((m, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        ctx.gemm_hn_f32(dA, dB, K, out, path)
        err[path] = float(np.abs(out.cpu().numpy() - ref).max() / scale)
    assert err[0] < 1e-5 and err[3] < 1e-5, err
    assert err[1] < 4e-3, err
    if K >= 64:
        # the lo parts are doing their job
        assert err[3] < err[1] / 20, err


def test_gram_is_hermitian_and_repeatable(ctx):
    rng = np.random.default_rng(7)
    K = 20011
    a = _draw(rng, 150, K, K)
    dA = torch.from_numpy(a).cuda()
    c1 = torch.zeros((150, 150), dtype=torch.complex128, device="cuda")
    c2 = torch.zeros_like(c1)
    ctx.gemm_hn_f32(dA, dA, K, c1, 3)
    ctx.gemm_hn_f32(dA, dA, K, c2, 3)
    g = c1.cpu().numpy()
    # fixed split and reduction order: bit-identical repeats
    assert np.array_equal(g, c2.cpu().numpy())
    scale = np.linalg.norm(a, axis=1).max() ** 2
    assert np.abs(g - g.conj().T).max() / scale < 1e-5
    assert np.all(np.diag(g).real > 0)
