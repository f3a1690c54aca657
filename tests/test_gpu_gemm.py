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


ROT_SHAPES = [
    # m (input rows), n (output rows), K, ldx, ldy, alpha, beta
    (72, 64, 2777, 2777, 2777, 1.0, 1.0),      # projector expansion added to H psi
    (192, 64, 5003, 5003, 5003, 1.0, 0.0),     # rotation of a 3 x 64 search space onto 64 bands
    (64, 130, 1000, 1001, 1003, -1.0, 1.0),    # two output-row tiles, ragged G tile, padded rows
    (1, 1, 1, 1, 1, 0.5, 0.0),                 # degenerate
    (17, 3, 129, 130, 129, 1.0, -2.0),         # partial k-tile, one G past a tile
]


@pytest.mark.parametrize("m,n,K,ldx,ldy,alpha,beta", ROT_SHAPES)
def test_combinations_match_fp64(ctx, m, n, K, ldx, ldy, alpha, beta):
    """Y = alpha sum_i U_ij X_i + beta Y.  Error measure: max |Y - Y_ref| over
    (|alpha| max_j |U_:j| max_g |X_:g| + |beta| max |Y|)."""
    rng = np.random.default_rng([m, n, K, 3])
    x = _draw(rng, m, ldx, K)
    u = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(m)
    y0 = _draw(rng, n, ldy, K)
    ref = y0.astype(np.complex128).copy()
    ref[:, :K] = alpha * (u.T @ x[:, :K].astype(np.complex128)) + beta * y0[:, :K]
    scale = abs(alpha) * np.linalg.norm(u, axis=0).max() * np.linalg.norm(x, axis=0).max() + abs(beta) * np.abs(y0).max()
    dX, dU = torch.from_numpy(x).cuda(), torch.from_numpy(u).cuda()
    err = {}
    for path in (0, 1, 3):
        dY = torch.from_numpy(y0.copy()).cuda()
        ctx.gemm_rot_f32(dX, dU, K, dY, alpha, beta, path)
        got = dY.cpu().numpy()
        assert np.array_equal(got[:, K:], y0[:, K:]), "columns beyond K must be untouched"
        err[path] = float(np.abs(got - ref).max() / scale)
    assert err[0] < 1e-5 and err[3] < 1e-5, err
    assert err[1] < 4e-3, err
    if m >= 16:
        assert err[3] < err[1] / 20, err


def test_stage_wait_timeout_returns_etimeout_and_recovers(ctx):
    """Every device wait of the tensor-core products is bounded.  With the stage-wait poll
    limit at 0, a product with several k-tiles per CTA runs out at its first stage wait: the
    kernel stops issuing, drains the MMAs it issued (full bound), frees its tensor memory,
    writes nothing, and the call returns FDE_ETIMEOUT.  Calls with the default limit then
    give correct results again (the context, the stream and tensor memory are intact)."""
    rng = np.random.default_rng(77)
    m, n, K = 64, 64, 4096
    a = _draw(rng, m, K, K)
    b = _draw(rng, n, K, K)
    dA, dB = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = torch.zeros((m, n), dtype=torch.complex128, device="cuda")
    U = torch.from_numpy(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).cuda()
    Y = torch.zeros((n, K), dtype=torch.complex64, device="cuda")
    fde.set_tc_wait_limit(0)
    try:
        with pytest.raises(fde.FDEError) as e:
            ctx.gemm_hn_f32(dA, dB, K, out, 3)
        assert e.value.status == fde.FDE_ETIMEOUT
        with pytest.raises(fde.FDEError) as e:
            ctx.gemm_rot_f32(dA, U, K, Y, 1.0, 0.0, 3)
        assert e.value.status == fde.FDE_ETIMEOUT
    finally:
        fde.set_tc_wait_limit(-1)
    ref = a.astype(np.complex128).conj() @ b.astype(np.complex128).T
    scale = np.linalg.norm(a, axis=1).max() * np.linalg.norm(b, axis=1).max()
    ctx.gemm_hn_f32(dA, dB, K, out, 3)
    assert np.abs(out.cpu().numpy() - ref).max() / scale < 1e-5
    ctx.gemm_rot_f32(dA, U, K, Y, 1.0, 0.0, 3)
    u = U.cpu().numpy()
    want = u.T @ a.astype(np.complex128)
    rscale = np.linalg.norm(u, axis=0).max() * np.linalg.norm(a, axis=0).max()
    assert np.abs(Y.cpu().numpy() - want).max() / rscale < 1e-5
