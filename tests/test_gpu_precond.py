"""Learned preconditioner: GPU forward/backward kernels against the oracle, training on
pairs harvested from converged eigensolves, and what the trained network gains over the
kinetic preconditioner it replaces (which stays the fallback and the yardstick)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import fde as ofde, precond as opre, scf as oscf  # noqa: E402
from paper_1406_7803_gb300 import fde, workloads  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1406_7803_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)


def _unflat(v):
    out, o = [], 0
    for fi, fo in opre.LAYERS:
        W = v[o:o + fi * fo].reshape(fo, fi).astype(np.float64)
        o += fi * fo
        b = v[o:o + fo].astype(np.float64)
        o += fo
        out.append([W, b])
    return out


@pytest.fixture(scope="module")
def pairs():
    """Oracle training pairs on the molecule-on-slab cell (molecule at Gamma, slab k=1)."""
    wl = workloads.molecule_on_slab_small()
    sy = ofde.System(wl)
    st = oscf.initial_state(sy)
    pot = sy.build_veff(st.rhos)
    out = []
    for I, k, n in ((1, 0, 3), (0, 1, 4)):
        s = sy.subs[I]
        w, v = oscf.eig_dense(sy, I, k, pot["veff"][I], s.nbands)
        r, d = opre.training_pairs(sy, I, k, pot["veff"][I], v, w, n, seed=17)
        kin = sy.basis[I][k][1]
        tb = np.real(np.sum(kin[None, :] * np.abs(v[:n]) ** 2, axis=1))
        out.append((I, k, r, d, tb, kin))
    return wl, out


def _weights(seed=4):
    p = opre.init_params(seed)
    rng = np.random.default_rng(seed)
    p[-1][0] = 0.2 * rng.standard_normal(p[-1][0].shape)
    p[-1][1] = np.array([0.1])
    return _flat(p)


@pytest.mark.parametrize("path", [1, 0])
def test_loss_and_gradient_match_oracle(pairs, path):
    """Loss and gradient of the training kernels against the oracle's backward pass (FP64 on
    the FP32 master weights): on the tensor cores (path 1: the hidden layers, the
    back-propagated errors and the weight gradients as BF16 MMAs with split operands) and on
    the CUDA cores (path 0)."""
    wl, data = pairs
    w = _weights()
    ctx = fde.context_from_workload(wl)
    ctx.precond_set_weights(w)
    for I, k, r, d, tb, _ in data:
        ctx.precond_add_pairs(I, k, r, d, tb)
    fde.set_precond_path(path)
    try:
        loss, g = ctx.precond_loss_grad()
    finally:
        fde.set_precond_path(1)
    p = _unflat(w)  # the FP32 master weights, evaluated in FP64
    L, gr = 0.0, None
    for I, k, r, d, tb, kin in data:
        l, gi = opre.backward(p, kin, tb, r, d)
        L += l
        gflat = np.concatenate([np.concatenate([a.ravel(), b.ravel()]) for a, b in gi])
        gr = gflat if gr is None else gr + gflat
    assert abs(loss - L) < 1e-5 * abs(L)
    assert np.abs(g - gr).max() < 2e-4 * np.abs(gr).max(), np.abs(g - gr).max() / np.abs(gr).max()


@pytest.mark.parametrize("path", [1, 0])
def test_inference_matches_oracle_with_bf16_weights(pairs, path):
    """Inference with the bf16 weights against the oracle's FP64 evaluation of the same
    weights: on the tensor cores (path 1: the two hidden layers as BF16 MMAs with the
    activations split into two bf16 terms) and on the CUDA cores (path 0)."""
    wl, data = pairs
    w = _weights(6)
    ctx = fde.context_from_workload(wl)
    ctx.precond_set_weights(w)
    _, wb = ctx.precond_get_weights()
    assert np.array_equal(wb.astype(np.float64), opre.bf16_round(w))
    pb = _unflat(opre.bf16_round(w))
    fde.set_precond_path(path)
    try:
        for I, k, r, d, tb, kin in data:
            want = opre.apply(pb, kin, tb, r)
            rr = torch.from_numpy(r).cuda()
            out = torch.zeros_like(rr)
            ctx.precond_apply(I, k, rr, out, r.shape[0], tb)
            got = out.cpu().numpy()
            assert np.abs(got - want).max() < 2e-5 * np.abs(want).max(), (path, np.abs(got - want).max() / np.abs(want).max())
    finally:
        fde.set_precond_path(1)


def test_tensor_core_inference_timeout_returns_etimeout_and_recovers(pairs):
    """The tensor-core inference waits for each layer's MMAs with a bounded poll; with the
    limit at 0 the first wait runs out, the kernel drains its issued MMAs (full bound), frees
    its tensor memory and the call returns FDE_ETIMEOUT; with the default limit the next call
    is correct again."""
    wl, data = pairs
    w = _weights(6)
    ctx = fde.context_from_workload(wl)
    ctx.precond_set_weights(w)
    pb = _unflat(opre.bf16_round(w))
    I, k, r, d, tb, kin = data[1]
    rr = torch.from_numpy(r).cuda()
    out = torch.zeros_like(rr)
    fde.set_tc_wait_limit(0)
    try:
        with pytest.raises(fde.FDEError) as e:
            ctx.precond_apply(I, k, rr, out, r.shape[0], tb)
        assert e.value.status == fde.FDE_ETIMEOUT
    finally:
        fde.set_tc_wait_limit(-1)
    ctx.precond_apply(I, k, rr, out, r.shape[0], tb)
    want = opre.apply(pb, kin, tb, r)
    assert np.abs(out.cpu().numpy() - want).max() < 2e-5 * np.abs(want).max()


def _solve_all(ctx, wl, precond, tol):
    its, eigs = 0, []
    for I, s in enumerate(wl.subsystems):
        for k in range(s.nk):
            st, it = ctx.subspace_solve(I, k, tol, 300, precond)
            assert st == fde.FDE_OK
            its += it
            npw = ctx.basis(I, k).shape[0]
            buf = torch.zeros((s.nbands, npw), dtype=torch.complex128, device="cuda")
            e, _ = ctx.get_orbitals(I, k, buf, s.nbands)
            eigs.append(e)
    return its, np.concatenate(eigs)


def test_trained_network_gain_over_kinetic_preconditioner():
    """Train on (residual, error) pairs recorded over whole eigensolves of the molecule-on-slab
    cell, then solve the same eigenproblems from the same seeded start with both
    preconditioners: identical eigenvalues (the answer does not change); the iteration counts
    are the gain.  Pairs from the first iterates only (8 per solve) teach the network the
    early error spectrum and it then slows the late iterations; pairs over the whole
    trajectory do not."""
    wl = workloads.molecule_on_slab_small()
    ctx = fde.context_from_workload(wl)
    fde.seed_workload(ctx, wl)
    ctx.build_vemb()
    ctx.precond_record(60)  # (residual, error) pairs of every iteration of every solve
    it_tpa, e_tpa = _solve_all(ctx, wl, fde.FDE_PRECOND_TPA, 1e-8)
    ctx.precond_record(0)
    ctx.precond_set_weights(_flat(opre.init_params(0)))
    l0, l1 = ctx.precond_train(400, 3e-3)
    assert l1 < l0
    fde.seed_workload(ctx, wl)
    it_learned, e_learned = _solve_all(ctx, wl, fde.FDE_PRECOND_LEARNED, 1e-8)
    print(f"\nkinetic preconditioner: {it_tpa} iterations; learned: {it_learned} iterations; "
          f"training loss {l0:.4g} -> {l1:.4g}")
    assert np.abs(e_learned - e_tpa).max() < 1e-8
    assert it_learned <= it_tpa


def test_learned_preconditioner_on_the_full_size_cell():
    """The network trained on the benchmark cell's own solves (72 x 72 x 180, FP64): (residual,
    error) pairs from 12 iterates of every (subsystem, k) solve started from the seeded
    orbitals, 200 Adam steps on the tensor cores, then every solve again from another seeded
    start with both preconditioners.  The eigenvalues must not change; the band-applies and
    iterations of both are printed (the network does not pay on this cell: see the design
    notes)."""
    wl = workloads.molecule_on_slab()
    ctx = fde.context_from_workload(wl, prec="fp64")

    def solve_all(precond, seed):
        fde.seed_workload(ctx, wl, seed=seed)
        ctx.build_vemb()
        _, b0 = ctx.stats()
        its, eigs = 0, []
        for I, s in enumerate(wl.subsystems):
            for k in range(s.nk):
                st, it = ctx.subspace_solve(I, k, 1e-7, 400, precond)
                assert st == fde.FDE_OK
                its += it
                npw = ctx.basis(I, k).shape[0]
                buf = torch.zeros((s.nbands, npw), dtype=torch.complex128, device="cuda")
                e, _ = ctx.get_orbitals(I, k, buf, s.nbands)
                eigs.append(e)
        _, b1 = ctx.stats()
        return its, b1 - b0, np.concatenate(eigs)

    ctx.precond_record(12)
    solve_all(fde.FDE_PRECOND_TPA, wl.seed)
    ctx.precond_record(0)
    ctx.precond_set_weights(_flat(opre.init_params(0)))
    l0, l1 = ctx.precond_train(200, 3e-3)
    assert l1 < l0
    it_t, ba_t, e_t = solve_all(fde.FDE_PRECOND_TPA, 2002)
    it_l, ba_l, e_l = solve_all(fde.FDE_PRECOND_LEARNED, 2002)
    print(f"\nbenchmark cell, FP64 solves to 1e-7: kinetic preconditioner {it_t} iterations, {ba_t} "
          f"band-applies; learned {it_l} iterations, {ba_l} band-applies; training loss {l0:.4g} -> {l1:.4g}")
    assert np.abs(e_l - e_t).max() < 1e-9
