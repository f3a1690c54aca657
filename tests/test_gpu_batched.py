"""GPU parity on the batched uneven cell (24 bohr cube, 96^3 grid, 20 Ha): a 54-atom slab with
96 bands x 2 k-points plus 16 molecules of 8..64 bands at Gamma, PBE + revAPBEK, KB projectors.

The embedding potentials of all 17 subsystems come out of one build (V_eff element by element
against the oracle), and one hot step runs H psi for all 778 bands in one launch per phase
(eagerly and replayed from a CUDA graph); sampled bands of every (subsystem, k) block are
compared with the oracle's H psi.  Tolerances: FP64 1e-10, mixed 1e-5 relative per band; for
V_eff 1e-10 (1e-5 mixed) of max|V_eff| widened point by point by ten times the oracle's own
change under rounding-level noise on its FFT gradients (the GGA potentials are ill-conditioned
where the density is low and its gradient near zero: between the sparse slab atoms and in the
vacuum)."""
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


@pytest.fixture(scope="module")
def cell():
    wl = workloads.batched_uneven()
    sy = ofde.System(wl)
    rhos = np.array([workloads.initial_density(wl, I) for I in range(wl.nsub)])
    pot = sy.build_veff(rhos)
    # The GGA potentials of this cell are ill-conditioned where the density is low and its
    # gradient near zero (between the sparse slab atoms, 8 bohr apart, and in the vacuum): there
    # s = |grad rho| / rho^{4/3} and the direction grad rho / |grad rho| follow the rounding of
    # the FFT gradients.  The oracle's own response to that rounding -- additive noise of
    # 1e-15 x max|grad rho| on its gradients, two seeded draws -- widens the FP64 tolerance
    # point by point (it exceeds 1e-11 of max|V_eff| at most points of this cell).
    from oracle import functionals as fn
    rng = np.random.default_rng(17)
    exact_gradient = fn.gradient

    def rounded_gradient(f, lattice):
        g = exact_gradient(f, lattice)
        scale = max(float(np.abs(c).max()) for c in g)
        return [c + 1e-15 * scale * rng.standard_normal(c.shape) for c in g]

    sens = np.zeros_like(pot["veff"])
    fn.gradient = rounded_gradient
    try:
        for _ in range(2):
            p = sy.build_veff(rhos)
            sens = np.maximum(sens, np.abs(np.array(p["veff"]) - np.array(pot["veff"])))
    finally:
        fn.gradient = exact_gradient
    # two draws sample the response; the conditioning itself is a local property, so each
    # point takes the largest response of its 3 x 3 x 3 neighbourhood
    from scipy.ndimage import maximum_filter
    sens = np.array([maximum_filter(x, size=3, mode="wrap") for x in sens])
    pot["sensitivity"] = sens
    return wl, sy, rhos, pot


def band_err(got, want):
    got, want = np.atleast_2d(got), np.atleast_2d(want)
    return float((np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)).max())


def test_batched_uneven_shape(cell):
    """The cell is what the workload states: uneven band counts within 8..64, 17 subsystems."""
    wl, sy, _, _ = cell
    bands = [s.nbands for s in wl.subsystems[1:]]
    assert wl.nsub == 17 and wl.subsystems[0].nk == 2 and wl.subsystems[0].nbands == 96
    assert min(bands) >= 8 and max(bands) <= 64 and len(set(bands)) > 8
    assert wl.band_k_pairs() == 2 * 96 + sum(bands)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_batched_uneven_veff_matches_oracle(cell, prec, tol):
    wl, sy, rhos, pot = cell
    ctx = fde.context_from_workload(wl, prec=prec)
    for I in range(wl.nsub):
        ctx.set_density(I, rhos[I])
    out = torch.zeros((wl.nsub,) + tuple(wl.grid), dtype=torch.float64, device="cuda")
    ctx.build_vemb(out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for I in range(wl.nsub):
        scale = np.abs(pot["veff"][I]).max()
        diff = np.abs(got[I] - pot["veff"][I])
        allowed = tol * scale + 10.0 * pot["sensitivity"][I]
        assert np.all(diff <= allowed), (I, diff.max() / scale, float(np.max(diff / allowed)))
        # where the potential is well conditioned the bound is the plain one
        assert np.median(diff) < 0.1 * tol * scale, (I, float(np.median(diff)) / scale)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
@pytest.mark.parametrize("graph", [False, True])
def test_batched_uneven_hot_step_matches_oracle(cell, prec, tol, graph):
    wl, sy, rhos, pot = cell
    stream = torch.cuda.Stream()
    ctx = fde.context_from_workload(wl, prec=prec, stream=stream.cuda_stream)
    picks = {}
    for I, s in enumerate(wl.subsystems):
        ctx.set_density(I, rhos[I])
        for k in range(s.nk):
            npw = sy.basis[I][k][0].shape[0]
            c = sy.initial_orbitals(I, k, workloads.raw_orbitals(41, I, k, s.nbands, npw))
            ctx.set_orbitals(I, k, torch.from_numpy(c).cuda())
            ctx.sync()  # the copy is read on the context's stream
            picks[I, k] = c[[0, s.nbands // 2, s.nbands - 1]]
    ctx.hot_step(graph)
    if graph:
        ctx.hot_step(graph)  # a replay of the captured graph
    torch.cuda.synchronize()
    for (I, k), c in picks.items():
        s = wl.subsystems[I]
        npw = sy.basis[I][k][0].shape[0]
        out = torch.zeros((s.nbands, npw), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()  # the zero fill runs on torch's stream, the context writes on its own
        ctx.get_hpsi(I, k, out)
        got = out.cpu().numpy()[[0, s.nbands // 2, s.nbands - 1]]
        want = sy.apply_h(I, k, c, pot["veff"][I])
        err = band_err(got, want)
        assert err < tol, (I, k, err)
