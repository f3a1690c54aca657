"""Pins of the learned-preconditioner oracle (CPU only)."""
import numpy as np
import pytest

from oracle import fde as ofde, precond, scf
from paper_1406_7803_gb300 import workloads


def test_bf16_round_to_nearest_even():
    one = 1.0
    ulp = 2.0 ** -7  # bfloat16 spacing at 1
    vals = np.array([one, one + ulp / 2, one + 1.5 * ulp, one + ulp / 4, -3.0, 1e-3], dtype=np.float32)
    got = precond.bf16_round(vals)
    assert got[0] == 1.0
    assert got[1] == 1.0  # tie -> even (1.0)
    assert got[2] == one + 2 * ulp  # tie -> even (odd mantissa rounds up)
    assert got[3] == 1.0
    assert got[4] == -3.0
    assert abs(got[5] - 1e-3) <= 1e-3 * 2 ** -8


def test_zero_output_layer_is_the_kinetic_preconditioner():
    rng = np.random.default_rng(1)
    kin = rng.uniform(0, 20, 50)
    r = rng.standard_normal((3, 50)) + 1j * rng.standard_normal((3, 50))
    tb = np.array([0.5, 1.3, 4.0])
    p = precond.init_params(3)
    m = precond.multiplier(p, kin, tb, r)
    y = kin[None, :] / tb[:, None]
    assert np.allclose(m, precond.tpa(y), rtol=1e-15)
    # TPA limits: K(0) = 1 and K(y) -> 1/(2y) for large y
    assert precond.tpa(np.array([0.0]))[0] == 1.0
    assert np.isclose(precond.tpa(np.array([1e6]))[0] * 2e6, 1.0, rtol=1e-5)


def test_kinetic_preconditioner_values_fix_every_coefficient():
    """The numerator of K is 27 sum_{n<4} (2y/3)^n, so K(3/2) = 4 x 27 / (4 x 27 + 81) = 4/7
    and K(1) = 65/81 (hand-evaluated); with K(0) = 1, the 1/(2y) tail and 1 - K = 16 y^4 / 27
    + O(y^5) at small y these values fix all five coefficients: a wrong one fails here."""
    K = precond.tpa(np.array([0.0, 1.0, 1.5, 1e-3, 1e7]))
    assert K[0] == 1.0
    assert abs(K[1] - 65.0 / 81.0) < 1e-15
    assert abs(K[2] - 4.0 / 7.0) < 1e-15
    assert abs((1.0 - K[3]) / 1e-12 - 16.0 / 27.0) < 1e-3
    assert abs(K[4] * 2e7 - 1.0) < 1e-6
    # monotone decreasing between the limits, never negative
    y = np.linspace(0.0, 50.0, 5001)
    k = precond.tpa(y)
    assert np.all(np.diff(k) < 0) and np.all(k > 0)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(2)
    kin = rng.uniform(0, 10, 40)
    r = rng.standard_normal((2, 40)) + 1j * rng.standard_normal((2, 40))
    d = rng.standard_normal((2, 40)) + 1j * rng.standard_normal((2, 40))
    tb = np.array([0.7, 2.1])
    p = precond.init_params(5)
    p[-1][0] = 0.1 * rng.standard_normal(p[-1][0].shape)  # a non-trivial output layer
    L, g = precond.backward(p, kin, tb, r, d)
    assert np.isclose(L, precond.loss(p, kin, tb, r, d), rtol=1e-13)
    h = 1e-6
    for (li, which, idx) in ((0, 0, (3, 1)), (1, 0, (7, 9)), (2, 1, (5,)), (3, 0, (0, 11)), (3, 1, (0,)), (0, 1, (2,))):
        arr = p[li][which]
        old = arr[idx]
        arr[idx] = old + h
        lp = precond.loss(p, kin, tb, r, d)
        arr[idx] = old - h
        lm = precond.loss(p, kin, tb, r, d)
        arr[idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[li][which][idx]) < 1e-7 * max(1.0, abs(fd)), (li, which, idx, fd, g[li][which][idx])


def test_training_pairs_are_residuals_of_the_ideal_correction():
    """r = (H - eps) d exactly, with d orthogonal to the converged block."""
    sy = ofde.System(workloads.molecule_on_slab_small())
    st = scf.initial_state(sy)
    pot = sy.build_veff(st.rhos)
    w, v = scf.eig_dense(sy, 1, 0, pot["veff"][1], 4)
    r, d = precond.training_pairs(sy, 1, 0, pot["veff"][1], v, w, 3, seed=9)
    assert np.abs(d @ v.conj().T).max() < 1e-12
    H = sy.dense_h(1, 0, pot["veff"][1])
    want = (H @ d.T).T - w[:3, None] * d
    assert np.abs(r - want).max() < 1e-11


def test_loss_is_the_squared_sine_of_the_angle_and_scale_free():
    """L_j = 1 - |<m r_j, d_j>|^2 / (|m r_j|^2 |d_j|^2): zero when m r_j is parallel to d_j
    (whatever the complex factor), unchanged when r_j is multiplied by a complex scalar."""
    rng = np.random.default_rng(4)
    kin = rng.uniform(0, 10, 30)
    r = rng.standard_normal((3, 30)) + 1j * rng.standard_normal((3, 30))
    d = rng.standard_normal((3, 30)) + 1j * rng.standard_normal((3, 30))
    tb = np.array([0.9, 1.7, 3.2])
    p = precond.init_params(6)
    p[-1][0] = 0.2 * rng.standard_normal(p[-1][0].shape)
    m = precond.multiplier(p, kin, tb, r)
    u = m * r
    cos2 = np.abs(np.sum(np.conj(u) * d, axis=1)) ** 2 / (np.sum(np.abs(u) ** 2, axis=1) * np.sum(np.abs(d) ** 2, axis=1))
    assert np.isclose(precond.loss(p, kin, tb, r, d), float(np.sum(1.0 - cos2)), rtol=1e-12)
    # d parallel to m r (complex factor 2 - 3i): zero loss
    assert precond.loss(p, kin, tb, r, (2 - 3j) * u) < 1e-24
    # the multiplier depends on |r| / rms|r| only, so a complex rescaling of a band's residual
    # leaves m and hence the loss unchanged
    s = np.array([[0.5 + 2j], [-3.0], [1j]])
    assert np.isclose(precond.loss(p, kin, tb, s * r, d), precond.loss(p, kin, tb, r, d), rtol=1e-12)
