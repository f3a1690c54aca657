"""Pins of the Methfessel-Paxton and Gaussian smearing of the oracle (CPU only)."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import erfc

from oracle import scf, smearing


@pytest.mark.parametrize("order", [0, 1, 2])
def test_delta_integrates_polynomials_up_to_degree_2n_plus_1(order):
    """The defining property of the order-N approximant: int delta_N(t) t^k dt = [k == 0] for
    every k <= 2N + 1, and not for k = 2N + 2 (so the order is exactly N)."""
    for k in range(2 * order + 3):
        v, _ = integrate.quad(lambda t: smearing.mp_delta(t, order) * t ** k, -30, 30, epsabs=1e-14, limit=400)
        if k <= 2 * order + 1:
            assert abs(v - (1.0 if k == 0 else 0.0)) < 1e-11, (order, k, v)
        else:
            assert abs(v) > 1e-3, (order, k, v)


@pytest.mark.parametrize("order", [0, 1, 2])
def test_occupation_is_one_minus_the_integrated_delta(order):
    x = np.linspace(-4, 4, 17)
    h = 1e-5
    fd = (smearing.mp_occupation(x + h, order) - smearing.mp_occupation(x - h, order)) / (2 * h)
    assert np.allclose(fd, -smearing.mp_delta(x, order), atol=1e-9)
    assert smearing.mp_occupation(np.array([-30.0]), order)[0] == pytest.approx(1.0, abs=1e-14)
    assert abs(smearing.mp_occupation(np.array([30.0]), order)[0]) < 1e-14
    assert smearing.mp_occupation(np.array([0.0]), order)[0] == pytest.approx(0.5, abs=1e-15)


def test_gaussian_order_is_erfc_and_its_entropy_closed_form():
    x = np.linspace(-3, 3, 13)
    assert np.allclose(smearing.mp_occupation(x, 0), 0.5 * erfc(x), atol=1e-16)
    assert np.allclose(smearing.mp_entropy_term(x, 0), np.exp(-x * x) / (2 * math.sqrt(math.pi)), atol=1e-13)


@pytest.mark.parametrize("order", [0, 1, 2])
def test_entropy_term_makes_the_free_energy_variational(order):
    """s'(x) = x f'(x): the condition under which E - sigma S is stationary in the occupations
    at fixed electron count (the Fermi-Dirac entropy satisfies the same relation)."""
    x = np.linspace(-3.5, 3.5, 15)
    h = 1e-4
    ds = (smearing.mp_entropy_term(x + h, order) - smearing.mp_entropy_term(x - h, order)) / (2 * h)
    df = (smearing.mp_occupation(x + h, order) - smearing.mp_occupation(x - h, order)) / (2 * h)
    assert np.allclose(ds, x * df, atol=1e-7)


def test_first_order_occupations_count_and_narrow_limit():
    rng = np.random.default_rng(4)
    eigs = [np.sort(rng.uniform(-1, 1, 12)) for _ in range(3)]
    wk = np.array([0.25, 0.25, 0.5])
    occ, mu, S = scf.occupations(eigs, wk, 13.0, 0.01, "mp")
    n = sum(2 * w * o.sum() for w, o in zip(wk, occ))
    assert abs(n - 13.0) < 1e-12
    # first order: occupations overshoot [0, 1] slightly near mu (a known feature)
    allo = np.concatenate(occ)
    assert allo.min() > -0.1 and allo.max() < 1.1
    # a gapped spectrum with a tiny width fills the lowest levels exactly
    e = [np.array([-0.5, -0.4, -0.3, 0.3, 0.4])]
    occ, mu, S = scf.occupations(e, np.ones(1), 6.0, 1e-4, "mp")
    assert np.allclose(occ[0], [1, 1, 1, 0, 0], atol=1e-12) and abs(S) < 1e-12
