"""Smeared occupations: Methfessel-Paxton of any order, and Gaussian.

Test infrastructure only (see ``oracle/__init__.py``).

Computational Details: the metallic subsystems use Methfessel-Paxton smearing.  The method
replaces the step function of the occupations by 1 - int_{-inf}^x delta_N(t) dt, with
x = (e - mu) / sigma and delta_N the Gaussian times its Hermite expansion up to order N:

    delta_N(t) = sum_{n=0}^{N} A_n H_{2n}(t) exp(-t^2),   A_n = (-1)^n / (n! 4^n sqrt(pi)),

(H the physicists' Hermite polynomials), chosen so that delta_N integrates every polynomial
of degree <= 2N + 1 exactly.  Since d/dt [H_{m-1}(t) e^{-t^2}] = -H_m(t) e^{-t^2}, the
occupation is

    f_N(x) = erfc(x) / 2 + sum_{n=1}^{N} A_n H_{2n-1}(x) exp(-x^2).

The free energy E - sigma S is variational in the occupations when each state contributes
s(x) = -int_{-inf}^x t delta_N(t) dt to S / (2 sum_k w_k) (the same condition s' = x f' that
the Mermin entropy satisfies for Fermi-Dirac occupations); it is evaluated here by
quadrature of that definition.  N = 0 is plain Gaussian smearing.  The paper quotes the
width only (1e-2 Ry); the order is the reading N = 1 (the usual first-order form).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate
from scipy.special import erfc, eval_hermite


def mp_coefficient(n):
    return (-1.0) ** n / (math.factorial(n) * 4.0 ** n * math.sqrt(math.pi))


def mp_delta(t, order):
    t = np.asarray(t, dtype=np.float64)
    return sum(mp_coefficient(n) * eval_hermite(2 * n, t) for n in range(order + 1)) * np.exp(-t * t)


def mp_occupation(x, order):
    x = np.asarray(x, dtype=np.float64)
    f = 0.5 * erfc(x)
    for n in range(1, order + 1):
        f = f + mp_coefficient(n) * eval_hermite(2 * n - 1, x) * np.exp(-x * x)
    return f


def mp_entropy_term(x, order):
    """s(x) = -int_{-inf}^x t delta_N(t) dt by adaptive quadrature (one state)."""
    def one(xx):
        if xx < -40.0:
            return 0.0
        v, _ = integrate.quad(lambda t: t * mp_delta(t, order), -40.0, xx, epsabs=1e-14, epsrel=1e-12, limit=200)
        return -v
    return np.vectorize(one)(np.asarray(x, dtype=np.float64))


def occupations(eigs, wk, nelec, sigma, order=1):
    """Occupations per k, chemical potential (bisection to 1e-13 electrons) and
    S = 2 sum_k w_k sum_j s(x_jk)."""
    eigs = [np.asarray(e, dtype=np.float64) for e in eigs]
    wk = np.asarray(wk, dtype=np.float64)

    def count(mu):
        return sum(2.0 * w * float(np.sum(mp_occupation((e - mu) / sigma, order))) for w, e in zip(wk, eigs))

    lo = min(e.min() for e in eigs) - 40.0 * sigma
    hi = max(e.max() for e in eigs) + 40.0 * sigma
    for _ in range(300):
        mu = 0.5 * (lo + hi)
        n = count(mu)
        if abs(n - nelec) < 1e-13:
            break
        if n < nelec:
            lo = mu
        else:
            hi = mu
    occ = [mp_occupation((e - mu) / sigma, order) for e in eigs]
    S = sum(2.0 * w * float(np.sum(mp_entropy_term((e - mu) / sigma, order))) for w, e in zip(wk, eigs))
    return occ, mu, S
