"""Learned per-G preconditioner of the subsystem eigensolver: plain NumPy statement.

Test infrastructure only (see ``oracle/__init__.py``).  The paper solves Eq. KS with the
plane-wave machinery of its host code and says nothing about preconditioning; the learned
preconditioner is a deployment pattern layered on the method, so there is no passage to
follow beyond Eq. KS itself.  What it computes is fixed here:

* For band j with residual r_j = (H - eps_j) x_j, the kinetic (Teter-Payne-Allan)
  preconditioner is W_jG = K(y) r_jG with y = (|k+G|^2/2) / T_j, T_j the band's kinetic
  energy, K(y) = (27 + 18y + 12y^2 + 8y^3) / (27 + 18y + 12y^2 + 8y^3 + 16y^4).
* The learned preconditioner multiplies K by exp(o_jG), o = MLP(f_jG), a per-G network of
  three tanh layers of width 64 and a linear output, on the features
  f = (log(1 + y), log T_j, |r_jG| / rms_G |r_j|).  A zero output layer reproduces the
  kinetic preconditioner exactly.
* Training pairs come from converged eigensolves: for converged (psi_j, eps_j), a seeded
  smooth perturbation d_j orthogonal to the converged block gives r_j = (H - eps_j) d_j, and
  the ideal correction of r_j is d_j.  The block eigensolver's Rayleigh-Ritz step picks the
  complex coefficient of every preconditioned residual itself, so only its direction
  matters: L = sum_j min_a |a m_j r_j - d_j|^2 / |d_j|^2, minimised by
  a_j = <m_j r_j, d_j> / |m_j r_j|^2 (L_j = 1 - cos^2 of the angle between m_j r_j and d_j).
  By the envelope theorem dL/dm = 2 Re(conj(e) a r) / |d_j|^2 with e = a m r - d at that a.
* Inference and training use weights rounded to bfloat16 (round to nearest even) with
  FP32 accumulation; the oracle evaluates the same rounded weights in FP64.

``forward`` / ``backward`` below are the plain chain rule, pinned by central finite
differences in the tests.
"""
from __future__ import annotations

import numpy as np

WIDTH = 64
NFEAT = 3
LAYERS = ((NFEAT, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, 1))


def bf16_round(a):
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed=0):
    """Seeded initial weights (scaled normal) with a zero output layer."""
    rng = np.random.default_rng([seed, 4099])
    params = []
    for i, (fi, fo) in enumerate(LAYERS):
        if i == len(LAYERS) - 1:
            W = np.zeros((fo, fi))
        else:
            W = rng.standard_normal((fo, fi)) / np.sqrt(fi)
        params.append([W, np.zeros(fo)])
    return params


def tpa(y):
    p = 27.0 + y * (18.0 + y * (12.0 + y * 8.0))
    return p / (p + 16.0 * y ** 4)


def features(kin, tband, r):
    """Features [nb, npw, 3] of residual rows r [nb, npw] (complex)."""
    y = kin[None, :] / np.maximum(tband, 1e-12)[:, None]
    amp = np.abs(r)
    rms = np.sqrt(np.mean(amp ** 2, axis=1, keepdims=True))
    f = np.empty(r.shape + (3,))
    f[..., 0] = np.log1p(y)
    f[..., 1] = np.log(np.maximum(tband, 1e-12))[:, None]
    f[..., 2] = amp / np.maximum(rms, 1e-300)
    return f, y


def forward(params, f):
    """MLP output o [...] and the activations needed by backward."""
    x = f.reshape(-1, f.shape[-1])
    acts = [x]
    h = x
    for i, (W, b) in enumerate(params):
        z = h @ W.T + b
        h = np.tanh(z) if i < len(params) - 1 else z
        acts.append(h)
    return h.reshape(f.shape[:-1]), acts


def multiplier(params, kin, tband, r):
    f, y = features(kin, tband, r)
    o, _ = forward(params, f)
    return tpa(y) * np.exp(o)


def apply(params, kin, tband, r):
    return multiplier(params, kin, tband, r) * r


def best_scale(m, r, d):
    """a_j = <m r_j, d_j> / |m r_j|^2 per band (0 where m r_j vanishes)."""
    u = m * r
    num = np.sum(np.conj(u) * d, axis=1)
    den = np.sum(np.abs(u) ** 2, axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)


def loss(params, kin, tband, r, d):
    m = multiplier(params, kin, tband, r)
    a = best_scale(m, r, d)[:, None]
    e = a * m * r - d
    return float(np.sum(np.sum(np.abs(e) ** 2, axis=1) / np.sum(np.abs(d) ** 2, axis=1)))


def backward(params, kin, tband, r, d):
    """Loss and its gradient with respect to every weight and bias (chain rule)."""
    f, y = features(kin, tband, r)
    o, acts = forward(params, f)
    K = tpa(y)
    m = K * np.exp(o)
    ar = best_scale(m, r, d)[:, None] * r
    e = m * ar - d
    nd = np.sum(np.abs(d) ** 2, axis=1, keepdims=True)
    L = float(np.sum(np.sum(np.abs(e) ** 2, axis=1, keepdims=True) / nd))
    # dL/dm = 2 Re(conj(e) a r) / |d_j|^2 at the optimal a (envelope theorem); dm/do = m
    g = (2.0 * np.real(np.conj(e) * ar) / nd * m).reshape(-1, 1)
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        W, b = params[i]
        h_in = acts[i]
        grads[i] = [g.T @ h_in, g.sum(axis=0)]
        if i > 0:
            g = (g @ W) * (1.0 - acts[i] ** 2)
    return L, grads


def training_pairs(system, I, k, veff_I, psi, eps, ntrain, seed):
    """Seeded smooth perturbations d (orthogonal to the converged block psi) and their
    residuals r = (H - eps_j) d for the first ntrain bands."""
    mil, kin = system.basis[I][k]
    rng = np.random.default_rng([seed, I, k, 131])
    npw = kin.size
    d = (rng.standard_normal((ntrain, npw)) + 1j * rng.standard_normal((ntrain, npw))) / (1.0 + kin)[None, :]
    d = d - (d @ psi.conj().T) @ psi
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    hd = system.apply_h(I, k, d, veff_I)
    r = hd - eps[:ntrain, None] * d
    return r, d
