"""FP64 oracle of the MCMC densification step the paper trains with (Sec. 3.3,
"stochastic density control via MCMC-based densification", and Algorithm 1's
"Relocate / add Gaussians"), whose rules the paper takes from 3DGS-as-MCMC
(Kheradmand et al. 2024) without restating them.  TEST INFRASTRUCTURE ONLY,
like the rest of this package.  Random numbers are inputs.

Readings (the cited method's published rules):
  * a Gaussian is dead when its opacity sigmoid(logit) <= 0.005;
  * relocation: each dead Gaussian takes the parameters of a live one drawn
    with probability proportional to opacity (draw j for uniform u: the
    first j whose cumulative opacity exceeds u times the total); a source
    drawn c times ends up as N = c + 1 identical Gaussians whose opacity
    and scale are reset so that, stacked and composited front to back, they
    render like the source did:
        o_N = 1 - (1 - o)^(1/N)                   (the same alpha at the centre)
        s_N = s * o / sum_{i=1..N} sum_{k=0..i-1} C(i-1, k) (-1)^k o_N^(k+1) / sqrt(k+1)
    (the same integral of the composited alpha along a line through the
    centre; scales per axis, so the covariance scales by the square);
    The reset opacity is then bounded to [0.005, 1 - 2^-23] (the cited
    method's bounds: a copy is never born dead, and its logit stays finite),
    the scale being computed from the unbounded o_N;
  * growth ("add Gaussians", up to the cap): n_add = min(cap, floor(1.05 n))
    - n new Gaussians, each drawn like a relocation source (probability
    proportional to opacity, live ones only) by its own uniform; the drawn
    sources are reset by the same rule (N = times drawn + 1) and the new
    Gaussians, appended after the n existing ones in the order of the
    uniforms, copy their source's reset parameters;
  * the Adam moments of every Gaussian written by relocation or growth (the
    copies and their sources) restart from zero;
  * noise on the means: mu += noise_lr * sigmoid(-100 (o - 0.005)) * Sigma eta
    with Sigma = R diag(s)^2 R^T the Gaussian's covariance and eta ~ N(0, I)
    given.
"""
from __future__ import annotations

from math import comb

import numpy as np

DEAD_OPACITY = 0.005
MAX_OPACITY = 1.0 - 2.0 ** -23     # 1 - float32 epsilon
GROWTH_RATE = 0.05
NOISE_K = 100.0


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def relocated_opacity_scale(o, s, N, bounded=True):
    """Opacity and per-axis scales of each of N identical Gaussians that
    replace one of opacity o and scales s (N = 1 leaves them unchanged);
    bounded: the opacity clipped to [0.005, 1 - 2^-23] after the scale is
    formed."""
    o = float(o)
    oN = 1.0 - (1.0 - o) ** (1.0 / N)
    den = 0.0
    for i in range(1, N + 1):
        for k in range(i):
            den += comb(i - 1, k) * (-1.0) ** k * oN ** (k + 1) / np.sqrt(k + 1.0)
    sN = np.asarray(s, np.float64) * o / den
    if bounded:
        oN = min(max(oN, DEAD_OPACITY), MAX_OPACITY)
    return oN, sN


def draw_sources(opacity, dead, u):
    """For each uniform u in [0, 1): the live Gaussian drawn with probability
    proportional to opacity (dead ones have weight 0)."""
    w = np.where(dead, 0.0, np.asarray(opacity, np.float64))
    c = np.cumsum(w)
    return np.searchsorted(c, np.asarray(u, np.float64) * c[-1], side="right")


def relocate(params, u):
    """params: dict of mean [N,3], log_scale [N,3], quat [N,4],
    opacity_logit [N], sh [N,K,3] (float64, not modified); u: one uniform per
    dead Gaussian, in index order.  Returns the relocated parameters and the
    source index of each dead Gaussian."""
    p = {k: np.array(v, np.float64, copy=True) for k, v in params.items()}
    o = sigmoid(p["opacity_logit"])
    dead = o <= DEAD_OPACITY
    dead_idx = np.nonzero(dead)[0]
    if len(dead_idx) == 0 or dead.all():
        return p, np.zeros(0, np.int64)
    src = draw_sources(o, dead, np.asarray(u)[:len(dead_idx)])
    _reset_sources(p, np.bincount(src, minlength=len(o)))
    for d, j in zip(dead_idx, src):
        for k in p:
            p[k][d] = p[k][j]
    return p, src


def n_grow(n, cap, rate=GROWTH_RATE):
    """Gaussians the growth step adds to n: min(cap, floor((1 + rate) n)) - n
    (never negative)."""
    return max(0, min(int(cap), int(np.floor((1.0 + rate) * n))) - int(n))


def _reset_sources(p, counts):
    o = sigmoid(p["opacity_logit"])
    for j in np.nonzero(counts)[0]:
        oN, sN = relocated_opacity_scale(o[j], np.exp(p["log_scale"][j]), int(counts[j]) + 1)
        p["opacity_logit"][j] = np.log(oN / (1.0 - oN))
        p["log_scale"][j] = np.log(sN)


def grow(params, u):
    """The growth step with one uniform per new Gaussian (len(u) of them):
    returns the n + len(u) Gaussians and each new one's source."""
    p = {k: np.array(v, np.float64, copy=True) for k, v in params.items()}
    o = sigmoid(p["opacity_logit"])
    dead = o <= DEAD_OPACITY
    u = np.asarray(u, np.float64)
    if len(u) == 0 or dead.all():
        return p, np.zeros(0, np.int64)
    src = draw_sources(o, dead, u)
    _reset_sources(p, np.bincount(src, minlength=len(o)))
    for k in p:
        p[k] = np.concatenate([p[k], p[k][src]], axis=0)
    return p, src


def covariance(log_scale, quat):
    q = np.asarray(quat, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1).reshape(q.shape[:-1] + (3, 3))
    s = np.exp(np.asarray(log_scale, np.float64))
    M = R * s[..., None, :]
    return M @ np.swapaxes(M, -1, -2)


def noise_means(mean, log_scale, quat, opacity_logit, eta, noise_lr):
    """mu + noise_lr * sigmoid(-100 (o - 0.005)) * Sigma eta."""
    o = sigmoid(opacity_logit)
    gate = sigmoid(-NOISE_K * (o - DEAD_OPACITY))
    S = covariance(log_scale, quat)
    return np.asarray(mean, np.float64) + noise_lr * gate[:, None] * np.einsum("nab,nb->na", S, eta)
