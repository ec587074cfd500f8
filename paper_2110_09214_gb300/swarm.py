"""Swarm parameters of a chamber from its per-step statistics (Sec. 4.1).

The cloud moments come from the device reductions of every step (obem_step /
obem_batch_step stats: electron count, sums of z and z^2); the parameters are
least-squares slopes over the steps:
  drift velocity      V_d = d<z>/dt                        (Eq. (vd))
  longitudinal diff.  D_L = (1/2) d var(z)/dt              (Eq. (diffusion))
  Townsend coeff.     alpha = (d ln N_e/dt) / V_d          (Eq. (townsend), G = exp(alpha d))
"""
from __future__ import annotations

import numpy as np


def slope(t, y):
    """Least-squares slope of y(t)."""
    t = np.asarray(t, np.float64)
    y = np.asarray(y, np.float64)
    tm, ym = t.mean(), y.mean()
    den = ((t - tm) ** 2).sum()
    return float(((t - tm) * (y - ym)).sum() / den) if den > 0 else 0.0


def electron_moments(hist):
    """Per step: electron count, mean z, variance of z."""
    n = np.array([h["n_electron"] for h in hist], np.float64)
    sz = np.array([h["sum_e"][2] for h in hist], np.float64)
    sz2 = np.array([h["sum2_e"][2] for h in hist], np.float64)
    nn = np.maximum(n, 1.0)
    mean = sz / nn
    return n, mean, sz2 / nn - mean ** 2


def swarm_params(hist, dt):
    """(V_d, D_L, alpha) from the stats of consecutive steps taken dt apart
    (moments after each step); alpha is 0 when V_d is 0."""
    t = dt * (1.0 + np.arange(len(hist)))
    n, mean, var = electron_moments(hist)
    vd = slope(t, mean)
    dl = 0.5 * slope(t, var)
    ok = n > 0
    alpha = slope(t[ok], np.log(n[ok])) / vd if vd != 0.0 and ok.sum() > 1 else 0.0
    return vd, dl, alpha
