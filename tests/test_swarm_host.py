"""Host logic of the package (no GPU): the swarm-parameter fits of swarm.py
(Eqs. (vd), (diffusion), (townsend) of Sec. 4.1) on per-step moments built
from closed forms, and the parsing of a batch's per-chamber statistics
blocks."""
import ctypes as C

import numpy as np
import torch

from paper_2110_09214_gb300 import obem, swarm


def _hist(n0, vd, dl, alpha, z0, dt, steps):
    """Per-step stats of a cloud whose electron count grows as
    n0 exp(alpha vd t), whose mean z drifts at vd and whose var(z) grows as
    2 dl t (t = dt, 2 dt, ...)."""
    out = []
    for k in range(steps):
        t = dt * (k + 1)
        n = n0 * np.exp(alpha * vd * t)
        m = z0 + vd * t
        v = 2.0 * dl * t
        out.append({"n_electron": n, "sum_e": [0.0, 0.0, n * m], "sum2_e": [0.0, 0.0, n * (v + m * m)]})
    return out


def test_swarm_params_recover_closed_forms():
    dt = 1e-12
    vd, dl, alpha = 2.5e4, 0.07, 3.0e4
    h = _hist(1e4, vd, dl, alpha, 3e-4, dt, 40)
    gv, gd, ga = swarm.swarm_params(h, dt)
    assert abs(gv / vd - 1) < 1e-9
    assert abs(gd / dl - 1) < 1e-6
    assert abs(ga / alpha - 1) < 1e-9


def test_swarm_params_without_drift_or_electrons():
    dt = 1e-12
    h = _hist(100.0, 0.0, 0.05, 0.0, 1e-3, dt, 10)
    gv, gd, ga = swarm.swarm_params(h, dt)
    assert abs(gv) < 1e-9 and ga == 0.0 and abs(gd / 0.05 - 1) < 1e-6
    # steps without electrons are left out of the growth fit and the moments
    # of an empty cloud are defined (count clamped to 1)
    h = _hist(100.0, 1e4, 0.05, 1e4, 1e-3, dt, 10)
    for s in h[6:]:
        s["n_electron"] = 0.0
        s["sum_e"][2] = s["sum2_e"][2] = 0.0
    n, mean, var = swarm.electron_moments(h)
    assert np.all(np.isfinite(mean)) and np.all(np.isfinite(var))
    _, _, ga = swarm.swarm_params(h, dt)
    assert np.isfinite(ga)


def test_read_batch_stats_splits_per_chamber_blocks():
    nb = 3
    raw = bytearray(nb * obem.STATS_BYTES)
    for c in range(nb):
        s = obem.obem_step_stats()
        s.status = -6 if c == 1 else 0
        s.n_before, s.n_after, s.n_electron = 10 * c + 1, 10 * c + 2, 10 * c + 3
        s.sum_e[2] = 0.5 * c
        s.sum2_e[2] = 0.25 * c
        raw[c * obem.STATS_BYTES:(c + 1) * obem.STATS_BYTES] = bytes(s)
    buf = torch.frombuffer(raw, dtype=torch.uint8).clone()
    got = obem.read_batch_stats(buf, nb)
    assert len(got) == nb
    for c, d in enumerate(got):
        assert d["status"] == (-6 if c == 1 else 0)
        assert (d["n_before"], d["n_after"], d["n_electron"]) == (10 * c + 1, 10 * c + 2, 10 * c + 3)
        assert d["sum_e"][2] == 0.5 * c and d["sum2_e"][2] == 0.25 * c
    assert C.sizeof(obem.obem_step_stats) == obem.STATS_BYTES
