"""Helpers shared by the GPU parity tests."""
import numpy as np


def guarded_rel_err(got, ref):
    """Max over points of |got - ref| / max(|ref|, 1e-2 rms|ref|): the field
    tolerance metric (the plain relative error is undefined where the field
    cancels)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if got.ndim == 1:
        got, ref = got[:, None], ref[:, None]
    mag = np.linalg.norm(ref, axis=1)
    rms = np.sqrt((mag ** 2).mean()) if len(mag) else 0.0
    den = np.maximum(mag, 1e-2 * rms)
    den = np.where(den > 0, den, 1.0)
    return float((np.linalg.norm(got - ref, axis=1) / den).max()) if len(mag) else 0.0


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def pts4(p):
    p = np.asarray(p, np.float32)
    out = np.zeros((len(p), 4), np.float32)
    out[:, :3] = p[:, :3]
    if p.shape[1] == 4:
        out[:, 3] = p[:, 3]
    return out


FIELD_TOL = 1e-5


def potential_err(got, ref, ref_abs):
    """Potential error relative to max(|V|, 0.1 V_abs), V_abs = sum of |terms|:
    binary32 partial sums of cancelling +- contributions fix V only to a few
    ulps of V_abs, so V is gated on that scale (E uses guarded_rel_err)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), 0.1 * np.abs(np.asarray(ref_abs, np.float64)))
    den = np.where(den > 0, den, 1.0)
    return float((np.abs(got - ref) / den).max()) if len(ref) else 0.0
