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


KC = 8.9875517923e9


def grad_abs_scales(pts, g, src=None, tri=None, sigma=None, self_exclude=False):
    """Sums of the magnitudes of the terms that make up each gradient of the
    field's backward evaluation (cells taken as points at their centroids with
    charge sigma * area): the scale to which binary32 arithmetic fixes a sum of
    terms whose signs come from an arbitrary upstream gradient g.
    Returns (A_sigma [np], A_pts [nt], A_src_pos [ns], A_src_q [ns])."""
    pts = np.asarray(pts, np.float64)[:, :3]
    g = np.asarray(g, np.float64)
    gE = np.linalg.norm(g[:, :3], axis=1)
    gV = np.abs(g[:, 3])
    A_pts = np.zeros(len(pts))
    A_sigma = A_sq = A_sp = None
    if src is not None:
        src = np.asarray(src, np.float64)
        d = np.linalg.norm(pts[:, None, :] - src[None, :, :3], axis=-1)        # nt x ns
        with np.errstate(divide="ignore"):
            inv = np.where(d > 0, 1.0 / d, 0.0)
        if self_exclude:
            np.fill_diagonal(inv, 0.0)
        aq = np.abs(src[:, 3])
        A_pts += KC * ((3 * gE[:, None] * inv ** 3 + gV[:, None] * inv ** 2) * aq[None, :]).sum(1)
        A_sp = KC * aq * (3 * gE[:, None] * inv ** 3 + gV[:, None] * inv ** 2).sum(0)
        A_sq = KC * (gE[:, None] * inv ** 2 + gV[:, None] * inv).sum(0)
    if tri is not None:
        tri = np.asarray(tri, np.float64)
        c = tri.mean(axis=1)
        area = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1)
        inv = 1.0 / np.linalg.norm(pts[:, None, :] - c[None], axis=-1)            # nt x np
        A_sigma = KC * area * (gE[:, None] * inv ** 2 + gV[:, None] * inv).sum(0)
        if sigma is not None:
            w = np.abs(np.asarray(sigma, np.float64)) * area
            A_pts += KC * ((3 * gE[:, None] * inv ** 3 + gV[:, None] * inv ** 2) * w[None, :]).sum(1)
    return A_sigma, A_pts, A_sp, A_sq


def grad_err(got, ref, abs_scale):
    """Gradient error per element (row norm for vectors) relative to
    max(|ref|, 1e-2 rms|ref|, 0.1 * abs_scale): like potential_err, a sum of
    signed terms evaluated in binary32 is fixed only to a few ulps of the sum
    of the terms' magnitudes, so that scale is part of the guard."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if got.ndim == 1:
        got, ref = got[:, None], ref[:, None]
    if len(ref) == 0:
        return 0.0
    mag = np.linalg.norm(ref, axis=1)
    rms = np.sqrt((mag ** 2).mean())
    den = np.maximum(np.maximum(mag, 1e-2 * rms), 0.1 * np.asarray(abs_scale, np.float64))
    den = np.where(den > 0, den, 1.0)
    return float((np.linalg.norm(got - ref, axis=1) / den).max())
