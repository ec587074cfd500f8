"""Host side of the far-cell groups (OBEM_STEP_CELL_GROUPS), run on the CPU
through a small native harness (tests/native/cellgroup_host.cu) that calls
the library's own group builder: group order, radii, smallest h^2, the fit
matrix (against numpy's pseudo-inverse), and the accuracy of the fitted
equivalent charges against the oracle's closed-form cell field."""
import os
import shutil
import struct
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2110_09214_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
K, M, NC = 32, 49, 147
KC = 8.9875517923e9
T1, T2 = -0.410426192315345, 0.696140478029631
W7 = [0.225] + [0.132394152788506] * 3 + [0.125939180544827] * 3


def _nvcc():
    p = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return p if os.path.exists(p) else shutil.which("nvcc")


@pytest.fixture(scope="module")
def groups():
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    mesh = inputs.gem_mesh_target(8000, inputs.GemGeometry(rings=1), tol=0.05)
    tri = mesh.tri.astype(np.float64)
    e = np.stack([tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 1], tri[:, 0] - tri[:, 2]], 1)
    h2 = (e ** 2).sum(2).max(1).astype(np.float32)
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "harness")
        r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", exe,
                            os.path.join(HERE, "native", "cellgroup_host.cu")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        fin, fout = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
        with open(fin, "wb") as f:
            f.write(struct.pack("i", mesh.n))
            f.write(tri.tobytes())
            f.write(h2.tobytes())
        r = subprocess.run([exe, fin, fout], capture_output=True, text=True)
        assert r.returncode == 0, (r.returncode, r.stderr)
        b = open(fout, "rb").read()
    o = [0]

    def take(dt, n):
        a = np.frombuffer(b, dt, n, o[0])
        o[0] += a.nbytes
        return a

    ng = int(take(np.int32, 1)[0])
    out = dict(ng=ng, perm=take(np.int32, mesh.n), cr=take(np.float32, 4 * ng).reshape(ng, 4),
               h2min=take(np.float32, ng), u=take(np.float32, 4 * M).reshape(M, 4)[:, :3].astype(np.float64),
               c64=take(np.float64, 4 * ng).reshape(ng, 4), v=take(np.float64, 3 * NC).reshape(NC, 3),
               P=take(np.float64, M * NC).reshape(M, NC))
    assert o[0] == len(b)
    return mesh, tri, h2, out


def test_groups_cover_every_cell_once_with_their_radius(groups):
    mesh, tri, h2, g = groups
    assert g["ng"] == (mesh.n + K - 1) // K
    assert np.array_equal(np.sort(g["perm"]), np.arange(mesh.n))
    for k in range(g["ng"]):
        idx = g["perm"][k * K:(k + 1) * K]
        c = g["cr"][k, :3].astype(np.float64)
        assert np.linalg.norm(tri[idx].reshape(-1, 3) - c, axis=1).max() <= g["cr"][k, 3]
        assert g["h2min"][k] == h2[idx].min()
        assert np.array_equal(g["c64"][k], g["cr"][k].astype(np.float64))
    # Morton-ordered groups are compact: the median radius is a few cell sizes
    assert np.median(g["cr"][:, 3]) < 6 * np.sqrt(np.median(h2))


def test_directions_and_fit_matrix(groups):
    _, _, _, g = groups
    assert np.allclose(np.linalg.norm(g["u"], axis=1), 1.0, atol=1e-7)
    assert np.allclose(np.linalg.norm(g["v"], axis=1), 1.0, atol=1e-15)
    A = 1.0 / np.linalg.norm(2.5 * g["v"][:, None, :] - g["u"][None, :, :], axis=2)
    P = np.linalg.pinv(A)
    assert np.abs(g["P"] - P).max() <= 1e-8 * np.abs(P).max()


def test_fitted_charges_reproduce_the_group_field(groups):
    """The device fit (7-point sources, potentials at the check points,
    charges = R P b) done here in FP64 with the builder's arrays: the field
    of the 49 charges at 9 radii from the centre against the closed form of
    the group's cells, relative to sum |q| / d^2."""
    mesh, tri, _, g = groups
    rng = np.random.default_rng(2)
    area = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1)
    sig = rng.normal(0.0, 1e-6, mesh.n)
    i = np.arange(100) + 0.5
    ph, th = np.arccos(1 - 2 * i / 100), np.pi * (1 + 5 ** 0.5) * i
    dirs = np.column_stack([np.cos(th) * np.sin(ph), np.sin(th) * np.sin(ph), np.cos(ph)])
    worst = 0.0
    for k in rng.choice(g["ng"], 25, replace=False):
        idx = g["perm"][k * K:(k + 1) * K]
        c, R = g["c64"][k, :3], g["c64"][k, 3]
        pts, q = [], []
        for j in idx:
            v = tri[j]
            m = v.mean(0)
            pts += [m] + [m + T1 * (v[a] - m) for a in range(3)] + [m + T2 * (v[a] - m) for a in range(3)]
            q += [KC * area[j] * sig[j] * w for w in W7]
        pts, q = np.array(pts) - c, np.array(q)
        b = (q[None, :] / np.linalg.norm(2.5 * R * g["v"][:, None, :] - pts[None, :, :], axis=2)).sum(1)
        x = (R * (g["P"] @ b)).astype(np.float32).astype(np.float64)
        D = c + 9.0 * R * dirs
        Eref, _ = oracle.panel_field(tri[idx], sig[idx], D)
        d = D[:, None, :] - (c + R * g["u"])[None, :, :]
        r = np.linalg.norm(d, axis=2)
        Eq = (x[None, :, None] * d / r[..., None] ** 3).sum(1)
        qabs = np.abs(KC * area[idx] * sig[idx]).sum()
        worst = max(worst, np.linalg.norm(Eq - Eref, axis=1).max() / (qabs / (9.0 * R) ** 2))
    assert worst <= 2e-6
