"""The C-ABI library builds for sm_103a, loads, and exports exactly what
include/obem.h declares; host-side argument checks (no GPU compute)."""
import os
import re
import subprocess

import numpy as np

from paper_2110_09214_gb300 import build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "obem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:int|void|const char \*)\s*\**(obem_\w+)\s*\(", src, flags=re.M))


def test_library_builds_and_exports_every_declared_symbol():
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (obem_\w+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    assert declared <= exported, "missing: %s" % sorted(declared - exported)
    assert exported <= declared, "undeclared exports: %s" % sorted(exported - declared)


def test_binding_loads_and_struct_sizes_match_header():
    from paper_2110_09214_gb300 import obem
    lib = obem.load()
    assert lib.obem_last_error(None).decode() == "null context"
    # obem_step_stats: 12 int32, 1 int64, 13 doubles
    assert obem.STATS_BYTES == 12 * 4 + 8 + 13 * 8
    assert __import__("ctypes").sizeof(obem.obem_config) == 4 * 4 + 8 * 9


def test_create_rejects_bad_config_without_touching_the_gpu():
    from paper_2110_09214_gb300 import obem
    import pytest
    for bad in (dict(capacity=0, dt=1e-12), dict(capacity=10, dt=-1.0),
                dict(capacity=10, dt=1e-12, trial_cap=0), dict(capacity=10, dt=1e-12, trial_cap=1000),
                dict(capacity=10, dt=1e-12, z_lo=1.0, z_hi=0.0)):
        with pytest.raises(obem.ObemError) as e:
            obem.obem_create(**bad)
        assert e.value.code == obem.OBEM_ERR_ARG


def test_inputs_gem_mesh_size_and_orientation():
    """The headline workload's mesh: 60,000 +- 1% triangles, dielectric hole
    walls with the kapton on the negative side (normals toward the axis)."""
    g = inputs.GemGeometry()
    m = inputs.gem_mesh_target(60000, g)
    assert abs(m.n - 60000) <= 600
    dd = m.kind == inputs.KIND_DIELECTRIC
    assert dd.sum() > 0 and np.all(m.eps_minus[dd] == g.eps_kapton) and np.all(m.eps_plus[dd] == 1.0)
    t = m.tri[dd]
    cen = t.mean(axis=1)
    nrm = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    hc = g.hole_centres()
    near = hc[np.argmin(((cen[:, None, :2] - hc[None]) ** 2).sum(-1), axis=1)]
    radial = cen[:, :2] - near
    assert np.all((nrm[:, :2] * radial).sum(1) < 0)
    assert set(np.unique(m.group[~dd]).tolist()) == {0, 1, 2, 3}
