"""The double-GEM workload's inputs (no GPU): two single-GEM foils 2 mm apart,
120,000 +- 1 % cells, six electrode groups, a 4096-point probe line through a
hole axis, and charge clouds outside the solids."""
import numpy as np

from paper_2110_09214_gb300 import inputs


def test_double_gem_mesh_size_groups_and_orientation():
    d = inputs.DoubleGemGeometry()
    m = inputs.double_gem_mesh_target(120000, d)
    assert abs(m.n - 120000) <= 1200
    dd = m.kind == inputs.KIND_DIELECTRIC
    assert set(np.unique(m.group[~dd]).tolist()) == {0, 1, 2, 3, 4, 5}
    # potentials rise from the drift plane to the anode, 400 V across each foil
    v = m.group_voltage
    assert np.all(np.diff(v) > 0) and v[5] == 0.0
    assert abs((v[2] - v[1]) - d.foil.dv_gem) < 1e-9 and abs((v[4] - v[3]) - d.foil.dv_gem) < 1e-9
    assert abs((v[3] - v[2]) - d.e_transfer * (d.spacing - 2 * d.foil.z_top)) < 1e-9
    # each foil is the single-GEM foil moved along z: same cell counts per group
    cnt = [int((m.group[~dd] == k).sum()) for k in range(6)]
    assert cnt[1] == cnt[2] == cnt[3] == cnt[4] and cnt[0] == cnt[5]
    # kapton walls of both foils, kapton on the negative side (normals toward the axis)
    t = m.tri[dd]
    cen = t.mean(axis=1)
    assert (np.abs(cen[:, 2] - d.z_upper) < d.foil.t_kapton).sum() == dd.sum() // 2
    assert (np.abs(cen[:, 2] - d.z_lower) < d.foil.t_kapton).sum() == dd.sum() // 2
    nrm = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    hc = d.foil.hole_centres()
    near = hc[np.argmin(((cen[:, None, :2] - hc[None]) ** 2).sum(-1), axis=1)]
    assert np.all((nrm[:, :2] * (cen[:, :2] - near)).sum(1) < 0)
    assert np.all(m.eps_minus[dd] == d.foil.eps_kapton) and np.all(m.eps_plus[dd] == 1.0)
    # every vertex lies between the anode and the drift plane
    z = m.tri[..., 2]
    assert z.min() >= d.z_anode - 1e-12 and z.max() <= d.z_drift + 1e-12


def test_double_gem_probe_line_and_charges():
    mesh, gas, ch, trk, d, probe = inputs.config_double_gem(seed=3, n=4000, target_panels=20000)
    assert probe.shape == (4096, 3)
    assert np.all(probe[:, :2] == 0.0)
    assert np.all(np.diff(probe[:, 2]) > 0)
    assert probe[0, 2] > d.z_anode and probe[-1, 2] < d.z_drift
    assert not inputs.double_gem_inside_solid(d, probe).any()
    # the probe passes through both foils (inside their holes)
    for zf in (d.z_upper, d.z_lower):
        assert (np.abs(probe[:, 2] - zf) < d.foil.z_top).sum() > 0
    p = ch.pos_q[:, :3].astype(np.float64)
    assert ch.n == 4000 and (ch.species == inputs.SP_ELECTRON).sum() == 2000
    assert not inputs.double_gem_inside_solid(d, p).any()
    # clouds around both foils
    assert (p[:, 2] > 0).sum() > 1000 and (p[:, 2] < 0).sum() > 1000
    assert trk.z_lo == d.z_anode and trk.z_hi == d.z_drift


def test_inside_solid_marks_copper_and_kapton_of_both_foils():
    d = inputs.DoubleGemGeometry()
    a = d.foil.pitch / 2.0           # between two holes: solid across the foil's thickness
    for zf in (d.z_upper, d.z_lower):
        pts = np.array([[a * 0.9, 0.0, zf + dz] for dz in (-0.9 * d.foil.z_top, 0.0, 0.9 * d.foil.z_top)])
        assert inputs.double_gem_inside_solid(d, pts).all()
        # on the hole axis and outside the foil: gas
        gas_pts = np.array([[0.0, 0.0, zf], [a * 0.9, 0.0, zf + 1.5 * d.foil.z_top]])
        assert not inputs.double_gem_inside_solid(d, gas_pts).any()
    # the transfer gap between the foils is gas
    assert not inputs.double_gem_inside_solid(d, np.array([[a * 0.9, 0.0, 0.0]])).any()
