"""Host logic of bench.py (no GPU): the all-pairs item count behind the
traffic figure, the traffic record's source check, and the clock sampler's
parsing of nvidia-smi output."""
import json
import os
import tempfile

import bench


def _items_by_rule(n):
    """Off-diagonal items of the cyclic tile pairing: item (I, d) pairs tile I
    with tile (I + d) mod n for d = 1 .. h_I, h_I = n // 2, less one for the
    upper half of the rows when n is even."""
    h = n // 2
    seen = set()
    for i in range(n):
        hi = h if (n % 2 == 1 or i < n // 2) else h - 1
        for d in range(1, hi + 1):
            j = (i + d) % n
            key = (min(i, j), max(i, j))
            assert key not in seen
            seen.add(key)
    return len(seen)


def test_sym_items_is_every_unordered_tile_pair_once():
    for n_tiles in range(1, 40):
        n = n_tiles * 1024 - 17
        assert bench.sym_items(n) == _items_by_rule(n_tiles) == n_tiles * (n_tiles - 1) // 2


def test_traffic_record_is_ignored_when_the_kernel_source_changed(monkeypatch):
    with open(bench.TRAFFIC_RECORD) as f:
        rec = json.load(f)
    fd, path = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    try:
        good = dict(rec, source_sha256=bench.kernel_source_sha256(rec["source"], rec["section_begin"],
                                                                  rec["section_end"]))
        with open(path, "w") as f:
            json.dump(good, f)
        monkeypatch.setattr(bench, "TRAFFIC_RECORD", path)
        n = 1_000_000
        want = rec["dram_bytes_per_item"] * bench.sym_items(n) + rec["dram_bytes_per_charge"] * n
        assert bench.nbody_traffic_per_launch(n) == want
        with open(path, "w") as f:
            json.dump(dict(rec, source_sha256="0" * 64), f)
        assert bench.nbody_traffic_per_launch(n) is None
    finally:
        os.unlink(path)


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parses_median_and_reasons():
    c = bench.Clocks(0)
    c.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    c.proc = _Proc()
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1300.4, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1210.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    c.f.write("\n".join(rows) + "\n")
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(c.f.name)


def test_clock_sampler_without_nvidia_smi():
    c = bench.Clocks(0)
    out = c.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
