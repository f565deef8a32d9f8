"""Host logic of bench.py: the algorithmic byte model behind the roofline
fractions, and the rule that the recorded DRAM traffic is reported only for
the push source and settings it was measured with.  No GPU."""
import hashlib
import importlib.util
import json
import os
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _wl(nx, ny, nz, n, sort_every, open_faces=0):
    return types.SimpleNamespace(
        params={"nx": nx, "ny": ny, "nz": nz, "sort_every": sort_every, "open_faces": open_faces},
        n_particles=n)


def test_step_bytes_of_the_2d_harris_benchmark():
    # 1024x512 cells, 100 ions per cell, sort every 8 steps: per ion 28 B read
    # (cell, ox, oz, vx, vy, vz, w) and 24 B written; per cell E, B read (24 B)
    # and n, J written (16 B); the rest of the field phase 84 B per cell; the
    # sort (20 B key inputs + 28 B read + 28 B written) / 8 per ion
    b = _bench()
    n, ncell = 52_428_800, 524_288
    d = b.step_bytes(_wl(1024, 1, 512, n, 8))
    assert d["push"] == n * 52 + ncell * 40 == 2_747_269_120
    assert d["field"] == ncell * 84
    assert d["sort"] == n * 76 / 8
    assert d["total"] == d["push"] + d["field"] + d["sort"] == 3_289_382_912
    assert b.push_bytes_per_launch(_wl(1024, 1, 512, n, 8)) == d["push"]


def test_step_bytes_3d_and_open_faces():
    b = _bench()
    n, ncell = 268_435_456, 256 * 128 * 128
    d = b.step_bytes(_wl(256, 128, 128, n, 20))
    assert d["push"] == n * 60 + ncell * 40  # 32 B read + 28 B written per ion
    assert d["sort"] == n * (28 + 2 * 32) / 20
    # open faces: the key is the cell alone; no sort means no sort bytes
    assert b.step_bytes(_wl(64, 1, 32, 1000, 4, open_faces=1))["sort"] == 1000 * (4 + 56) / 4
    assert b.step_bytes(_wl(64, 1, 32, 1000, 0))["sort"] == 0.0


def test_traffic_reported_only_for_the_recorded_sources(tmp_path, monkeypatch):
    b = _bench()
    csrc = tmp_path / "paper_2305_05600_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "hv_push.cu").write_bytes(b"push source")
    (csrc / "hv_internal.cuh").write_bytes(b"#define HV_PUSH_SPLIT 2")
    h = hashlib.sha256(b"push source" + b"#define HV_PUSH_SPLIT 2").hexdigest()[:16]
    rec = tmp_path / "profiles" / "push_traffic.json"
    rec.write_text(json.dumps({"harris2d": {"source_sha": h, "dram_bytes_per_launch": 123}}))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.traffic_record("harris2d") == 123.0
    assert b.traffic_record("beam3d") is None
    # a changed setting (or source) voids the record
    (csrc / "hv_internal.cuh").write_bytes(b"#define HV_PUSH_SPLIT 4")
    assert b.traffic_record("harris2d") is None
    rec.unlink()
    assert b.traffic_record("harris2d") is None
