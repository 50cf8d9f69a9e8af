"""Host logic of bench.py on CPU: the profiled-traffic lookup (kept only while
the kernel sources match the capture) and the roofline arithmetic of the
Jacobi object."""
import hashlib

import pytest

import bench


def _write_profile(root, src_text, traffic="1234000", sha=None):
    (root / "profiles").mkdir(exist_ok=True)
    (root / "k.cu").write_text(src_text)
    digest = sha or hashlib.sha256(src_text.encode()).hexdigest()
    (root / "profiles" / "p.md").write_text(
        "# a capture\n\ntraffic_bytes: %s\ntraffic_unit: per launch\nsources: k.cu\n"
        "sources_sha256: %s\n" % (traffic, digest))


def test_profiled_traffic_kept_while_sources_match(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write_profile(tmp_path, "kernel v1")
    tr = bench.profiled_traffic("p.md")
    assert tr == {"bytes": 1234000.0, "unit": "per launch", "source": "profiles/p.md"}
    (tmp_path / "k.cu").write_text("kernel v2")          # the kernel changed since
    assert bench.profiled_traffic("p.md") is None


def test_profiled_traffic_missing_fields_or_files(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("absent.md") is None
    _write_profile(tmp_path, "kernel", sha="0" * 64)       # recorded hash is wrong
    assert bench.profiled_traffic("p.md") is None
    (tmp_path / "profiles" / "q.md").write_text("traffic_bytes: 5\n")  # no sources
    assert bench.profiled_traffic("q.md") is None


def test_jacobi_roofline_arithmetic():
    st = {"jacobi_pair_rows": 1_000_000, "jacobi_rot_rows": 400_000, "jacobi_alg_bytes": 3_000,
          "jacobi_sweeps": 50, "svds": 10}
    steps, t_local = 2, 1.0                 # 2 steps in 1 s
    prof_jac = (600.0, 20)                  # 600 ms over 20 launches (10 per step)
    prof_lq = (100.0, 20)
    r = bench.jacobi_roofline(st, prof_jac, steps, t_local, 50.0, "test peak", prof_lq)
    alg = 8 * 1_000_000 + 18 * 400_000      # flops of the counted pairs
    per_launch = alg / 10
    assert r["alg_flops_per_launch"] == pytest.approx(per_launch)
    assert r["avg_launch_ms"] == pytest.approx(30.0)
    assert r["achieved"] == pytest.approx(per_launch / 0.030 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 50.0)
    assert r["share_of_step"] == pytest.approx(0.6)
    assert r["sweeps_per_svd"] == pytest.approx(5.0)
    assert r["alg_bytes_per_launch"] == pytest.approx(300.0)
    pre = r["preconditioner"]
    assert pre["ms_per_step"] == pytest.approx(50.0)
    assert pre["launches_per_step"] == pytest.approx(10.0)
    assert pre["share_of_step"] == pytest.approx(0.1)
    assert bench.jacobi_roofline(st, prof_jac, steps, t_local, 50.0, "p", (0.0, 0))[
        "preconditioner"] is None
