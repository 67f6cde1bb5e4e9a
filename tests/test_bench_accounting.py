"""Host-side accounting of bench.py: the algorithmic bytes the roofline divides by, and the
rule that the DRAM traffic figure is reported only for the kernel sources it was measured on.
No GPU is used."""
import os

import pytest

import bench
from paper_2607_24214_b300 import config


def test_bytes_per_update_c2_is_172():
    # C2 (4 plasma, 8 beam particles per cell): 4 x 32 B of plasma state, 8 x 60 B of beam
    # state, 2 x 16 B of sources and 2 x 24 B of fields per cell and slice = 688 B per cell,
    # 172 B per plasma particle-slice update.
    assert bench.bytes_per_update(config.c2_mixed_electron_beam()) == pytest.approx(172.0)


def test_launch_bytes_add_up():
    p = config.c2_mixed_electron_beam()
    cells = p.nx * p.ny
    ppc = p.ppc_plasma_x * p.ppc_plasma_y
    updates = ppc * cells * p.nxi
    # one step's sweep and push together carry every byte of the per-update count
    assert bench.sweep_bytes(p) + bench.push_bytes(p) == pytest.approx(
        bench.bytes_per_update(p) * updates)
    assert bench.pipe_bytes(p, 16) == pytest.approx(16 * bench.bytes_per_update(p) * updates)
    # 738.7 GB per 16-step launch at C2
    assert bench.pipe_bytes(p, 16) / 1e9 == pytest.approx(738.73, rel=1e-4)


def _summary(tmp_path, sha, workload, nbytes):
    f = tmp_path / "traffic.md"
    f.write_text(
        "# a capture\n\nsome text\n\n"
        f"- kernel sources sha256: {sha}\n"
        f"- workload: {workload}\n"
        f"- dram bytes per launch: {nbytes}\n")
    return str(f)


def test_traffic_reported_only_for_the_measured_sources(tmp_path, monkeypatch):
    p = config.c2_mixed_electron_beam()
    work = f"nx {p.nx}, ny {p.ny}, nxi {p.nxi}, steps per launch 16"
    sha = bench.kernel_sources_sha256()
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _summary(tmp_path, sha, work, 123456789))
    assert bench.measured_traffic(p, 16) == 123456789.0
    # another launch length or grid: not this capture
    assert bench.measured_traffic(p, 8) is None
    assert bench.measured_traffic(p.with_(nxi=512), 16) is None
    # another kernel: the counters no longer describe it
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _summary(tmp_path, "0" * 64, work, 123456789))
    assert bench.measured_traffic(p, 16) is None
    # no summary, or an unreadable figure
    monkeypatch.setattr(bench, "TRAFFIC_FILE", os.path.join(str(tmp_path), "missing.md"))
    assert bench.measured_traffic(p, 16) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _summary(tmp_path, sha, work, "n/a"))
    assert bench.measured_traffic(p, 16) is None


def test_sources_hash_covers_every_cuda_source(tmp_path, monkeypatch):
    # the hash follows every .cu, .cuh and .h file of the library's csrc, and nothing else
    csrc = tmp_path / "paper_2607_24214_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text("kernel a\n")
    (csrc / "b.cuh").write_text("header b\n")
    (csrc / "c.h").write_text("header c\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_sha256()
    assert len(h0) == 64 and h0 == bench.kernel_sources_sha256()
    (csrc / "notes.txt").write_text("not a source\n")
    assert bench.kernel_sources_sha256() == h0
    for name in ("a.cu", "b.cuh", "c.h"):
        old = (csrc / name).read_text()
        (csrc / name).write_text(old + " ")
        assert bench.kernel_sources_sha256() != h0, name
        (csrc / name).write_text(old)
    assert bench.kernel_sources_sha256() == h0
