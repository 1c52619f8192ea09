"""Host logic of bench.py's roofline fields, on CPU: the recorded ncu traffic is
reported only while the CUDA sources match the digest stored with it, and the
algorithmic bytes follow the per-particle and per-node counts of each kernel."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, kernel, traffic, digest):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / f"{kernel}_tissue_block_1m.md").write_text(
        f"# summary\n\n| metric | value |\n\ntraffic_bytes_per_launch: {traffic}\nsource_digest: {digest}\n")


def test_recorded_traffic_follows_the_digest(tmp_path, monkeypatch):
    digest = bench.kernel_source_digest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: digest)
    assert bench.recorded_traffic("g2p") is None  # no summary
    _summary(tmp_path, "g2p", 123456, digest)
    assert bench.recorded_traffic("g2p") == 123456
    _summary(tmp_path, "g2p", 123456, "0" * 16)  # the kernels changed since the capture
    assert bench.recorded_traffic("g2p") is None


def test_source_digest_changes_with_any_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2502_18437_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text("kernel A")
    (csrc / "b.cuh").write_text("header B")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.kernel_source_digest()
    (csrc / "b.cuh").write_text("header B changed")
    d1 = bench.kernel_source_digest()
    (csrc / "notes.txt").write_text("not a source")
    assert d0 != d1 and bench.kernel_source_digest() == d1


def test_algorithmic_bytes_per_unit():
    N, bricks, nodes = 1 << 20, 64 ** 3, 3150 * 64
    ab = bench.algorithmic_bytes(N, bricks, nodes)
    assert ab["sort"] == 8 * bricks + 17 * N
    assert ab["p2g"] == 93 * N + 16 * nodes
    assert ab["grid"] == 48 * nodes
    assert ab["g2p"] == 188 * N + 16 * nodes
    # per-particle materials add mu and lambda to G2P's reads and writes
    assert bench.algorithmic_bytes(N, bricks, nodes, pp_mat=True)["g2p"] == ab["g2p"] + 16 * N


@pytest.mark.parametrize("world,units,ms", [(1, 1000, 10.0), (4, 2500, 8.0)])
def test_whole_job_rate_counts_every_rank(world, units, ms):
    assert bench.whole_job_rate(world, units, ms) == pytest.approx(world * units / (ms / 1e3))
