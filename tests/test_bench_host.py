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


def test_issue_roofline_from_the_recorded_instructions(tmp_path, monkeypatch):
    digest = bench.kernel_source_digest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: digest)
    assert bench.issue_roofline("g2p", 0.07, 152, 2070.0) is None  # no summary
    d = tmp_path / "profiles"
    d.mkdir()
    (d / "g2p_tissue_block_1m.md").write_text(
        f"traffic_bytes_per_launch: 1\nwarp_instructions_per_launch: 46000000\nsource_digest: {digest}\n")
    r = bench.issue_roofline("g2p", 0.0736, 152, 2070.0)
    peak = 152 * 4 * 2.070  # G warp instructions per second
    assert r["peak"] == round(peak, 1)
    assert abs(r["frac"] - 46e6 / 0.0736e-3 / 1e9 / peak) < 1e-4
    assert abs(r["floor_ms"] - 46e6 / (peak * 1e9) * 1e3) < 1e-5
    assert bench.issue_roofline("g2p", 0.0736, 152, None) is None  # no clock sample


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
    # whole-line comments and blank lines are documentation, not kernel code
    (csrc / "b.cuh").write_text("// a note\n\nheader B changed\n   // another note\n")
    assert bench.kernel_source_digest() == d1
    (csrc / "b.cuh").write_text("header B changed  // a trailing comment is part of the line\n")
    assert bench.kernel_source_digest() != d1


def test_algorithmic_bytes_per_unit():
    # The method's bytes per particle-substep: P2G reads x, v, C, F (96 B), G2P
    # reads x, F and writes x, v, C, F (144 B), the sort writes and reads key and
    # permutation (16 B); the grid moves 72 B per active node.
    N, nodes = 1 << 20, 3150 * 64
    ab = bench.algorithmic_bytes(N, nodes)
    assert ab == {"sort": 16 * N, "p2g": 96 * N, "grid": 72 * nodes, "g2p": 144 * N}
    assert (sum(ab.values()) / N) == pytest.approx(256 + 72 * nodes / N)
    # ~270 B per particle-substep at 8 particles per cell and ~1.5 active nodes per cell
    assert 265 < 256 + 72 * (1.5 / 8) < 271


def test_implementation_bytes_per_unit():
    N, bricks, nodes = 1 << 20, 64 ** 3, 3150 * 64
    ib = bench.implementation_bytes(N, bricks, nodes)
    assert ib["sort"] == 8 * bricks + 17 * N
    assert ib["p2g"] == 93 * N + 16 * nodes
    assert ib["grid"] == 48 * nodes
    assert ib["g2p"] == 188 * N + 16 * nodes
    # per-particle materials add mu and lambda to G2P's reads and writes
    assert bench.implementation_bytes(N, bricks, nodes, pp_mat=True)["g2p"] == ib["g2p"] + 16 * N


def test_roofline_fraction_reproduces_from_the_survey_bytes():
    # frac = algorithmic bytes of the dominant kernel x N / its launch time / peak
    N, nodes = 1 << 20, 201600
    per = {"sort": 0.017, "p2g": 0.069, "grid": 0.011, "g2p": 0.0805}
    r = bench.roofline_fields(N, 64 ** 3, nodes, per, 0.162, 6790.7, "measured")
    assert r["kernel"] == "g2p"
    assert r["frac"] == pytest.approx(144 * N / (0.0805e-3) / 1e9 / 6790.7, abs=1e-4)
    assert r["whole_substep_frac"] == pytest.approx((256 * N + 72 * nodes) / 0.162e-3 / 1e9 / 6790.7, abs=1e-4)
    assert r["implementation_bytes_per_launch"] == 188 * N + 16 * nodes


@pytest.mark.parametrize("world,units,ms", [(1, 1000, 10.0), (4, 2500, 8.0)])
def test_whole_job_rate_counts_every_rank(world, units, ms):
    assert bench.whole_job_rate(world, units, ms) == pytest.approx(world * units / (ms / 1e3))
