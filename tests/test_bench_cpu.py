"""Host logic of bench.py (no GPU): the ncu records it cites are used only while the kernel source
they were taken on is unchanged, and the measured-peak fallback."""
import os
import shutil

import bench

REPO = bench.ROOT


def _tree(tmp_path, traffic_lines, pipes_lines):
    csrc = tmp_path / "paper_2003_03590_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(REPO, "paper_2003_03590_gb300", "csrc")
    for f in ("gp_fft.cuh", "gp_sweep.cuh", "gp_tma.cuh", "gp_plane.cuh"):
        shutil.copy(os.path.join(src, f), csrc / f)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.txt").write_text("# comment\n" + "\n".join(traffic_lines) + "\n")
    (prof / "ncu_pipes.txt").write_text("# comment\n" + "\n".join(pipes_lines) + "\n")
    return csrc


def test_records_follow_the_kernel_source(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()                  # of the repository's headers (copied below)
    assert len(h) == 16 and int(h, 16) >= 0
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = _tree(tmp_path,
                 [f"k_tma_plane<256> 256 301206528 {h}", "k_tma_plane<256> 512 999 0000000000000000",
                  f"k_tma_strided<256> 256 204509184 {h}"],
                 [f"k_tma_plane<256> 256 43.01 48.82 {h}"])
    assert bench.kernel_source_hash() == h
    assert bench.ncu_traffic("k_tma_plane<256>", 256) == 301206528.0
    assert bench.ncu_traffic("k_tma_strided<256>", 256) == 204509184.0
    assert bench.ncu_traffic("k_tma_plane<256>", 512) is None          # another hash
    assert bench.ncu_traffic("k_tma_contig<256>", 256) is None         # no record
    p = bench.ncu_pipes("k_tma_plane<256>", 256)
    assert p["fma_pipe_active_pct"] == 43.01 and p["issue_active_pct"] == 48.82
    # any change of a kernel header makes the records stale: reported as unknown
    with open(csrc / "gp_sweep.cuh", "a") as f:
        f.write("\n// changed\n")
    assert bench.kernel_source_hash() != h
    assert bench.ncu_traffic("k_tma_plane<256>", 256) is None
    assert bench.ncu_pipes("k_tma_plane<256>", 256) is None


def test_peak_fallback_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, src = bench.peaks()
    assert peak == 6800.0 and "fallback" in src
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6788.6}')
    peak, src = bench.peaks()
    assert peak == 6788.6 and "measured" in src
