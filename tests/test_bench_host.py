"""bench.py's host logic: the recorded DRAM traffic is used only while the
kernel's source still matches the hash stored with it, the algorithmic bytes
follow their per-unit definitions, and the measured peaks are read from
MEASURED_PEAKS.json when it is there."""

import os

import bench


def test_recorded_traffic_follows_the_source_hash_and_scales_by_units(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha("read_kernel")
    assert len(sha) == 12
    f = tmp_path / "traffic.md"
    f.write_text("| kernel | case | unit | units | dram bytes | source |\n|---|---|---|---|---|---|\n"
                 f"| read_kernel | w | read | 1000 | 12345 | {sha} |\n"
                 "| flatten_kernel | w | element | 10 | 999 | 000000000000 |\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.recorded_traffic("read_kernel", 1000) == 12345
    assert bench.recorded_traffic("read_kernel", 4000) == 4 * 12345     # scaled by the units of the launch
    assert bench.recorded_traffic("flatten_kernel", 10) is None         # recorded on other source
    assert bench.recorded_traffic("sweep_b_kernel", 10) is None         # not recorded
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.md"))
    assert bench.recorded_traffic("read_kernel", 1000) is None


def test_every_kernel_with_sources_hashes_existing_files():
    for k, files in bench.KERNEL_SOURCES.items():
        assert files
        for f in files:
            assert os.path.exists(bench.kernel_source_path(f)), (k, f)


def test_algorithmic_bytes_per_unit():
    N, R, L, T, E, n = 1000, 3, 4, 8, 4, 64
    ab = bench.algorithmic_bytes(N, R, L, T, E, n)
    assert ab["insert"] == R * L * T * 4 + 2 * N * E
    assert ab["read"] == ab["write"] == n * (8 + 2 * E)
    assert ab["rw_b"] == ab["rw_g"] == ab["flatten"] == 2 * N * E


def test_peaks_come_from_the_measured_file():
    peak, src = bench.peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured" and peak > 1000
    else:
        assert peak > 1000
