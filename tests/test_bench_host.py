"""Host-side logic of bench.py that needs no GPU: the committed ncu figures
are reported only while the kernel source matches the recorded hash, and
the clock record is parsed from nvidia-smi's CSV rows."""
import hashlib
import tempfile

import bench


def test_committed_profile_follows_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cuh"
    src.write_text("__global__ void k() {}\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "voronoi_annulus_1e6.md").write_text(
        "traffic_bytes_per_launch: 1234\nwarp_instructions_per_launch: 5678\n"
        f"voronoi_cuh_sha256_16: {digest}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.committed_profile(str(src)) == (1234.0, 5678.0)
    assert bench.committed_profile(str(src), 200_000) == (None, None)  # captured on 1e6 points only
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.committed_profile(str(src)) == (None, None)
    (prof / "voronoi_annulus_1e6.md").unlink()
    assert bench.committed_profile(str(src)) == (None, None)


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_parsing():
    s = bench.ClockSampler(0)
    s.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.f.write("2026/12/04 12:00:00.000, 0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "2026/12/04 12:00:00.020, 0, 2055, 2070, 1200.5, 0x4, Not Active, Not Active, Not Active, Active\n"
              "2026/12/04 12:00:00.040, 0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "garbage line\n")
    s.proc = _Proc()
    rec = s.stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_clock_rows_inside_the_timed_window():
    import datetime

    def row(t, mhz, cap="Not Active"):
        ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return [ts, "0", str(mhz), "2070", "1000", "0x0", "Not Active", "Not Active", "Not Active", cap]

    t = 1_800_000_000.0
    rows = [row(t, 1500, "Active"), row(t + 0.02, 2070), row(t + 0.04, 2060), row(t + 0.06, 1400, "Active")]
    rec = bench.ClockSampler.parse(rows, t + 0.01, t + 0.05)
    assert rec["samples"] == 2 and rec["sm_mhz"] == 2065.0 and rec["reasons"] == []
    # a window between two rows takes the nearest row on each side
    rec = bench.ClockSampler.parse(rows, t + 0.041, t + 0.045)
    assert rec["samples"] == 2 and rec["reasons"] == ["sw_power_cap"]
