"""Host logic of bench.py that needs no GPU: the clock sampler's parsing of
nvidia-smi output, the peaks' fallbacks, and the traffic figure read from a
committed ncu summary only while the kernel source is the one profiled."""
import hashlib
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class FakeProc:
    def __init__(self, out):
        self.out = out
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def communicate(self, timeout=None):
        return self.out, ""


def sampled(out):
    s = bench.ClockSampler(None)
    s.proc = FakeProc(out)
    return s.stop()


def test_clock_sampler_median_max_and_reasons():
    out = "\n".join([
        "2032, 2032, 650.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1980, 2032, 700.4, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2032, 2032, 690.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbled line",
        "[N/A], 2032, 1.0, 0x0, Active, Active, Active, Active",  # unparsable clock: skipped whole
    ])
    r = sampled(out)
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2032.0 and r["sm_max_mhz"] == 2032.0 and r["power_w_max"] == 700.4
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_sampler_reports_every_throttle_reason_seen():
    out = "\n".join([
        "1500, 2032, 900, 0x1, Active, Not Active, Not Active, Not Active",
        "1400, 2032, 910, 0x1, Not Active, Active, Active, Not Active",
    ])
    r = sampled(out)
    assert r["sm_mhz"] == 1450.0
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(None)
    s.err = "not found"
    r = s.stop()
    assert r["sm_mhz"] is None and r["reasons"] == [] and r["error"] == "not found"


def test_peaks_fall_back_without_the_measurements(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6400.0, "of fallback")
    assert bench.measured_tensor_peak()[0] == 1400.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6493.4, "bf16_tflops_sustained": 1368.7}')
    assert bench.measured_peaks() == (6493.4, "of measured")
    assert bench.measured_tensor_peak()[0] == 1368.7


def test_committed_hash_kernel_profile_is_read_only_for_its_source():
    """The s24 summary under profiles/ gives its traffic figure exactly when
    its recorded sha256 is that of today's tc_hash.cu."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "profiles", "k_tc_hash_rmat24.md")).read()
    rec = text.split("kernel_source_sha256:")[1].split()[0]
    src = os.path.join(root, "paper_2209_04541_b300", "csrc", "tc_hash.cu")
    cur = hashlib.sha256(open(src, "rb").read()).hexdigest()
    t = bench.kernel_traffic("k_tc_hash", "rmat24")
    if rec == cur:
        assert isinstance(t, int) and t > 0
    else:
        assert t is None


def test_traffic_is_dropped_once_the_source_changes(monkeypatch, tmp_path):
    src_dir = tmp_path / "paper_2209_04541_b300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "tc_hash.cu"
    src.write_text("// kernel v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "k_tc_hash_w.md").write_text(
        f"kernel_source_sha256: {sha}\ntraffic_bytes_per_launch: 1234\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k_tc_hash", "w") == 1234
    src.write_text("// kernel v2\n")
    assert bench.kernel_traffic("k_tc_hash", "w") is None
    assert bench.kernel_traffic("k_tc_hash", "absent") is None
