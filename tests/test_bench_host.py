"""Host logic of bench.py on the CPU: the clock record taken during the timed region and the
DRAM-traffic lookup that the roofline line carries."""
import json
import os
import tempfile


class _Done:
    """Stands in for the finished nvidia-smi process."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(rows):
    import bench
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.index = 0
    s.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.f.write("\n".join(rows) + "\n")
    s.f.flush()
    s.p = _Done()
    return s


def test_clock_record_takes_the_median_and_the_active_reasons():
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    ck = _sampler(rows).stop()
    assert ck["sm_mhz"] == 2070.0 and ck["sm_max_mhz"] == 2070.0 and ck["samples"] == 3
    assert ck["reasons"] == ["sw_power_cap"]


def test_clock_record_reports_thermal_slowdown():
    rows = ["0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active"]
    ck = _sampler(rows).stop()
    assert ck["reasons"] == ["hw_thermal_slowdown"] and ck["sm_mhz"] == 1500.0


def test_clock_record_without_nvidia_smi():
    import bench
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.p = None
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_lookup_follows_the_source_hash(monkeypatch):
    """The committed counters count only while the kernel's source is the one they were taken
    on: a different hash gives null."""
    import bench
    with tempfile.TemporaryDirectory() as d:
        os.makedirs(os.path.join(d, "profiles"))
        os.makedirs(os.path.join(d, "paper_1905_04356_gb300", "csrc"))
        src = os.path.join(d, "paper_1905_04356_gb300", "csrc", "k.cu")
        with open(src, "w") as f:
            f.write("__global__ void k() {}\n")
        entry = {"k_demo": {"source_sha": bench.sha(src), "dram_bytes_per_launch": 1234}}
        with open(os.path.join(d, "profiles", "traffic.json"), "w") as f:
            json.dump(entry, f)
        monkeypatch.setattr(bench, "ROOT", d)
        assert bench.traffic_for("k_demo", "k.cu") == 1234
        assert bench.traffic_for("k_other", "k.cu") is None
        with open(src, "a") as f:
            f.write("// changed\n")
        assert bench.traffic_for("k_demo", "k.cu") is None


def test_committed_traffic_entries_name_existing_captures():
    import bench
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for name, e in t.items():
        assert os.path.exists(os.path.join(bench.ROOT, e["capture"])), name
        assert e["dram_bytes_per_launch"] > 0
