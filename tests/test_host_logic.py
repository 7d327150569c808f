"""Host-side logic of the benchmark that needs no GPU."""
import bench


def test_kernel_identity_ignores_comments_only():
    a = "int f(int x) {  // add one\n  return x + 1; /* done */ }\n"
    b = "int f(int x) {\n  /* a longer\n     comment */ return x + 1;   }  // new note\n"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_tokens(a) == bench.code_tokens(b) == "int f(int x) { return x + 1; }"
    assert bench.code_tokens(c) != bench.code_tokens(a)


def test_kernel_source_sha_is_stable():
    assert bench.kernel_source_sha() == bench.kernel_source_sha()
    assert len(bench.kernel_source_sha()) == 16


class _Done:
    def join(self, timeout=None):
        pass

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _FakeNvml:
    def nvmlShutdown(self):
        return 0


def test_nvml_sampler_summary_maps_event_reasons():
    s = bench.NvmlSampler(0)
    s.thread, s.lib, s.max_mhz = _Done(), _FakeNvml(), 2070
    s.samples = [(2070, 0x0), (2055, 0x4), (2070, 0x1), (1900, 0x4 | 0x40)]
    out = s.stop()
    assert out["sm_mhz"] == 2062.5 and out["sm_max_mhz"] == 2070 and out["samples"] == 4
    # 0x1 (idle) is not a slowdown; 0x4 power cap, 0x40 hardware thermal
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_nvidia_smi_sampler_parses_its_csv(tmp_path):
    import tempfile
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False, dir=tmp_path)
    s.file.write("0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Active\n"
                 "0, 1980, 2070, 1390.0, 0x8, Active, Not Active, Not Active, Active\n"
                 "garbage line\n")
    out = s.stop()
    assert out["samples"] == 2 and out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2025.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_profiled_traffic_needs_the_current_kernel_sources(tmp_path, monkeypatch):
    """The committed ncu traffic is reported only while its kernel_source_sha
    matches the kernel sources' code."""
    sha = bench.kernel_source_sha()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ok.md").write_text(
        f"table\ntraffic_bytes_per_launch: 12345\nkernel_source_sha: {sha}\n")
    (tmp_path / "profiles" / "stale.md").write_text(
        "traffic_bytes_per_launch: 12345\nkernel_source_sha: 0123456789abcdef\n")
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("ok.md") == 12345.0
    assert bench.profiled_traffic("stale.md") is None
    assert bench.profiled_traffic("missing.md") is None
    monkeypatch.setattr(bench, "ROOT", real_root)
