"""Host logic of bench.py without a device: the summary of the clock samples that decides
whether a run is valid (median SM clock, throttle reasons), and the sampler around a stand-in
nvidia-smi process."""
import io

import bench


LINE = "{sm}, 2070, {pw}, 0x0000000000000000, {hw}, Not Active, Not Active, {cap}"


def test_summarise_clocks():
    lines = [LINE.format(sm=s, pw=p, hw="Not Active", cap="Not Active")
             for s, p in ((2070, 250.0), (2070, 261.9), (1995, 240.0))]
    lines.append(LINE.format(sm=2070, pw="[N/A]", hw="Not Active", cap="Active"))  # no power reading
    lines.append("garbage line")
    lines.append("[N/A], [N/A], [N/A], x, x, x, x, x")
    out = bench.summarise_clocks(lines)
    assert out["samples"] == 4 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["power_w_max"] == 261.9
    out = bench.summarise_clocks([LINE.format(sm=1200, pw=300, hw="Active", cap="Not Active")])
    assert out["reasons"] == ["hw_slowdown"] and out["sm_mhz"] == 1200.0
    out = bench.summarise_clocks([])
    assert out["sm_mhz"] is None and out["samples"] == 0 and out["reasons"] == []


class _FakeProc:
    def __init__(self, text):
        self.stdout = io.StringIO(text)
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def test_clock_sampler_with_a_stand_in_nvidia_smi(monkeypatch):
    procs = []

    def popen(cmd, **kw):
        assert cmd[0] == "nvidia-smi" and "--format=csv,noheader,nounits" in cmd
        assert "--query-gpu=" + bench.ClockSampler.FIELDS in cmd
        procs.append(_FakeProc("\n".join(LINE.format(sm=s, pw=200, hw="Not Active", cap="Not Active")
                                         for s in (2070, 2070, 2055)) + "\n"))
        return procs[-1]

    monkeypatch.setattr(bench.subprocess, "Popen", popen)
    s = bench.ClockSampler(0)
    s.start()
    out = s.stop()
    assert procs[0].terminated and out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["reasons"] == []

    def missing(cmd, **kw):
        raise OSError("no nvidia-smi")

    monkeypatch.setattr(bench.subprocess, "Popen", missing)
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_profiled_counters_need_the_same_kernel_sources(monkeypatch, tmp_path):
    """The roofline's ncu counters (DRAM bytes per launch, FP64 pipe active) come from the
    committed summary only while the hash of the sweep sources recorded there matches the
    sources being timed."""
    import os
    import shutil

    csrc = tmp_path / "paper_2410_05489_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.SWEEP_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2410_05489_gb300", "csrc", name), csrc / name)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.sweep_sources_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    prof = tmp_path / "profiles" / bench.SWEEP_PROFILE[9]
    assert bench.profiled_counters(9)[0] is None  # no summary
    prof.write_text("| table |\n\n    kernel-sources-sha256: %s\n    dram-bytes-per-launch: 5.8e7\n"
                    "    fp64-pipe-active: 0.85\n" % h)
    assert bench.profiled_counters(9)[:2] == (5.8e7, 0.85)
    with open(csrc / bench.SWEEP_SOURCES[1], "a") as f:
        f.write("\n// edited\n")
    assert bench.sweep_sources_hash() != h
    traffic, pipe, note = bench.profiled_counters(9)
    assert traffic is None and pipe is None and "changed" in note
