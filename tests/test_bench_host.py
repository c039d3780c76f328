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
