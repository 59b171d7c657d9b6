"""The benchmark's clock record, on CPU against a fake nvidia-smi: the samples kept are
those nvidia-smi stamped inside the timed region, whether it writes each line at once or
holds them in a buffer until it exits; a region shorter than the sampling interval is
described by the samples on either side of it, labelled as such; throttle reasons are
read per sample; a missing nvidia-smi gives an explicit "unavailable"."""
import os
import stat
import sys
import time

import pytest

FAKE = r'''#!{python}
import datetime, os, signal, sys, time
ms = int(sys.argv[sys.argv.index("-lms") + 1])
buffered = os.environ.get("FAKE_SMI_BUFFERED") == "1"
reason = os.environ.get("FAKE_SMI_POWER_CAP", "Not Active")
out = open(sys.stdout.fileno(), "w", buffering=(1 << 20) if buffered else 1, closefd=False)
signal.signal(signal.SIGTERM, lambda *a: (out.flush(), os._exit(0)))
while True:
    now = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    out.write(f"{{now}}, 2070, 2070, 612.50, Not Active, Not Active, Not Active, {{reason}}\n")
    time.sleep(ms / 1000.0)
'''


@pytest.fixture
def fake_smi(tmp_path, monkeypatch):
    d = tmp_path / "bin"
    d.mkdir()
    exe = d / "nvidia-smi"
    exe.write_text(FAKE.format(python=sys.executable))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{d}{os.pathsep}{os.environ['PATH']}")
    monkeypatch.setenv("MVP_BENCH_OUT", str(tmp_path / "out"))
    return monkeypatch


def _sampler(**kw):
    import bench

    return bench.ClockSampler(0, **kw)


@pytest.mark.parametrize("buffered", ["0", "1"])
def test_samples_inside_the_region(fake_smi, buffered):
    fake_smi.setenv("FAKE_SMI_BUFFERED", buffered)
    with _sampler(interval_ms=40, start_timeout_s=0.5) as clk:
        time.sleep(0.5)
    s = clk.summary()
    assert s["window"] == "timed region"
    assert 6 <= s["samples"] <= 14, s
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == []


def test_power_cap_reason_is_reported(fake_smi):
    fake_smi.setenv("FAKE_SMI_POWER_CAP", "Active")
    with _sampler(interval_ms=40) as clk:
        time.sleep(0.2)
    assert clk.summary()["reasons"] == ["sw_power_cap"]


def test_short_region_is_bracketed(fake_smi):
    with _sampler(interval_ms=300) as clk:
        pass
    s = clk.summary()
    assert s["window"].startswith("bracketing")
    assert 1 <= s["samples"] <= 2 and s["sm_mhz"] == 2070.0


def test_missing_tool_is_unavailable(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    monkeypatch.setenv("MVP_BENCH_OUT", str(tmp_path / "out"))
    with _sampler() as clk:
        pass
    assert clk.summary()["reasons"] == ["unavailable"]
