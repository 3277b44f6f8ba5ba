"""Host logic of bench.py's clock record (no GPU): the sampler runs nvidia-smi during the timed
region and summarises its CSV lines into the median SM clock, the maximum clock and the
throttle reasons seen active."""
import os
import time

import bench

# nvidia-smi's csv,noheader,nounits line for the sampler's fields: index, clocks.sm,
# clocks.max.sm, power.draw, reasons bitmask, hw_slowdown, hw_thermal_slowdown,
# sw_thermal_slowdown, sw_power_cap
FAKE = """#!/bin/sh
i=0
while [ $i -lt 100 ]; do
  if [ $i -eq 2 ]; then
    echo "0, 1800, 2032, 1090.0, 0x4, Not Active, Not Active, Not Active, Active"
  else
    echo "0, 2032, 2032, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
  fi
  sleep 0.02
  i=$((i+1))
done
"""


def test_clock_sampler_summarises_samples(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    with bench.ClockSampler(0) as clk:
        time.sleep(0.5)
    s = clk.summary()
    assert s["samples"] >= 5
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0   # the median ignores one dip
    assert s["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(clk.path)                            # the sample file is removed


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # an empty directory: no nvidia-smi
    with bench.ClockSampler(0) as clk:
        pass
    s = clk.summary()
    assert s["sm_mhz"] is None and s["sm_max_mhz"] is None and s["reasons"] == ["no samples"]
