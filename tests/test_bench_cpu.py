"""The benchmark's host-side pieces without a GPU: the reference arm (the FP64
oracle timed on the host cores) prints the contract's JSON line, and the clock
sampler keeps only the samples stamped inside the timed region."""
import datetime
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is True
    assert d["unit"] == "Mpixel/s" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "Mpixel/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "4096x4096-gauss3-L5"
    assert d["config"]["stop"].startswith("discrepancy")


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _sampler_with(rows, t_begin, t_end):
    sys.path.insert(0, ROOT)
    import bench

    c = bench.ClockSampler()
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    with open(c.path, "w") as f:
        for (ts, mhz, reasons) in rows:
            stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
            flags = ["Active" if r else "Not Active" for r in reasons]
            f.write(f"{stamp}, 0, {mhz}, 2070, 900.00, 0x0, " + ", ".join(flags) + "\n")
    c.proc = _Proc()
    c.t_begin, c.t_end = t_begin, t_end
    return c


def test_clock_sampler_keeps_the_timed_window():
    now = time.time()
    quiet = (False, False, False, False)
    rows = [(now - 0.30, 1500, (True, False, False, False)),  # before the region: ignored
            (now + 0.05, 2070, quiet), (now + 0.10, 2060, (False, False, False, True)),
            (now + 0.15, 2070, quiet),
            (now + 0.50, 900, (False, True, False, False))]  # after the region: ignored
    clk = _sampler_with(rows, now, now + 0.2).stop()
    assert clk["samples"] == 3 and clk["window"] == "timed region"
    assert clk["sm_mhz"] == 2070 and clk["sm_max_mhz"] == 2070
    assert clk["reasons"] == ["sw_power_cap"]


def test_clock_sampler_short_region_takes_the_nearest_sample():
    now = time.time()
    quiet = (False, False, False, False)
    rows = [(now - 0.2, 2000, quiet), (now + 0.06, 2070, quiet), (now + 0.4, 1000, quiet)]
    clk = _sampler_with(rows, now, now + 0.01).stop()
    assert clk["samples"] == 1 and clk["sm_mhz"] == 2070
    assert clk["window"].startswith("nearest sample")


def test_committed_traffic_profiles_match_the_sources():
    """The DRAM traffic the bench reports comes from committed ncu summaries; each
    one names a hash of the kernel sources it was taken on, and a summary taken
    on other sources is not used."""
    import bench

    tr, src = bench.profiled_traffic("4096x4096-gauss3-L5", 4)
    assert tr is not None, src
    assert abs(tr - 2.08e9) < 0.05e9
    vt, vsrc = bench.volume_traffic(bench.VOLUME["workload"])
    assert vt is not None, vsrc
    assert abs(vt - 2.97e9) < 0.05e9
    assert bench.volume_traffic("no-such-workload")[0] is None
