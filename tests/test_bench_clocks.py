"""The benchmark's clock record: only nvidia-smi samples inside the timed
window count (or the two bracketing it when the window is shorter than the
sampling period), with the throttle reasons that were active in them."""

import datetime
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _row(ts, mhz, active="Not Active", power_cap="Not Active"):
    return "%s, 0, %d, 2070, 900.0, 0x0, %s, Not Active, Not Active, %s" % (
        ts.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3], mhz, active, power_cap)


def _clocks(bench, tmp_path, rows, t0, t1):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    c.fh = open(c.path, "a")
    c.proc = _Done()
    c.t0, c.t1 = t0, t1
    return c.stop()


def test_samples_inside_the_window(bench, tmp_path):
    base = datetime.datetime(2026, 1, 1, 12, 0, 0)
    ms = datetime.timedelta(milliseconds=1)
    rows = [_row(base + k * 50 * ms, mhz) for k, mhz in enumerate([1200, 2070, 2070, 1980, 900])]
    rows[3] = _row(base + 150 * ms, 1980, power_cap="Active")
    r = _clocks(bench, tmp_path, rows, base + 40 * ms, base + 160 * ms)
    assert r["samples"] == 3  # 50, 100, 150 ms
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]


def test_short_window_takes_the_bracketing_samples(bench, tmp_path):
    base = datetime.datetime(2026, 1, 1, 12, 0, 0)
    ms = datetime.timedelta(milliseconds=1)
    rows = [_row(base + k * 50 * ms, mhz) for k, mhz in enumerate([1500, 2070, 2040])]
    r = _clocks(bench, tmp_path, rows, base + 60 * ms, base + 80 * ms)
    assert r["samples"] == 2  # the last sample before the window's end (50 ms) and the next one (100 ms)
    assert r["sm_mhz"] == pytest.approx((2070 + 2040) / 2.0)
