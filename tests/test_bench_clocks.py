"""The bench's clock record on CPU: samples of nvidia-smi's csv output are kept
by timestamp inside the timed window (widened by one sampling period), the
median SM clock, the maximum clock and every active throttle reason are
reported, and a window with no sample gives no record."""
import datetime
import sys

from _tpt import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _line(t, sm, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ", ".join([t.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3], "0", str(sm), "2070", "512.5", "0x0"] + flags)


def _sampler(lines, t0, t1):
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    c.window = [t0, t1]
    c.proc = None
    return c


def _stop(c):
    # stop() without a running nvidia-smi: reuse its parsing on the stored lines
    class _P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    class _T:
        def join(self, timeout=None):
            pass

    c.proc, c._t = _P(), _T()
    return c.stop()


def test_samples_inside_the_window_are_kept():
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    t1 = t0 + datetime.timedelta(milliseconds=100)
    ms = datetime.timedelta(milliseconds=1)
    lines = [_line(t0 - 200 * ms, 900),                 # before: idle clocks, left out
             _line(t0 + 10 * ms, 2070),
             _line(t0 + 50 * ms, 2055, {"sw_power_cap"}),
             _line(t1 + 15 * ms, 2040),                 # within one period after the end
             _line(t1 + 300 * ms, 1000),                # after: left out
             "garbage line"]
    rec = _stop(_sampler(lines, t0, t1))
    assert rec["samples"] == 3 and rec["samples_outside_window"] == 2
    assert rec["sm_mhz"] == 2055.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert abs(rec["power_w"] - 512.5) < 1e-9


def test_no_sample_in_the_window_gives_no_record():
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    t1 = t0 + datetime.timedelta(milliseconds=40)
    lines = [_line(t0 - datetime.timedelta(seconds=1), 2070)]
    assert _stop(_sampler(lines, t0, t1)) is None
