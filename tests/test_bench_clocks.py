"""bench.py's clock record from nvidia-smi lines (CPU only, synthetic
lines): the median SM clock and the throttle reasons of the samples inside
the timed window, and every sample when none arrived inside it."""
import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _line(mhz, hw_slow="Not Active", power="Not Active"):
    return f"0, {mhz}, 2032, 700.00, 0x0000000000000000, {hw_slow}, Not Active, Not Active, {power}"


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.proc = _Proc()
    c.lines = list(lines)
    return c


def test_window_keeps_timed_samples():
    c = _sampler([(0.0, _line(1000, hw_slow="Active")), (10.0, _line(2032)), (10.1, _line(2000, power="Active")),
                  (10.2, _line(2032)), (30.0, _line(500))])
    r = c.stop(window=(9.95, 10.2))
    assert r["samples"] == 3 and r["sm_mhz"] == 2032.0 and r["sm_max_mhz"] == 2032.0
    assert r["reasons"] == ["sw_power_cap"] and r["window"] == "timed region"


def test_no_sample_in_window_uses_all():
    c = _sampler([(0.0, _line(2032)), (5.0, _line(1990))])
    r = c.stop(window=(2.0, 2.1))
    assert r["samples"] == 2 and r["window"] == "whole sampling run"


def test_unavailable():
    c = bench.ClockSampler(0)
    r = c.stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]
