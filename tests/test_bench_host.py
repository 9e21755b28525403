"""Host logic of bench.py (no GPU): the counted-work arithmetic behind the roofline
entry, the clock sampler's parsing of nvidia-smi lines (median SM clock, throttle
reasons that reject a run), and the command line's defaults (one GPU, at least three
warm-up steps)."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_counted_work_is_the_stated_per_unit_sum(bench):
    c = [0] * 16
    c[3], c[4], c[5], c[12] = 1000, 300, 50, 20          # node visits, triangle tests, texels, env lookups
    c[8], c[9], c[10], c[11] = 7, 5, 3, 2                 # shaded vertices per BSDF type
    c[7], c[13] = 40, 10                                  # gradient terms, of which texel terms
    flops, nbytes, grad = bench.counted_work(c, "wide")
    assert flops == 140 * 1000 + 45 * 300 + 250 * 7 + 415 * 5 + 130 * 3 + 450 * 2 + 60 * 20
    assert nbytes == 80 * 1000 + 48 * 300 + 16 * 50 + 16 * 20
    assert grad == 16 * 10 + 4 * 30
    f2, b2, _ = bench.counted_work(c, "binary")
    assert f2 == 44 * 1000 + 45 * 300 + 250 * 7 + 415 * 5 + 130 * 3 + 450 * 2 + 60 * 20
    assert b2 == 64 * 1000 + 48 * 300 + 16 * 50 + 16 * 20


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(bench, lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = list(lines)
    return s.stop()


def test_clock_sampler_median_and_reasons(bench):
    ok = "2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "1500, 2070, 1200.0, 0x40, Not Active, Active, Not Active, Not Active"
    r = _sampler(bench, [ok, ok, cap, ok, "garbage line", ""])
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 4
    assert r["reasons"] == ["sw_power_cap"]                 # kept and noted
    r = _sampler(bench, [ok, hot, hot])
    assert r["sm_mhz"] == 1500.0 and "hw_thermal_slowdown" in r["reasons"]   # a run to reject


def test_clock_sampler_without_nvidia_smi(bench):
    s = bench.ClockSampler(0)
    r = s.stop()                                            # never started
    assert r["sm_mhz"] is None and r["reasons"]


def test_command_line_defaults(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"])
    a = bench.parse()
    assert a.impl == "reference" and a.steps == 2
