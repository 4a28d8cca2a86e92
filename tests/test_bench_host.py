"""Host logic of bench.py that needs no GPU: the clock record taken during the
timed region (median SM clock, the highest max clock, throttle reasons seen)."""
import importlib.util
import os
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def test_clock_record_parses_samples_and_reasons():
    b = _bench()
    c = b.ClockSampler(0)
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    os.write(fd, b"0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Active\n"
                 b"0, 2065, 2070, 910.0, 0x4, Not Active, Not Active, Not Active, Not Active\n"
                 b"0, 1900, 2070, 905.0, 0x8, Not Active, Active, Not Active, Not Active\n"
                 b"garbage line\n")
    os.close(fd)
    c.proc, c.f = _Done(), open(os.devnull, "w")
    rec = c.stop()
    assert rec == {"sm_mhz": 2065.0, "sm_max_mhz": 2070.0, "reasons": ["hw_thermal_slowdown", "sw_power_cap"],
                   "samples": 3}
    assert not os.path.exists(c.path)  # the temporary record is removed


def test_clock_record_without_nvidia_smi_is_none(monkeypatch):
    b = _bench()
    monkeypatch.setenv("PATH", "")
    c = b.ClockSampler(0)
    c.start()
    if c.proc is not None:  # pragma: no cover - nvidia-smi found outside PATH
        pytest.skip("nvidia-smi available")
    assert c.stop() is None and not os.path.exists(c.path)


def test_launch_count_follows_the_library_plan():
    """The claimed launch count per solve: the FP64 sketch's column slabs (at most
    48e6 bytes of Y, a multiple of 32 columns), the blocked QR's 9 kernels per
    64-column panel, and the fixed kernels around them -- the counts the ncu launch
    list of the 5e6 x 2000 bench line showed (298 plain, 297 mixed)."""
    b = _bench()
    assert b.sketch_slabs(8000, 2001) == 3   # 736 columns of 64 KB each per slab
    assert b.sketch_slabs(2000, 501) == 1    # Y of 8 MB: one launch
    assert b.sketch_slabs(10 ** 6, 33) == 2  # d so large that a slab is the 32-column minimum
    assert b.launches_per_solve(2000, 8000, 0, True) == 298
    assert b.launches_per_solve(2000, 8000, 1, True) == 297
    assert b.launches_per_solve(500, 2000, 0, False) == 9
