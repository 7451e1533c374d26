"""Host-side arithmetic of bench.py, checked on the CPU: the roofline of the
dominant kernel family, the clock record's parsing, the FP64 ALU peak from
unit counts and clocks, and the whole-job throughput of replicas."""
import importlib.util
import os

import numpy as np
import pytest
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_roofline_picks_the_dominant_family_and_its_bound(bench):
    # 1 TFLOP/s FP64 and 5000 GB/s: balance 0.2 flop/byte
    prof = {
        "dense": {"ms": 300.0, "groups": 10, "launches": 100, "bytes": 1e9, "flops": 2.4e11},
        "stream": {"ms": 100.0, "groups": 100, "launches": 200, "bytes": 4e11, "flops": 1e10},
    }
    roof, table = bench.pick_roofline(prof, hbm_gbs=5000.0, fp64_tflops=1.0)
    assert roof["kernel"] == "dense" and roof["bound"] == "alu"
    assert roof["achieved"] == pytest.approx(2.4e11 / 0.3 / 1e12)      # 0.8 TFLOP/s
    assert roof["frac"] == pytest.approx(0.8)
    assert roof["avg_launch_ms"] == pytest.approx(3.0)
    assert roof["algorithmic_flops_per_launch"] == pytest.approx(2.4e9)
    assert roof["traffic"] is None
    assert sum(v["share"] for v in table.values()) == pytest.approx(1.0, abs=1e-3)
    assert list(table) == ["dense", "stream"]
    # the same families with the streaming one dominant: an HBM bound
    prof["stream"]["ms"] = 1000.0
    roof, _ = bench.pick_roofline(prof, hbm_gbs=5000.0, fp64_tflops=1.0)
    assert roof["kernel"] == "stream" and roof["bound"] == "hbm"
    assert roof["achieved"] == pytest.approx(400.0) and roof["unit"] == "GB/s"
    assert roof["frac"] == pytest.approx(400.0 / 5000.0)
    assert bench.pick_roofline({}, 5000.0, 1.0) == (None, {})
    # a composite wall-time family (two concurrent inversions) is never chosen
    prof["gje_invert"] = {"ms": 5000.0, "groups": 1, "launches": 10, "bytes": 1e9, "flops": 1e13}
    roof, table = bench.pick_roofline(prof, hbm_gbs=5000.0, fp64_tflops=1.0)
    assert roof["kernel"] == "stream" and "gje_invert" in table


def test_roofline_bounds_of_the_tensor_core_engine(bench):
    """With the tensor-core engine the emulated FP64 products are rated
    against the tensor cores' FP64-equivalent peak (sustained BF16 / 36) and
    the whitening products against HBM, whatever their FP64 intensity; with
    the FP64 engine the intensity rule holds."""
    prof = {
        "gje_update_H": {"ms": 400.0, "groups": 4, "launches": 40, "bytes": 1e9, "flops": 4e12},
        "whiten_qt_dot": {"ms": 300.0, "groups": 3, "launches": 30, "bytes": 6e11, "flops": 6e11},
    }
    roof, table = bench.pick_roofline(prof, 5000.0, 1.0, 1700.0 / 36, "tensor")
    assert roof["kernel"] == "gje_update_H" and roof["bound"] == "tensor"
    assert roof["achieved"] == pytest.approx(10.0) and roof["peak"] == pytest.approx(1700.0 / 36)
    assert table["whiten_qt_dot"]["bound"] == "hbm"
    roof, table = bench.pick_roofline(prof, 5000.0, 1.0, 1700.0 / 36, "fp64")
    assert roof["bound"] == "alu" and table["whiten_qt_dot"]["bound"] == "alu"
    prof["gje_update_H"]["ms"] = 100.0
    roof, _ = bench.pick_roofline(prof, 5000.0, 1.0, 1700.0 / 36, "tensor")
    assert roof["kernel"] == "whiten_qt_dot" and roof["bound"] == "hbm"
    assert roof["achieved"] == pytest.approx(2000.0) and roof["frac"] == pytest.approx(0.4)


def test_fp64_alu_peak_from_units_and_clock(bench):
    peak, mhz = bench.fp64_alu_peak(152)
    assert peak == pytest.approx(152 * 2 * 2 * mhz * 1e6 / 1e12)
    assert mhz > 1000.0


def test_clock_record_parsing(bench):
    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.proc = FakeProc()
    cs.lines = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.1, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = cs.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_replica_throughput_is_whole_job(bench):
    # 4 replicas, 3 solves each, slowest rank 6 s -> 2 solves/s for the job
    assert bench.replica_throughput(4, 3, 6000.0) == pytest.approx(2.0)
