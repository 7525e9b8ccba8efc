"""Host-side logic of bench.py that needs no GPU: the clock summary taken from
nvidia-smi's CSV lines and the workload descriptions."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_median_max_and_reasons(bench):
    lines = [
        "0, 2070, 2070, 850.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2002, 2070, 1388.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = bench.summarize_clocks(lines)
    assert s["sm_mhz"] == 2002.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_empty_input(bench):
    hot = ["0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Not Active"]
    assert bench.summarize_clocks(hot)["reasons"] == ["hw_thermal_slowdown"]
    empty = bench.summarize_clocks([])
    assert empty["sm_mhz"] is None and empty["samples"] == 0 and empty["reasons"] == []


def test_workload_table_names_the_benchmark_shapes(bench):
    assert {"h50", "fe2s2", "h18"} <= set(bench.WORKLOADS)
    n_default = bench.WORKLOADS["h50"][1]
    assert n_default == 4096
