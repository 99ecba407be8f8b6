"""Host logic of bench.py that decides what a bench line reports: the clock and
throttle-reason summary taken from nvidia-smi samples, and the whole-job value."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def summary_of(tmp_path, lines):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    c.proc = object()   # as if nvidia-smi had run
    return c.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    s = summary_of(tmp_path, [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hw_slowdown(tmp_path):
    s = summary_of(tmp_path, [
        "0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active",
    ])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples(tmp_path):
    assert summary_of(tmp_path, ["nothing"])["reasons"] == ["no samples"]
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_replica_value_is_the_whole_job():
    assert bench.replica_value(262144, 1, 0.2) == 262144 / 0.2
    assert bench.replica_value(262144, 4, 0.2) == 4 * 262144 / 0.2


def test_sample_parity_against_the_oracle_sample():
    """The oracle's own sample read back as the 'GPU' result agrees exactly; planted
    differences (a lost certification, a real/non-real swap, a moved endpoint) are
    counted."""
    import numpy as np
    from paper_1104_5497_gb300 import inputs
    inst = inputs.workload_n4()
    P = 4 ** (inst.N - 1)
    r, n, cores, dt, sample = bench.oracle_sample_rate(inst, 64, collect=True)
    assert n == 64 and len(sample["path"]) == 64 and sample["z"].shape == (64, 2 * (inst.N - 1))
    cls = np.zeros(P, np.int32)
    z = np.zeros((P, 2 * (inst.N - 1)), complex)
    cls[sample["path"]] = sample["cls"]
    z[sample["path"]] = sample["z"]
    par = bench.sample_parity(sample, cls, z)
    assert par["class_mismatches"] == 0 and par["real_mismatches"] == 0 and par["max_rel_err"] == 0
    assert par["certified"] == int(np.isin(sample["cls"], [2, 3, 4, 5]).sum()) > 0
    cert = sample["path"][np.isin(sample["cls"], [2, 3])]
    real = sample["path"][sample["cls"] == 2]
    cls2, z2 = cls.copy(), z.copy()
    cls2[cert[0]] = 1                       # singular on the "GPU"
    z2[cert[-1], 0] += 1e-6
    if len(real):
        cls2[real[-1]] = 3                  # real -> non-real
    par = bench.sample_parity(sample, cls2, z2)
    assert par["class_mismatches"] == 1
    assert par["real_mismatches"] == (1 if len(real) else 0) + int(cert[0] in real)
    assert 1e-7 < par["max_rel_err"] < 1e-6
