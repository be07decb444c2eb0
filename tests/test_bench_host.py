"""Host-side logic of bench.py that the reported numbers rest on (no GPU):

* the clock sampler's reading of nvidia-smi's CSV (median SM clock under
  load, the highest maximum clock, and which throttle reasons were active:
  a run that saw hw_slowdown or a thermal slowdown must say so);
* the roofline record: achieved = model flops (or bytes) per launch over the
  event-timed launch, frac = achieved / peak, the bound taken from whichever
  ceiling the launch's own model puts first;
* the whole-step record against both ceilings.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

PK = {"hbm_gbs": 6000.0, "fp64_tflops": 1.0, "fp32_tflops": 64.0, "src": "measured",
      "fp64_src": "probe", "fp32_src": "probe"}


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def sampled(lines):
    c = bench.ClockSampler(0)
    c.f.write("".join(x + "\n" for x in lines))
    c.f.flush()
    c.proc = _Done()
    return c.stop()


def test_clock_sampler_reads_clocks_and_reasons():
    row = "0, {sm}, 2070, 900.5, 0x0, {hw}, Not Active, Not Active, {cap}"
    r = sampled([row.format(sm=2070, hw="Not Active", cap="Not Active"),
                 row.format(sm=1995, hw="Active", cap="Not Active"),
                 row.format(sm=2055, hw="Not Active", cap="Active"),
                 "0, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
                 "garbage"])
    assert r["samples"] == 4
    assert r["sm_mhz"] == 2055.0          # median of 2070, 1995, 2055
    assert r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_sampler_quiet_run_and_no_samples():
    r = sampled(["0, 2070, 2070, 700, 0x0, Not Active, Not Active, Not Active, Not Active"] * 3)
    assert r["reasons"] == [] and r["sm_mhz"] == 2070.0
    assert sampled([]) is None


def test_roofline_of_one_launch_per_step_is_the_whole_step():
    # two phases of the step model, cells per step as the eager profile counts
    prof = {"mom_jacobi": {"ms": 0.3, "launches": 3, "cells": 3 * 1000},
            "H": {"ms": 0.1, "launches": 1, "cells": 1000}}
    words = bench.KERNEL_MODEL["mom_jacobi"][0] * 3000 + bench.KERNEL_MODEL["H"][0] * 1000
    flops = bench.KERNEL_MODEL["mom_jacobi"][1] * 3000 + bench.KERNEL_MODEL["H"][1] * 1000
    r = bench.roofline(prof, PK, 0.5, True, "none")
    assert r["launches_per_step"] == 1 and r["avg_launch_ms"] == 0.5
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(8.0 * words)
    assert r["algorithmic_flops_per_launch"] == pytest.approx(flops)
    t = 0.5e-3
    # FP64 time flops / 1 TF against bytes / 6000 GB/s: this model is FP64-bound
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops / t / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / PK["fp64_tflops"])
    assert r["phase_share_of_eager_step"] == {"mom_jacobi": 0.75, "H": 0.25}


def test_roofline_of_the_dominant_kernel_and_its_bound():
    prof = {"mom_jacobi": {"ms": 0.4, "launches": 4, "cells": 4 * 10 ** 6},
            "H": {"ms": 0.1, "launches": 1, "cells": 10 ** 6}}
    words, flops, _ = bench.KERNEL_MODEL["mom_jacobi"]
    r = bench.roofline(prof, PK, 2.0, False, "none")
    assert r["kernel"] == "mom_jacobi" and r["launches_per_step"] == 4
    t = 0.1e-3
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(words * 8 * 10 ** 6)
    assert r["achieved"] == pytest.approx(flops * 10 ** 6 / t / 1e12)
    # an HBM-heavy machine turns the same launch HBM-bound
    slow_hbm = dict(PK, hbm_gbs=100.0)
    r = bench.roofline(prof, slow_hbm, 2.0, False, "none")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(words * 8 * 10 ** 6 / t / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 100.0)


def test_whole_step_against_both_ceilings():
    prof = {"cg_pspmv": {"ms": 1.0, "launches": 10, "cells": 10 * 10 ** 6}}
    words, flops, _ = bench.KERNEL_MODEL["cg_pspmv"]
    w = bench.whole_step(prof, PK, 2.0)
    t = 2.0e-3
    t_alu = flops * 1e7 / 1e12
    t_hbm = words * 8 * 1e7 / (6000.0 * 1e9)
    assert w["frac_fp64"] == pytest.approx(flops * 1e7 / t / 1e12)
    assert w["frac_hbm"] == pytest.approx(words * 8 * 1e7 / t / 6000e9)
    assert w["bound"] == ("alu" if t_alu >= t_hbm else "hbm")
    assert w["frac_binding"] == pytest.approx(max(t_alu, t_hbm) / t)
    assert w["ms_at_binding_roofline"] == pytest.approx(max(t_alu, t_hbm) * 1e3)


def test_job_rate_of_one_rank():
    rate, t = bench.job_rate(2.0, 10 ** 6, 1)
    assert t == 2.0 and rate == 5e5
