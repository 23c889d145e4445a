"""Host-side contract of bench.py on the CPU: the reference arm (the FP64 oracle
timed on a bounded sample) prints one JSON line with the fields the driver
reads, and the speed-limit profile helper gives per-cell factors in (0, 1]."""
import argparse
import contextlib
import io
import json

import numpy as np

import bench


def test_v0_profile_shape_and_range():
    assert bench.v0_profile("none", 4096) is None
    lam = bench.v0_profile("sine", 4096)
    assert lam.dtype == np.float32 and lam.shape == (4096,)
    assert 0.5 < lam.min() < 0.501 and 0.999 < lam.max() <= 1.0
    assert np.allclose(lam, lam[::-1])  # symmetric about the centre
    assert "varying in space" in bench.workload_config(1, "sine")["workload"]
    assert "varying in space" not in bench.workload_config(1)["workload"]


def test_reference_arm_prints_the_contract_line(monkeypatch):
    monkeypatch.setenv("RANK", "0")
    args = argparse.Namespace(steps=3, warmup=3, gpus=1, v0_profile="none")
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        assert bench.run_reference(args) == 0
    line = json.loads(out.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["steps"] == 3 and line["warmup"] == 3 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"] == bench.workload_config(1)


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=3, warmup=3, gpus=2, v0_profile="none")
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        assert bench.run_reference(args) == 0
    assert out.getvalue() == ""


def test_oracle_on_all_cores_sums_independent_copies():
    from paper_1511_08225_gb300 import inputs
    prob = inputs.sheath_problem(n_cells=64, ppc=50, v0=0.05)
    state = inputs.load_state(prob)
    rate, workers, per = bench.oracle_rate_all_cores(prob, state, 3.0, per_worker=2000,
                                                     workers=2)
    assert workers == 2 and per == 1.5 and rate > 0
    one, _, _, _ = bench.oracle_rate(prob, state, 1.5, max_particles=2000)
    assert 0.8 * one < rate < 3.0 * one  # two cores, not a fluke
