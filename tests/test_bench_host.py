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
    one, done, dt, nst = bench.oracle_rate(prob, state, budget_s=1.0, max_particles=2000)
    assert nst >= 1 and done > 0 and one > 0
    # the copies run the one-core run's step range, each on its own subsample
    rate, workers, slow = bench.oracle_rate_all_cores(prob, state, nst, per_worker=2000,
                                                      workers=2, timeout=120)
    assert workers == 2 and rate > 0 and slow > 0
    assert 0.8 * one < rate < 2.6 * one  # two cores, not a fluke


def test_oracle_rate_runs_exact_step_count():
    from paper_1511_08225_gb300 import inputs
    prob = inputs.sheath_problem(n_cells=64, ppc=20, v0=0.05)
    state = inputs.load_state(prob)
    _, done, _, nst = bench.oracle_rate(prob, state, n_steps=3, max_particles=500)
    assert nst == 3 and done > 0


def test_cpu_baseline_line_fields():
    from paper_1511_08225_gb300 import inputs
    prob = inputs.sheath_problem(n_cells=64, ppc=50, v0=0.05)
    state = inputs.load_state(prob)
    cpu = bench.cpu_baseline(prob, state, 1.0, per_worker=2000)
    assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["unit"] == bench.UNIT
    assert cpu["cores"] >= 1 and "steps 1.." in cpu["sample"]
    if cpu["cores"] > 1:
        assert cpu["single_core"]["cores"] == 1
        # independent copies cannot beat cores x the one-core rate (beyond the timing
        # noise of runs this short)
        assert cpu["value"] <= 1.5 * cpu["cores_x_single_core"]
