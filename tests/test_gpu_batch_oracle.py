"""Batches of independent sheaths (slpic_create_batch) against the FP64 oracle.

Each instance of a batch is held to the bars of a single simulation:
  * its deposit is the quantised rule (slpic_charge_raw) on its own particles,
    bit for bit, after the load and after steps that include a compacting step,
    source injection and absorption;
  * one step from a strongly non-neutral start, source off, matches the oracle's
    push of that instance particle by particle, the oracle pushing in the instance's
    own field (its FP32 nodal E, the field the GPU gathers; the field itself is held to
    the oracle's solve of the same integer charge by the single-simulation tests):
    |dv| <= 1e-5 |v| plus the FP32 rounding of the gather (4 2^-24 of the two nodal
    fields, times |q/m| dt), and the position within the displacement that velocity
    error causes plus 8 ulp of the offset.  (Against the oracle's own FP64 field the
    kick also carries the field's ~1e-7 relative difference, which comes from the
    FP32 speed limit and beta of the quantised deposit; where the field crosses zero
    under a slow particle that difference alone reaches 2e-5 of |v|.)
Batches: 40 instances of 256..2,048 cells, 20..120 particles per cell, m_i/m_e of
1,836 or 73,440 and v0 log-uniform in 0.01..0.5 v_te (dt = dx / v0); and the
benchmark's 256 instances (512..8,192 cells, the same masses and limits) at a
tenth of its particles per cell, all 256 deposits checked and one step of 16 of
them against the oracle.  Inputs are generated in a spawn-started process pool."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1511_08225_gb300 import binding, inputs

from _stepcheck import compare_step

pytestmark = pytest.mark.gpu


def _gen(prob):
    from paper_1511_08225_gb300 import inputs as inp
    return inp.load_state(prob)


def _nonneutral(args):
    """Strong fields: electrons only in the left half, Gaussian velocities."""
    prob, seed = args
    from paper_1511_08225_gb300 import inputs as inp
    rng = inp.make_rng(seed)
    N = prob["n_cells"]
    out = []
    for s, sp in enumerate(prob["species"]):
        n = int(sp["ppc"]) * N // 4
        c, o = inp.uniform_cells(rng, n, N, 0.0, N / 2 if s == 0 else N)
        v = rng.normal(0.0, sp["vth"], (n, 3)).astype(np.float32)
        out.append((c, o, v))
    return out


def _pool_map(f, jobs):
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(f, jobs, chunksize=1)


def _check_deposits(b, probs, which):
    for i in which:
        for s, sp in enumerate(probs[i]["species"]):
            c, o, v = b.particles(i, s)
            q = orc.deposit_q40(probs[i]["n_cells"], False, c, o, v, sp["kind"],
                                np.float32(sp["v0"]))
            assert np.array_equal(b.charge_raw(i, s), q), (i, s)


def _batch(probs, states):
    b = binding.Batch(probs)
    for i, st in enumerate(states):
        b.load_state(i, st)
    b.prepare()
    return b


def _one_step_against_oracle(probs, states, which):
    b = _batch(probs, states)
    E0 = {i: b.fields(i)[2] for i in which}
    b.step(1)
    b.synchronize()

    class _Inst:  # one instance seen through the single-simulation interface
        def __init__(self, i):
            self.i = i

        def particles(self, s):
            return b.particles(self.i, s)

    for i in which:
        o = orc.OracleSim(probs[i])
        for s, (c, off, v) in enumerate(states[i]):
            o.load_cells(s, c, off, v)
        o.start()
        o.E = E0[i].astype(np.float64)  # push in the instance's own field
        o.step(1)
        compare_step(probs[i], states[i], _Inst(i), o, E=E0[i].astype(np.float64))
    b.close()


def test_batch_of_40_deposits_and_one_step_match_oracle():
    probs = inputs.batch_problems(m=40, seed=77, cells=(256, 2048), ppc=(20, 120))
    states = _pool_map(_gen, probs)
    b = _batch(probs, states)
    _check_deposits(b, probs, range(len(probs)))
    b.step(20)  # a compacting step, the source and the walls
    b.synchronize()
    _check_deposits(b, probs, range(len(probs)))
    assert all(b.diagnostics(i)["injected"][1] > 0 for i in range(len(probs)))
    b.close()
    quiet = [dict(p, source=dict(p["source"], mode=inputs.SRC_NONE)) for p in probs]
    nn_states = _pool_map(_nonneutral, [(p, 100 + i) for i, p in enumerate(quiet)])
    _one_step_against_oracle(quiet, nn_states, range(len(quiet)))


def test_benchmark_batch_of_256_at_a_tenth_of_its_particles():
    probs = inputs.batch_problems(m=256, ppc=(10, 100))
    states = _pool_map(_gen, probs)
    b = _batch(probs, states)
    b.step(17)
    b.synchronize()
    _check_deposits(b, probs, range(len(probs)))
    b.close()
    pick = list(range(0, 256, 16))
    quiet = [dict(p, source=dict(p["source"], mode=inputs.SRC_NONE)) for p in probs]
    nn_states = _pool_map(_nonneutral, [(quiet[i], 500 + i) for i in range(256)])
    _one_step_against_oracle(quiet, nn_states, pick)
