"""Failure detection without a GPU fault: a bounded device-side wait that runs out.

The particle kernel's pipeline waits (a tile's bulk copy landing in its shared-memory
ring, the consumer warps freeing a stage) give up after a limit of SM clock cycles
(slpic_set_wait_limit).  Set far below a copy's latency (200 cycles), the first wait
of every CTA runs out: the kernel records SLPIC_ERR_TIMEOUT, waits for its own copies
still in flight and returns.  slpic_synchronize reports the error, the CUDA context
stays usable, reading the cut-short handle back is safe, and a fresh handle then
steps normally: its deposit is the quantised rule on its own particles."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1511_08225_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _sim(prob):
    sim = binding.Simulation(prob)
    sim.load_state(inputs.load_state(prob))
    sim.prepare()
    return sim


def test_wait_that_runs_out_is_reported_and_the_context_survives():
    prob = inputs.sheath_problem(n_cells=512, ppc=200, v0=0.05)
    sim = _sim(prob)
    assert binding.slpic_get_tuning(sim.h)["particle_kernel"] == 0  # the TMA-staged kernel
    sim.step(2)
    sim.synchronize()
    binding.slpic_set_wait_limit(sim.h, 200)
    sim.step(3)
    with pytest.raises(binding.SlpicError) as err:
        sim.synchronize()
    assert err.value.code == binding.SLPIC_ERR_TIMEOUT
    # the error was reported once; the handle can still be read back safely
    sim.synchronize()
    for s in range(2):
        c, o, v = sim.particles(s)
        assert ((c >= 0) & (c < prob["n_cells"])).all()
    sim.fields()
    with pytest.raises(binding.SlpicError):
        binding.slpic_set_wait_limit(sim.h, -1)
    sim.close()
    # the context is usable: a torch kernel and a fresh handle at the default limit
    x = torch.arange(1000, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 499500.0
    sim2 = _sim(prob)
    sim2.step(3)
    sim2.synchronize()
    for s, sp in enumerate(prob["species"]):
        c, o, v = sim2.particles(s)
        q = orc.deposit_q40(prob["n_cells"], False, c, o, v, sp["kind"], np.float32(sp["v0"]))
        assert np.array_equal(sim2.charge_raw(s), q)
    sim2.close()


def test_default_limit_restored_steps_like_a_fresh_handle():
    prob = inputs.sheath_problem(n_cells=512, ppc=100, v0=0.05)
    a, b = _sim(prob), _sim(prob)
    binding.slpic_set_wait_limit(b.h, 10_000_000)
    binding.slpic_set_wait_limit(b.h, 0)
    a.step(20)
    b.step(20)
    for s in range(2):
        assert np.array_equal(a.charge_raw(s), b.charge_raw(s))
    assert a.diagnostics()["count"] == b.diagnostics()["count"]
    a.close()
    b.close()
