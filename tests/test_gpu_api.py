"""Entry points that change how results are read, not what they are."""
import numpy as np
import pytest

from paper_1511_08225_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def test_fields_async_gives_the_fields_of_each_step():
    """Steps and asynchronous read-backs queued back to back, one synchronisation at
    the end: every step's buffers hold what slpic_fields gives for that step."""
    prob = inputs.sheath_problem(n_cells=256, ppc=100, v0=0.05)
    st = inputs.load_state(prob)
    a, b = binding.Simulation(prob), binding.Simulation(prob)
    for sim in (a, b):
        sim.load_state(st)
        sim.prepare()
    nn = prob["n_cells"] + 1
    L = binding.load_library()
    bufs = []
    for _ in range(5):
        a.step(3)
        rho, phi, E = np.zeros(nn), np.zeros(nn), np.zeros(nn, np.float32)
        assert L.slpic_fields_async(a.h, 0, binding._ptr(rho), binding._ptr(phi),
                                    binding._ptr(E)) == 0
        bufs.append((rho, phi, E))
    a.synchronize()
    for rho, phi, E in bufs:
        b.step(3)
        r2, p2, e2 = b.fields()
        assert np.array_equal(rho, r2) and np.array_equal(phi, p2) and np.array_equal(E, e2)
    a.close()
    b.close()


def test_fields_async_on_a_batch_instance():
    probs = inputs.batch_problems(m=3, seed=9, cells=(64, 300), ppc=(20, 40))
    b = binding.Batch(probs)
    for i, p in enumerate(probs):
        b.load_state(i, inputs.load_state(p))
    b.prepare()
    b.step(5)
    L = binding.load_library()
    got = []
    for i, p in enumerate(probs):
        nn = p["n_cells"] + 1
        rho, phi, E = np.zeros(nn), np.zeros(nn), np.zeros(nn, np.float32)
        assert L.slpic_fields_async(b.h, i, binding._ptr(rho), binding._ptr(phi),
                                    binding._ptr(E)) == 0
        got.append((rho, phi, E))
    b.synchronize()
    for i in range(len(probs)):
        r2, p2, e2 = b.fields(i)
        assert np.array_equal(got[i][0], r2) and np.array_equal(got[i][1], p2)
        assert np.array_equal(got[i][2], e2)
    b.close()
