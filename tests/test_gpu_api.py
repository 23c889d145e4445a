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
