"""Performance settings and the autotuner (slpic_set_tuning / slpic_autotune):
whatever the compaction interval, the in-place particle kernel or a batch's work
split, the same steps give bit for bit the same particles (as a set), deposits,
fields and diagnostics, because the source draws its random numbers by (seed,
step, species, particle index) and the deposit is an integer sum."""
import numpy as np
import pytest

from paper_1511_08225_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _sorted(c, o, v):
    key = np.lexsort((v[:, 2], v[:, 1], v[:, 0], o, c))
    return c[key], o[key], v[key]


def _same(a, b, species=2):
    """a, b: objects with diagnostics(), fields(), charge_raw(s), particles(s)."""
    da, db = a.diagnostics(), b.diagnostics()
    for k in ("step", "count", "absorbed", "injected", "iterative"):
        assert da[k] == db[k], k
    ra, pa, ea = a.fields()
    rb, pb, eb = b.fields()
    assert np.array_equal(pa, pb) and np.array_equal(ea, eb) and np.array_equal(ra, rb)
    for s in range(species):
        assert np.array_equal(a.charge_raw(s), b.charge_raw(s))
        for x, y in zip(_sorted(*a.particles(s)), _sorted(*b.particles(s))):
            assert np.array_equal(x, y)


class _Inst:
    """One instance of a batch seen as a simulation."""

    def __init__(self, b, i):
        self.b, self.i = b, i

    def diagnostics(self):
        return self.b.diagnostics(self.i)

    def fields(self):
        return self.b.fields(self.i)

    def charge_raw(self, s):
        return self.b.charge_raw(self.i, s)

    def particles(self, s):
        return self.b.particles(self.i, s)


def _sheath():
    return inputs.sheath_problem(n_cells=512, ppc=200, v0=0.05, capacity_factor=2.0)


@pytest.mark.parametrize("settings", [dict(compact_every=4), dict(compact_every=37),
                                      dict(particle_kernel=1), dict(compact_every=64, particle_kernel=1)])
def test_every_setting_gives_the_same_run(settings):
    prob = _sheath()
    st = inputs.load_state(prob)
    ref, alt = binding.Simulation(prob), binding.Simulation(prob)
    for sim in (ref, alt):
        sim.load_state(st)
        sim.prepare()
    binding.slpic_set_tuning(alt.h, **settings)
    got = binding.slpic_get_tuning(alt.h)
    for k, v in settings.items():
        assert got[k] == v
    for n in (5, 40, 81):
        ref.step(n)
        alt.step(n)
        _same(ref, alt)
    # changed again mid-run
    binding.slpic_set_tuning(alt.h, compact_every=16, particle_kernel=0)
    ref.step(33)
    alt.step(33)
    _same(ref, alt)
    ref.close()
    alt.close()


def test_autotune_keeps_the_run_and_picks_a_listed_setting():
    prob = _sheath()
    st = inputs.load_state(prob)
    ref, tuned = binding.Simulation(prob), binding.Simulation(prob)
    for sim in (ref, tuned):
        sim.load_state(st)
        sim.prepare()
    tuned.step(20)
    chosen, ms = binding.slpic_autotune(tuned.h, steps_per_trial=32)
    assert chosen == binding.slpic_get_tuning(tuned.h)
    assert chosen["compact_every"] in (8, 16, 32, 64) and chosen["particle_kernel"] in (0, 1)
    assert ms > 0
    n = tuned.diagnostics()["step"]
    ref.step(n)
    _same(ref, tuned)
    ref.step(50)
    tuned.step(50)
    _same(ref, tuned)
    ref.close()
    tuned.close()


def test_batch_work_split_and_autotune_keep_every_instance():
    probs = inputs.batch_problems(m=4, seed=5, cells=(64, 600), ppc=(20, 60))
    states = [inputs.load_state(p) for p in probs]
    ref, alt = binding.Batch(probs), binding.Batch(probs)
    for b in (ref, alt):
        for i, st in enumerate(states):
            b.load_state(i, st)
        b.prepare()
    binding.slpic_set_tuning(alt.h, batch_waves=1, batch_min_share=1024, compact_every=8)
    ref.step(45)
    alt.step(45)
    for i in range(len(probs)):
        _same(_Inst(ref, i), _Inst(alt, i))
    chosen, _ = binding.slpic_autotune(alt.h, steps_per_trial=16)
    assert chosen["batch_waves"] in (1, 2, 4, 8)
    ref.step(alt.diagnostics(0)["step"] - ref.diagnostics(0)["step"])
    for i in range(len(probs)):
        _same(_Inst(ref, i), _Inst(alt, i))
    ref.close()
    alt.close()


def test_tuning_rejects_out_of_range_values():
    sim = binding.Simulation(_sheath())
    for bad in (dict(compact_every=1), dict(compact_every=2000), dict(particle_kernel=2),
                dict(batch_waves=0), dict(batch_min_share=100)):
        with pytest.raises(binding.SlpicError) as ei:
            binding.slpic_set_tuning(sim.h, **bad)
        assert ei.value.code == binding.SLPIC_ERR_INVALID
    with pytest.raises(binding.SlpicError):
        binding.slpic_autotune(sim.h, steps_per_trial=0)
    sim.close()
