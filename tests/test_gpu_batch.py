"""Batches of independent sheaths (slpic_create_batch): every instance of a
batch advanced by the batched kernels gives exactly what the same instance
gives alone (same particles bit for bit, same deposits, same fields), for
instances of different size, species mass, speed limit and step."""
import numpy as np
import pytest

from paper_1511_08225_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _small_batch(m=5, seed=3):
    return inputs.batch_problems(m=m, seed=seed, cells=(64, 700), ppc=(20, 60))


def _sorted(c, o, v):
    key = np.lexsort((v[:, 2], v[:, 1], v[:, 0], o, c))
    return c[key], o[key], v[key]


def test_batch_matches_single_instances_bitwise():
    probs = _small_batch()
    states = [inputs.load_state(p) for p in probs]
    b = binding.Batch(probs)
    for i, st in enumerate(states):
        b.load_state(i, st)
    b.prepare()
    singles = []
    for p, st in zip(probs, states):
        s = binding.Simulation(p)
        s.load_state(st)
        s.prepare()
        singles.append(s)
    for n in (1, 3, 16, 20):  # crosses compacting steps and whole cycles
        b.step(n)
        for s in singles:
            s.step(n)
        b.synchronize()
        for i, s in enumerate(singles):
            db, ds = b.diagnostics(i), s.diagnostics()
            assert db["step"] == ds["step"]
            assert db["count"] == ds["count"] and db["absorbed"] == ds["absorbed"]
            assert db["injected"] == ds["injected"]
            for sp in range(2):
                assert np.array_equal(b.charge_raw(i, sp), s.charge_raw(sp))
                cb, ob, vb = _sorted(*b.particles(i, sp))
                cs, os_, vs = _sorted(*s.particles(sp))
                assert np.array_equal(cb, cs) and np.array_equal(ob, os_)
                assert np.array_equal(vb, vs)
            rb, pb, eb = b.fields(i)
            rs, ps, es = s.fields()
            assert np.array_equal(pb, ps) and np.array_equal(eb, es)
    for s in singles:
        s.close()
    b.close()


def test_batch_rejects_bad_instance_and_whole_handle_calls():
    probs = _small_batch(m=2)
    b = binding.Batch(probs)
    with pytest.raises(binding.SlpicError) as ei:
        b.count(2, 0)
    assert ei.value.code == binding.SLPIC_ERR_INVALID
    with pytest.raises(binding.SlpicError):
        binding.slpic_save(b.h)
    b.close()


def test_batch_create_reports_failing_instance():
    probs = _small_batch(m=3)
    probs[1]["dt"] = 10 * probs[1]["dx"] / probs[1]["species"][0]["v0"]
    with pytest.raises(binding.SlpicError) as ei:
        binding.Batch(probs)
    assert ei.value.code == binding.SLPIC_ERR_CFL
    assert "instance 1" in str(ei.value)
