"""The allocation-free particle step, through the C ABI, against the handle path.

slpic_particle_step_noalloc is for callers that may not allocate device memory
(a framework that owns the device's memory pool, a service that reserves all
memory at start-up, a loop that cannot afford cudaMalloc's synchronisation).
It keeps its scratch in a fixed device array shared by all calls, so this test
calls it twice in a row and checks that each call's output equals what the
simulation handle (slpic_step, which allocates its own scratch) computes for
the same particles and field: the deposit bit for bit (the bar of the deposit
parity tests) and the surviving particles bit for bit.

This file is collected last on purpose, and passes both alone in a fresh
process and after the other tests.
"""
import numpy as np
import pytest

from paper_1511_08225_gb300 import binding, inputs

from _match import key_of, match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_08225_gb300 import build
    build.build()
    binding.load_library()
    return torch


def _problem(periodic, kind, N):
    v0 = 0.3
    sps = [{"name": "e", "q": -1.0, "m": 1.0, "w": 1e-3, "v0": v0, "kind": kind, "T": 0.0,
            "capacity": 1 << 18},
           {"name": "i", "q": 1.0, "m": 80.0, "w": 2e-3, "v0": v0, "kind": kind, "T": 0.0,
            "capacity": 1 << 18}]
    return {"n_cells": N, "dx": 0.5, "dt": 0.5 / v0, "periodic": periodic, "phi_lo": 0.0,
            "phi_hi": 0.0 if periodic else 2.0, "eps0": 1.0, "seed": 3, "species": sps,
            "source": {"mode": binding.SLPIC_SRC_NONE}}


def _state(N, n_per, seed):
    rng = inputs.make_rng(seed)
    out = []
    for s, n in enumerate(n_per):
        cell, off = inputs.uniform_cells(rng, n, N, 0.0, N / 2 if s == 0 else N)
        v = rng.normal(0.0, 1.0 / np.sqrt(1.0 if s == 0 else 80.0), (n, 3)).astype(np.float32)
        out.append((cell, off, v))
    return out


def _handle_reference(prob, state):
    """E^0 and, per species, the survivors and deposit of one handle step."""
    sim = binding.Simulation(prob)
    sim.load_state(state)
    sim.prepare()
    _, _, E0 = sim.fields()
    sim.step(1)
    sim.synchronize()
    out = [(sim.particles(s), sim.charge_raw(s), sim.count(s)) for s in range(len(state))]
    sim.close()
    return E0, out


@pytest.mark.parametrize("periodic,kind,N", [(False, 1, 96), (True, 2, 200)])
def test_noalloc_step_matches_handle_step_twice(torch_cuda, periodic, kind, N):
    torch = torch_cuda
    prob = _problem(periodic, kind, N)
    state = _state(N, (30_000, 20_001), seed=N + kind)
    E0, ref = _handle_reference(prob, state)
    cfg = binding.config_from_problem(prob)
    dev = torch.device("cuda")
    E = torch.from_numpy(E0).to(dev)
    for call in range(2):  # two calls in a row share the same scratch
        for s, (cell, off, v) in enumerate(state):
            n = cell.size
            cin = torch.from_numpy(cell).to(dev)
            sin = torch.from_numpy(np.concatenate([off[:, None], v], axis=1)
                                   .astype(np.float32)).to(dev).contiguous()
            cout = torch.zeros(n, dtype=torch.int32, device=dev)
            sout = torch.zeros((n, 4), dtype=torch.float32, device=dev)
            charge = torch.zeros(cfg.n_cells + (0 if periodic else 1), dtype=torch.int64,
                                 device=dev)
            n_out, absorbed = binding.slpic_particle_step_noalloc(cfg, s, cin, sin, E, cout,
                                                                  sout, charge)
            (cg, og, vg), acc_ref, cnt_ref = ref[s]
            assert n_out == cnt_ref
            assert n_out + sum(absorbed) == n
            assert np.array_equal(charge.cpu().numpy(), acc_ref), f"call {call} species {s}"
            c2 = cout[:n_out].cpu().numpy()
            st2 = sout[:n_out].cpu().numpy()
            ia, ib = match(key_of(st2[:, 1:]), key_of(vg))
            assert ia.size == n_out
            assert np.array_equal(c2[ia], cg[ib])
            assert np.array_equal(st2[ia, 0], og[ib])
            assert np.array_equal(st2[ia, 1:], vg[ib])


def test_noalloc_rejects_grids_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    prob = _problem(True, 1, 20_000)  # 20,000 nodes > 16,384
    cfg = binding.config_from_problem(prob)
    dev = torch.device("cuda")
    z = torch.zeros(4, dtype=torch.float32, device=dev)
    with pytest.raises(binding.SlpicError) as ei:
        binding.slpic_particle_step_noalloc(
            cfg, 0, torch.zeros(1, dtype=torch.int32, device=dev), torch.zeros((1, 4), device=dev),
            torch.zeros(20_000, device=dev), torch.zeros(1, dtype=torch.int32, device=dev),
            torch.zeros((1, 4), device=dev), torch.zeros(20_000, dtype=torch.int64, device=dev))
    assert ei.value.code == binding.SLPIC_ERR_CAPACITY
    del z
