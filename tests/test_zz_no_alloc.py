"""The allocation-free particle step, through the C ABI, against the handle path.

slpic_particle_step_noalloc is for callers that may not allocate device memory
(a framework that owns the device's memory pool, a service that reserves all
memory at start-up, a loop that cannot afford cudaMalloc's synchronisation).
It keeps its scratch in a fixed device array shared by all calls, so this test
calls it twice in a row and checks that each call's output equals what the
simulation handle (slpic_step, which allocates its own scratch) computes for
the same particles and field: the deposit bit for bit (the bar of the deposit
parity tests) and the surviving particles bit for bit.  The deposit is also held,
bit for bit, to the oracle's quantised deposit rule applied to the survivors the
call returns, so the check does not rest on the handle path alone.

This file is collected last on purpose, and passes both alone in a fresh
process and after the other tests.
"""
import numpy as np
import pytest

from oracle import oracle as orc
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
            sp = prob["species"][s]
            acc_orc = orc.deposit_q40(N, periodic, c2, st2[:, 0], st2[:, 1:], sp["kind"],
                                      np.float32(sp["v0"]))
            assert np.array_equal(charge.cpu().numpy(), acc_orc), f"call {call} species {s}"
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


def test_noalloc_rejects_overlapping_arrays(torch_cuda):
    """Survivors are packed across thread blocks, so outputs that overlap the inputs
    could overwrite unread particles: the call refuses them before any work."""
    torch = torch_cuda
    prob = _problem(False, 1, 96)
    cfg = binding.config_from_problem(prob)
    dev = torch.device("cuda")
    n = 1000
    cells = torch.zeros(2 * n, dtype=torch.int32, device=dev)
    states = torch.zeros((2 * n, 4), dtype=torch.float32, device=dev)
    E = torch.zeros(97, device=dev)
    charge = torch.zeros(97, dtype=torch.int64, device=dev)
    for cin, sin, cout, sout in ((cells[:n], states[:n], cells[:n], states[n:]),
                                 (cells[:n], states[:n], cells[n:], states[n // 2:n // 2 + n])):
        with pytest.raises(binding.SlpicError) as ei:
            binding.slpic_particle_step_noalloc(cfg, 0, cin, sin, E, cout, sout, charge)
        assert ei.value.code == binding.SLPIC_ERR_INVALID


def test_noalloc_skips_and_reports_particles_outside_the_grid(torch_cuda):
    """A cell outside [0, n_cells) or an offset outside [0, 1) would index the
    kernel's shared-memory grid out of range: such particles are skipped, the others
    stepped, and the call reports SLPIC_ERR_INVALID.  The deposit is then that of the
    valid particles alone."""
    torch = torch_cuda
    N = 96
    prob = _problem(False, 1, N)
    cfg = binding.config_from_problem(prob)
    dev = torch.device("cuda")
    (c, o, v), _ = _state(N, (5000, 1), seed=9)
    c = c.copy()
    o = o.copy()
    c[0::291] = -5      # below the grid
    c[97::291] = N + 3  # beyond it
    o[194::291] = 1.5   # offset outside [0, 1)
    bad = (c < 0) | (c >= N) | (o >= 1.0)
    assert bad.sum() > 10
    st = np.concatenate([o[:, None], v], axis=1).astype(np.float32)
    E = torch.tensor(np.linspace(-0.5, 0.5, N + 1, dtype=np.float32), device=dev)

    def run(cc, ss):
        cin = torch.tensor(cc, device=dev)
        sin = torch.tensor(ss, device=dev)
        cout = torch.empty_like(cin)
        sout = torch.empty_like(sin)
        charge = torch.zeros(N + 1, dtype=torch.int64, device=dev)
        return cin, sin, cout, sout, charge

    cin, sin, cout, sout, charge = run(c, st)
    with pytest.raises(binding.SlpicError) as ei:
        binding.slpic_particle_step_noalloc(cfg, 0, cin, sin, E, cout, sout, charge)
    assert ei.value.code == binding.SLPIC_ERR_INVALID
    got = charge.cpu().numpy()
    cin2, sin2, cout2, sout2, charge2 = run(c[~bad], st[~bad])
    n_out, _ = binding.slpic_particle_step_noalloc(cfg, 0, cin2, sin2, E, cout2, sout2, charge2)
    assert n_out > 0
    assert np.array_equal(got, charge2.cpu().numpy())
