"""The learned initial guess of the 2D field solve: (rho, phi) pairs from the 2D
runs themselves, training of the U-Net on them, and the conversions between the
solver's nodal arrays and the network's images.

Host-side orchestration only: the simulation steps, the CG solves, the network's
forward and backward passes and the Adam steps all run in libslpic.so.

Images: the network sees rows 0..ny-1 of the (ny+1, nx) nodal grid, as an
(H, W) = (ny, nx) FP32 image.  Input: rho with row 0 (a plate) set to zero.
Target: phi minus the straight line between the plate potentials (zero on both
plates), so the network learns the linear zero-plate problem.
"""
from __future__ import annotations

import numpy as np

from . import binding2d, inputs


def rho_image(rho: np.ndarray) -> np.ndarray:
    x = np.array(rho[:-1], dtype=np.float32)
    x[0] = 0.0
    return x


def plate_line(ny: int, nx: int, phi_lo: float, phi_hi: float) -> np.ndarray:
    j = np.arange(ny + 1, dtype=np.float64)[:, None]
    return np.broadcast_to(phi_lo + (phi_hi - phi_lo) * j / ny, (ny + 1, nx))


def phi_image(phi: np.ndarray, phi_lo: float = 0.0, phi_hi: float = 0.0) -> np.ndarray:
    ny, nx = phi.shape[0] - 1, phi.shape[1]
    return np.array((phi - plate_line(ny, nx, phi_lo, phi_hi))[:-1], dtype=np.float32)


def guess_from_image(y: np.ndarray, phi_lo: float = 0.0, phi_hi: float = 0.0) -> np.ndarray:
    """The solver's initial guess: the plate line plus the image on rows 1..ny-1."""
    ny, nx = y.shape[0], y.shape[1]
    g = np.array(plate_line(ny, nx, phi_lo, phi_hi))
    g[1:ny] += y[1:ny]
    return g


def collect_pairs(prob: dict, seeds, pairs_per_seed: int, every: int, skip: int,
                  keep_prev: bool = False):
    """Run the 2D problem from each seed's load, skip `skip` steps, then take a
    (rho, phi) pair every `every` steps.  Returns a dict of numpy arrays:
    rho, phi (N, ny+1, nx) FP64 and, with keep_prev, rho_prev and phi_prev, those
    of the step before each pair (phi_prev is the previous-step guess)."""
    rho, phi, prev, rprev = [], [], [], []
    for seed in seeds:
        p = dict(prob, seed=int(seed))
        sim = binding2d.Simulation2D(p)
        sim.load_state(inputs.load_state2d(p, seed=int(seed)))
        sim.prepare()
        sim.step(skip)
        for _ in range(pairs_per_seed):
            if every > 1:
                sim.step(every - 1)
            if keep_prev:
                r0, f0, _, _ = sim.fields()
                rprev.append(r0)
                prev.append(f0)
            sim.step(1)
            r, f, _, _ = sim.fields()
            rho.append(r)
            phi.append(f)
        sim.close()
    out = {"rho": np.stack(rho), "phi": np.stack(phi)}
    if keep_prev:
        out["phi_prev"] = np.stack(prev)
        out["rho_prev"] = np.stack(rprev)
    return out


def collect_delta_images(prob: dict, seed: int, n_pairs: int, every: int, skip: int):
    """delta_images of collect_pairs(prob, (seed,), n_pairs, every, skip,
    keep_prev=True), made pair by pair into float32 device tensors (N, ny, nx), so
    that a large set (10k pairs of a 1024 x 1024 grid: 80 GB) never sits in host
    memory.  Returns (x, t)."""
    import torch

    ny, nx = int(prob["ny"]), int(prob["nx"])
    x = torch.empty((n_pairs, ny, nx), dtype=torch.float32, device="cuda")
    t = torch.empty_like(x)
    p = dict(prob, seed=int(seed))
    sim = binding2d.Simulation2D(p)
    sim.load_state(inputs.load_state2d(p, seed=int(seed)))
    sim.prepare()
    sim.step(skip)
    for i in range(n_pairs):
        if every > 1:
            sim.step(every - 1)
        r0, f0, _, _ = sim.fields()
        sim.step(1)
        r, f, _, _ = sim.fields()
        x[i].copy_(torch.from_numpy(rho_image(r - r0)))
        t[i].copy_(torch.from_numpy(phi_image(f - f0)))
    sim.close()
    return x, t


def images(pairs: dict, phi_lo: float = 0.0, phi_hi: float = 0.0):
    """(x, t): the network's input and target images, (N, ny, nx) FP32."""
    x = np.stack([rho_image(r) for r in pairs["rho"]])
    t = np.stack([phi_image(f, phi_lo, phi_hi) for f in pairs["phi"]])
    return x, t


def delta_images(pairs: dict):
    """(x, t) for the change between consecutive steps (pairs collected with
    keep_prev): x = image(rho - rho_prev), t = image(phi - phi_prev) (the plate
    potentials cancel)."""
    x = np.stack([rho_image(a - b) for a, b in zip(pairs["rho"], pairs["rho_prev"])])
    t = np.stack([phi_image(a - b) for a, b in zip(pairs["phi"], pairs["phi_prev"])])
    return x, t


def output_scale(x: np.ndarray, t: np.ndarray) -> float:
    """The median over the pairs of rms(target) / rms(input): the network's
    out_scale, so that its normalised targets are of order one."""
    rx = np.sqrt((x.astype(np.float64) ** 2).mean(axis=(1, 2)))
    rt = np.sqrt((t.astype(np.float64) ** 2).mean(axis=(1, 2)))
    ok = rx > 0
    return float(np.median(rt[ok] / rx[ok]))


def fit(net, x, t, steps: int, batch: int, lr: float, seed: int = 0, lr_final: float | None = None,
        log_every: int = 0):
    """Adam on random mini-batches of the device tensors x, t (N, H, W); the
    learning rate falls geometrically from lr to lr_final (default lr / 10).
    Returns the losses taken every log_every steps (and at the last)."""
    import torch

    g = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0]
    lr_final = lr / 10 if lr_final is None else lr_final
    losses = []
    for k in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).to(x.device)
        xb = x.index_select(0, idx).contiguous()
        tb = t.index_select(0, idx).contiguous()
        rate = lr * (lr_final / lr) ** (k / max(steps - 1, 1))
        want = (log_every and k % log_every == 0) or k == steps - 1
        loss = net.train_step(xb, tb, rate, want_loss=bool(want))
        if want:
            losses.append((k, loss))
    return losses
