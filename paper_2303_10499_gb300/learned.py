"""The learned pressure-correction network trained on the solver's own
pressure systems (an extension beyond the paper).

Samples are the initial residuals r0 = b - A p' of the first corrector's
pressure solve (Section 3, eq. p_prime_sd) and the operator A of the same
step (c, a_x, a_z), taken from a run of the FP64 solver. The network is
trained on crops of them with the energy loss of include/gea_net.h, whose
minimiser is the exact correction A^-1 r0 up to scale; attached to a
context, it gives each pressure solve its starting point (gea_attach_net).

Every arithmetic step runs in the library's kernels; this module moves
arrays between the C ABI calls (torch tensors serve as device memory only).
"""
from __future__ import annotations

import time
from typing import Dict, List

import numpy as np

from . import gea


def initial_params(seed: int) -> np.ndarray:
    """He-scaled normal weights (std sqrt(2 / fan-in)) and zero biases, in the
    parameter order of the network's layer table."""
    rng = np.random.default_rng(seed)
    parts = []
    for cin, cout, k, _, _, _ in gea.net_layout():
        fan = cin * k * k
        parts.append(rng.standard_normal(cout * k * k * cin) * np.sqrt(2.0 / fan))
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)


def collect(wl, steps: int, every: int = 1, const=None) -> List[Dict]:
    """Run the FP64 solver on workload wl for `steps` steps and keep, every
    `every` steps, r0 and the operator of that step as float32 CUDA tensors."""
    import torch
    const = const or wl.const
    s = gea.Solver(wl.grid, const, graph=True, keep_r0=True)
    s.set_conservative(wl.fields)
    out = []
    for k in range(steps):
        s.step(1)
        if (k + 1) % every == 0:
            out.append({n: torch.tensor(s.field(n), dtype=torch.float32, device="cuda")
                        for n in ("r0", "hc", "hax", "haz")})
    s.close()
    return out


def crops(samples: List[Dict], n: int, h: int, w: int, rng):
    """n random h x w crops (walls included) of random samples: r, c, a_x,
    a_z batches. Faces on a crop's edge are not used by the loss (the crop is
    treated as closed there)."""
    import torch
    r = torch.empty((n, h, w), dtype=torch.float32, device="cuda")
    c = torch.empty((n, h, w), dtype=torch.float32, device="cuda")
    ax = torch.empty((n, h, w + 1), dtype=torch.float32, device="cuda")
    az = torch.empty((n, h + 1, w), dtype=torch.float32, device="cuda")
    for b in range(n):
        smp = samples[int(rng.integers(len(samples)))]
        H, W = smp["r0"].shape
        y0 = int(rng.integers(0, H - h + 1))
        x0 = int(rng.integers(0, W - w + 1))
        r[b].copy_(smp["r0"][y0:y0 + h, x0:x0 + w])
        c[b].copy_(smp["hc"][y0:y0 + h, x0:x0 + w])
        ax[b].copy_(smp["hax"][y0:y0 + h, x0:x0 + w + 1])
        az[b].copy_(smp["haz"][y0:y0 + h + 1, x0:x0 + w])
    return r, c, ax, az


def train(net, samples: List[Dict], iters: int, n: int = 8, h: int = 256, w: int = 256,
          lr: float = 2e-3, seed: int = 0) -> Dict:
    """Adam on random crops, learning rate decayed linearly to lr / 10.
    Returns the losses and the wall time."""
    import torch
    rng = np.random.default_rng(seed)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(iters):
        r, c, ax, az = crops(samples, n, h, w, rng)
        rate = lr * (1.0 - 0.9 * it / max(1, iters - 1))
        losses.append(net.train_step(r, c, ax, az, rate))
    torch.cuda.synchronize()
    return {"losses": losses, "seconds": time.perf_counter() - t0}
