"""Tile-shape and block-partition autotuner of an ensemble launch
(gea_ensemble_*, gea_set_tile_shape).

An ensemble step lasts as long as its slowest member, and a member's time
is its work -- tiles times the phases of its step, most of them the
iterations of its pressure and transport solves -- divided by its share of
the thread blocks. The tuner weights member m by

    w_m = tiles_m * (1 + iterations_m) ** beta

with iterations_m the Jacobi sweeps and CG iterations of its last step
(beta = 0: tiles only; members whose weight is worth less than a block are
packed onto shared blocks by the library, so a heavy weight on the large
members is not capped by one block for every small one), times a few real
steps of the run with each beta,
and keeps the fastest partition. It does so for each tile shape of the
persistent kernels (one thread per cell of a 32 x 8, 16 x 16 or 64 x 4
tile; squarer tiles load smaller halos, wider ones longer rows, and the
tile count of a member changes its share of blocks) and keeps the fastest
shape and partition together. The trial steps advance the simulation like
any other step.
"""
from __future__ import annotations

import statistics
from typing import Dict, Sequence, Tuple

import numpy as np

from . import gea


SHAPE_DIMS = {0: (32, 8), 1: (16, 16), 2: (64, 4)}


def member_work(solvers, shape: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """(tiles of the shape, iterations of the last step) per member."""
    bx, bz = SHAPE_DIMS[shape]
    tiles = np.array([((sv.grid.nx + bx - 1) // bx) * ((sv.grid.nz + bz - 1) // bz) for sv in solvers],
                     dtype=np.float64)
    its = []
    for sv in solvers:
        st = sv.stats()
        its.append(st["jac_u"] + st["jac_h"] + sum(st["cg_iters"]))
    return tiles, np.array(its, dtype=np.float64)


def autotune(solvers, stream=None, betas: Sequence[float] = (0.0, 0.5, 1.0, 1.5, 2.0, 2.5),
             trial_steps: int = 2, shapes: Sequence[int] = (0, 1, 2)) -> Tuple["gea.Ensemble", Dict]:
    """Return the ensemble with the fastest tile shape and block partition
    and a report of the trials (ms per step for each shape and beta). The
    members must hold a state; every trial advances them by trial_steps
    steps. The members keep the chosen shape."""
    import torch
    stream = stream or torch.cuda.current_stream()
    for sv in solvers:
        sv.set_tile_shape(shapes[0])
    E = gea.Ensemble(solvers, stream=stream)
    E.step(1)                                   # one step to measure the iterations
    E.close()
    _, its = member_work(solvers)
    trials = {}
    best = None
    for shape in shapes:
        for sv in solvers:
            sv.set_tile_shape(shape)
        tiles, _ = member_work(solvers, shape)
        for beta in betas:
            w = tiles * (1.0 + its) ** beta
            E = gea.Ensemble(solvers, stream=stream, weights=w)
            ms = []
            for _ in range(trial_steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                E.step_async(1)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            E.sync()
            t = statistics.median(ms)
            trials[(shape, beta)] = t
            if best is None or t < best[0]:
                if best is not None:
                    best[3].close()
                best = (t, shape, beta, E)
            else:
                E.close()
    # the kept ensemble was built with the best shape: set it on the members
    # again (the loop left them at the last candidate)
    for sv in solvers:
        sv.set_tile_shape(best[1])
    by_shape = {}
    for (shape, beta), t in trials.items():
        by_shape.setdefault(gea.TILE_SHAPES[shape], {})[str(beta)] = round(t, 3)
    report = {"ms_per_step_by_shape_and_beta": by_shape, "tile_shape": gea.TILE_SHAPES[best[1]],
              "beta": best[2], "blocks": best[3].blocks()}
    return best[3], report
