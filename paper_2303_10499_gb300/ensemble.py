"""Block-partition autotuner of an ensemble launch (gea_ensemble_*).

An ensemble step lasts as long as its slowest member, and a member's time
is its work -- tiles times the phases of its step, most of them the
iterations of its pressure and transport solves -- divided by its share of
the thread blocks. The tuner weights member m by

    w_m = tiles_m * (1 + iterations_m) ** beta

with iterations_m the Jacobi sweeps and CG iterations of its last step
(beta = 0: tiles only), times a few real steps of the run with each beta,
and keeps the fastest partition. The trial steps advance the simulation like
any other step.
"""
from __future__ import annotations

import statistics
from typing import Dict, Sequence, Tuple

import numpy as np

from . import gea


def member_work(solvers) -> Tuple[np.ndarray, np.ndarray]:
    """(tiles, iterations of the last step) per member."""
    tiles = np.array([((sv.grid.nx + 31) // 32) * ((sv.grid.nz + 7) // 8) for sv in solvers], dtype=np.float64)
    its = []
    for sv in solvers:
        st = sv.stats()
        its.append(st["jac_u"] + st["jac_h"] + sum(st["cg_iters"]))
    return tiles, np.array(its, dtype=np.float64)


def autotune(solvers, stream=None, betas: Sequence[float] = (0.0, 0.5, 1.0, 1.5),
             trial_steps: int = 2) -> Tuple["gea.Ensemble", Dict]:
    """Return the ensemble with the fastest block partition and a report of
    the trials (ms per step for each beta). The members must hold a state;
    every trial advances them by trial_steps steps."""
    import torch
    stream = stream or torch.cuda.current_stream()
    E = gea.Ensemble(solvers, stream=stream)
    E.step(1)                                   # one step to measure the iterations
    E.close()
    tiles, its = member_work(solvers)
    trials = {}
    best = None
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
        trials[beta] = t
        if best is None or t < best[0]:
            if best is not None:
                best[2].close()
            best = (t, beta, E)
        else:
            E.close()
    report = {"ms_per_step_by_beta": {str(b): round(v, 3) for b, v in trials.items()},
              "beta": best[1], "blocks": best[2].blocks()}
    return best[2], report
