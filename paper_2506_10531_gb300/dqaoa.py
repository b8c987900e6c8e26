"""Multi-cycle DQAOA driver (Section V: decompose, solve the sub-QUBOs in parallel, aggregate,
repeat) over one libqaoa session, with per-cycle timing and a time-to-solution stopping rule.

Stopping rule (the paper's T.t.S. of Section VI counts cycles until the approximation ratio stays
within a band for five consecutive cycles): with a reference energy, stop once
|E(x) / E_ref - 1| <= tol for `patience` consecutive cycles; without one, stop once E(x) has not
decreased for `patience` consecutive cycles. `max_cycles` bounds the run either way. Every step of
the cycle runs in the library (index draw and merge on the host, sub-QUBO matrices, energies,
layers, <C> and top-k on the device); this module only loops and records.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import (DQAOA_RANDOM, dqaoa_session_create, dqaoa_session_cycle, dqaoa_session_destroy,
               dqaoa_session_timing)


@dataclass
class SolveResult:
    x: np.ndarray
    energy: float
    energies: list = field(default_factory=list)     # E(x) after each cycle
    accepted: list = field(default_factory=list)     # accepted candidates per cycle
    timing: list = field(default_factory=list)       # per-cycle {decompose_ms, device_ms, merge_ms, cycle_ms}
    cycles: int = 0
    converged: bool = False
    tts_s: float | None = None                       # wall time until the stopping window began
    wall_s: float = 0.0


def solve(ctx, Q, m, k, p, K, gamma, beta, x0, seed=0, method=DQAOA_RANDOM, conditioned=True,
          max_cycles=100, patience=5, ref_energy=None, tol=1e-3, stream=None) -> SolveResult:
    """Run DQAOA cycles on the dense QUBO Q (N x N float64) from the bit vector x0."""
    N = Q.shape[0]
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    x = np.array(x0, dtype=np.uint8, copy=True)
    sess = dqaoa_session_create(ctx, N, m, k, p, K, method, conditioned, gamma, beta)
    res = SolveResult(x=x, energy=float("nan"))
    try:
        t0 = time.perf_counter()
        streak, best, window_start = 0, None, None
        for c in range(max_cycles):
            e, acc = dqaoa_session_cycle(sess, Q, 1 if c == 0 else 0, x, seed, c, stream)
            now = time.perf_counter() - t0
            res.energies.append(e)
            res.accepted.append(acc)
            res.timing.append(dqaoa_session_timing(sess))
            res.cycles = c + 1
            if ref_energy is not None:
                ok = abs(e / ref_energy - 1.0) <= tol
            else:
                ok = best is not None and e >= best
            best = e if best is None else min(best, e)
            if ok:
                if streak == 0:
                    window_start = now
                streak += 1
                if streak >= patience:
                    res.converged = True
                    res.tts_s = window_start
                    break
            else:
                streak = 0
        res.wall_s = time.perf_counter() - t0
    finally:
        dqaoa_session_destroy(sess)
    res.x = x
    res.energy = res.energies[-1] if res.energies else float("nan")
    return res
