"""Seeded synthetic inputs for the QAOA / DQAOA hot path.

This module holds input generation only: random QUBO matrices, parameter vectors, instance
mixes and initial global solutions. It contains none of the method's arithmetic (no energies,
no state vectors, no decomposition or merge) so that both the FP64 oracle under ``oracle/`` and
the CUDA library can be fed from it without sharing any computation.

Random source: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator: output ``i`` of stream ``s`` is
``mix(s + (i+1) * 0x9E3779B97F4A7C15)``, which is exactly the sequential SplitMix64 output
sequence started from state ``s``.

Distributions:
  * uniform double u in [0,1): ``(x >> 11) * 2**-53``;
  * uniform on [-1,1]: ``2u - 1``;
  * standard normal: Box-Muller on consecutive pairs (u1 from ``((x>>11)+1) * 2**-53`` so it is
    never 0), ``sqrt(-2 ln u1) * cos(2 pi u2)`` (only the cosine branch is used);
  * symmetric Q: the stream fills the upper triangle including the diagonal in row-major order,
    then the lower triangle is mirrored.

The workloads mirror the shapes the paper runs (dense QUBOs of N = 300-1000 decomposed into
sub-QUBOs of size 4-28, Section VI) with uniform or normal entries, because the metamaterial and
Max-Cut instances the paper uses are not distributed with it.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 sequence seeded with ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    x = splitmix64(seed, count, start)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int, start: int = 0) -> np.ndarray:
    return 2.0 * uniform01(seed, count, start) - 1.0


def normal(seed: int, count: int, start: int = 0) -> np.ndarray:
    x = splitmix64(seed, 2 * count, 2 * start)
    u1 = ((x[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (x[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def symmetric_q(n: int, seed: int, dist: str = "uniform", stream_start: int = 0) -> np.ndarray:
    """Dense symmetric n x n QUBO matrix (float64) from the seeded stream."""
    m = n * (n + 1) // 2
    if dist == "uniform":
        v = uniform_pm1(seed, m, stream_start)
    elif dist == "normal":
        v = normal(seed, m, stream_start)
    else:
        raise ValueError(dist)
    q = np.zeros((n, n), dtype=np.float64)
    iu = np.triu_indices(n)
    q[iu] = v
    q = q + np.triu(q, 1).T
    return q


def bits(seed: int, count: int) -> np.ndarray:
    """Seeded 0/1 bytes (initial global solution x0): bit 0 of each SplitMix64 output."""
    return (splitmix64(seed, count) & np.uint64(1)).astype(np.uint8)


def maxcut_form_q(n: int, seed: int, edge_prob: float = 0.5) -> np.ndarray:
    """Field-free Ising-form QUBO: random graph with weights in [-1,1], Q_ii = -sum_j Q_ij.

    With s = 1 - 2z this Q gives E(z) = const + sum_{i<j} J_ij s_i s_j with J = Q_offdiag / 2,
    i.e. no linear field, which is the setting of the closed-form p = 1 expectation.
    """
    w = uniform_pm1(seed, n * n).reshape(n, n)
    keep = uniform01(seed ^ 0x5A5A5A5A, n * n).reshape(n, n) < edge_prob
    a = np.triu(np.where(keep, w, 0.0), 1)
    a = a + a.T
    np.fill_diagonal(a, -a.sum(axis=1))
    return a


def maxcut_graph_q(n: int, seed: int, edges: int | None = None) -> np.ndarray:
    """Max-Cut QUBO of an unweighted random graph with exactly ``edges`` edges (default
    n(n-1)/8, the edge count of the paper's Max-Cut study, Section VI).

    The edge set is the ``edges`` vertex pairs (i < j, row-major order) with the smallest
    SplitMix64 keys of stream ``seed``: a uniform subset of that size. The QUBO is
    Q_ij = Q_ji = 1 for every edge and Q_ii = -deg(i), so that x^T Q x = -cut(x).
    """
    if edges is None:
        edges = n * (n - 1) // 8
    iu, ju = np.triu_indices(n, 1)
    keys = splitmix64(seed, iu.size)
    pick = np.argsort(keys, kind="stable")[:edges]
    q = np.zeros((n, n))
    q[iu[pick], ju[pick]] = 1.0
    q = q + q.T
    np.fill_diagonal(q, -q.sum(axis=1))
    return q


def cut_value(Q: np.ndarray, x: np.ndarray) -> float:
    """Cut size of the bit vector x on the graph of a ``maxcut_graph_q`` matrix (its off-diagonal
    ones), counted edge by edge."""
    a = np.triu(Q, 1) != 0
    xb = np.asarray(x).astype(bool)
    return float(np.sum(a & (xb[:, None] != xb[None, :])))


# ---------------------------------------------------------------------------------------------
# Workload recipes (sizes and seeds of the measured configurations)
# ---------------------------------------------------------------------------------------------

def grid_params(points: int = 16):
    """16 x 16 grid: gamma_i = i*pi/15, beta_j = j*(pi/2)/15 (both endpoints included)."""
    g = np.arange(points) * np.pi / (points - 1)
    b = np.arange(points) * (np.pi / 2) / (points - 1)
    gg, bb = np.meshgrid(g, b, indexing="ij")
    return gg.reshape(-1).copy(), bb.reshape(-1).copy()


def random_params(p: int, seed: int):
    """gamma uniform on [0, pi], beta uniform on [0, pi/2]."""
    u = uniform01(seed, 2 * p)
    return u[:p] * np.pi, u[p:] * (np.pi / 2)


def uneven_mix(count: int, seed: int, n_lo: int, n_hi: int, p_lo: int, p_hi: int):
    """(n, p) per instance: n uniform on n_lo..n_hi, p uniform on p_lo..p_hi (inclusive)."""
    x = splitmix64(seed, 2 * count)
    n = n_lo + (x[0::2] % np.uint64(n_hi - n_lo + 1)).astype(np.int64)
    p = p_lo + (x[1::2] % np.uint64(p_hi - p_lo + 1)).astype(np.int64)
    return n, p


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential gaps -ln(1-u)/rate."""
    u = uniform01(seed, count)
    return np.cumsum(-np.log1p(-u) / rate)


# Config of the DQAOA batch cycle: dense N=1000 QUBO, 256 sub-QUBOs of 16 variables, p=3.
DQAOA_BATCH = dict(seed=2, N=1000, m=256, k=16, p=3,
                   gamma=(0.2, 0.4, 0.6), beta=(0.6, 0.4, 0.2), topk=8)


def uneven_batch(count: int, seed: int, n_lo: int, n_hi: int, p_lo: int, p_hi: int,
                 dist: str = "normal"):
    """Instances of an uneven batch: (n, p) from uneven_mix, instance i's Q from the stream seeded
    with output i of the seed's own sequence, and its initial (gamma, beta) from random_params
    seeded with that value XOR 0x5151."""
    ns, ps = uneven_mix(count, seed, n_lo, n_hi, p_lo, p_hi)
    seeds = splitmix64(seed ^ 0xA5A5A5A5, count)
    out = []
    for i in range(count):
        s = int(seeds[i])
        g, b = random_params(int(ps[i]), s ^ 0x5151)
        out.append((symmetric_q(int(ns[i]), s, dist), g, b))
    return out


# Config of the uneven training batch: 4096 instances, n in 8..24, p in 1..6, normal Q,
# 20 Adam steps at learning rate 0.05.
UNEVEN_BATCH = dict(seed=3, count=4096, n=(8, 24), p=(1, 6), dist="normal", steps=20, lr=0.05)
