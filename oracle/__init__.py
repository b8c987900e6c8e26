"""FP64 CPU oracle for the QAOA / DQAOA hot path (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import this package; the product library never does, and this package imports
nothing from it. The arithmetic lives in ``qaoa_oracle.c`` (plain C, FP64, complex128), built
with gcc into ``liboracle.so`` beside it; this module only marshals numpy arrays.

Functions mirror the paper's steps (arXiv 2506.10531):
  energies          - E(z) = z^T Q z for all z (Section IV, QUBO -> diagonal problem Hamiltonian)
  state             - Eq. 2 ansatz from |+>, p layers of cost then mixer
  expect, topk      - <C> and the k most probable bitstrings (the sub-solution, Section IV)
  grad              - adjoint d<C>/d(gamma, beta)
  decompose, merge  - Section V-A random / IFD (Algorithm 1) decomposition and Section V step 3
                      aggregation
Parity of each function is pinned by the ``-m "not gpu"`` tests against closed forms, brute
force and invariants (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qaoa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP, fp-contract off). Returns the path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=gnu11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    dp, ip, u8p, u64p, i32p = (C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_uint8),
                               C.POINTER(C.c_uint64), C.POINTER(C.c_int32))
    L.orc_energies.argtypes = [C.c_int, dp, dp]
    L.orc_qubo_energy.argtypes = [dp, C.c_int, u8p]
    L.orc_qubo_energy.restype = C.c_double
    L.orc_state.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_int, dp]
    L.orc_apply_layers.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_int, dp]
    L.orc_expect.argtypes = [C.c_int, dp, dp]
    L.orc_expect.restype = C.c_double
    L.orc_probs.argtypes = [C.c_int64, dp, dp]
    L.orc_topk_probs.argtypes = [C.c_int64, dp, C.c_int, u64p, dp]
    L.orc_sample_probs.argtypes = [C.c_int64, dp, C.c_int64, dp, u64p]
    L.orc_grad.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_int, dp, dp, dp]
    L.orc_splitmix64.argtypes = [C.c_uint64, C.c_int, u64p]
    L.orc_impact.argtypes = [dp, C.c_int, u8p, dp]
    L.orc_decompose.argtypes = [dp, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                C.c_uint64, i32p, dp]
    L.orc_merge.argtypes = [dp, C.c_int, u8p, C.c_int, C.c_int, i32p, C.c_int, u64p, dp, ip]


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _chk(rc):
    if rc != 0:
        raise RuntimeError(f"oracle call failed with status {rc}")


def energies(Q) -> np.ndarray:
    Q = _f64(Q)
    n = Q.shape[0]
    E = np.empty(1 << n, dtype=np.float64)
    _chk(lib().orc_energies(n, _p(Q, C.c_double), _p(E, C.c_double)))
    return E


def qubo_energy(Q, x) -> float:
    Q = _f64(Q)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    return lib().orc_qubo_energy(_p(Q, C.c_double), Q.shape[0], _p(x, C.c_uint8))


def state(n, gamma, beta, E, mixer_sign: int = 1) -> np.ndarray:
    g, b, E = _f64(np.atleast_1d(gamma)), _f64(np.atleast_1d(beta)), _f64(E)
    psi = np.empty(1 << n, dtype=np.complex128)
    _chk(lib().orc_state(n, len(g), _p(g, C.c_double), _p(b, C.c_double), _p(E, C.c_double),
                         mixer_sign, _p(psi.view(np.float64), C.c_double)))
    return psi


def apply_layers(psi, gamma, beta, E, mixer_sign: int = 1) -> np.ndarray:
    psi = np.array(psi, dtype=np.complex128, copy=True)
    n = int(np.log2(psi.size))
    g, b, E = _f64(np.atleast_1d(gamma)), _f64(np.atleast_1d(beta)), _f64(E)
    _chk(lib().orc_apply_layers(n, len(g), _p(g, C.c_double), _p(b, C.c_double),
                                _p(E, C.c_double), mixer_sign, _p(psi.view(np.float64), C.c_double)))
    return psi


def expect(psi, E) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    E = _f64(E)
    n = int(np.log2(psi.size))
    return lib().orc_expect(n, _p(psi.view(np.float64), C.c_double), _p(E, C.c_double))


def probs(psi) -> np.ndarray:
    """|psi|^2 in FP64 as re*re + im*im (no FMA). For complex64 input the squares are exact."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty(psi.size, dtype=np.float64)
    lib().orc_probs(psi.size, _p(psi.view(np.float64), C.c_double), _p(out, C.c_double))
    return out


def topk_probs(prob, k):
    prob = _f64(prob)
    idx = np.empty(k, dtype=np.uint64)
    pk = np.empty(k, dtype=np.float64)
    _chk(lib().orc_topk_probs(prob.size, _p(prob, C.c_double), k, _p(idx, C.c_uint64),
                              _p(pk, C.c_double)))
    return idx, pk


def topk(psi, k):
    return topk_probs(probs(psi), k)


def sample_probs(prob, u):
    """Inverse-CDF shots: for each uniform u_s, the first z with cumsum(prob)[z] > u_s * sum(prob)."""
    prob, u = _f64(prob), _f64(np.atleast_1d(u))
    out = np.empty(u.size, dtype=np.uint64)
    _chk(lib().orc_sample_probs(prob.size, _p(prob, C.c_double), u.size, _p(u, C.c_double),
                                _p(out, C.c_uint64)))
    return out


def sample(psi, u):
    return sample_probs(probs(psi), u)


def grad(n, gamma, beta, E, mixer_sign: int = 1):
    g, b, E = _f64(np.atleast_1d(gamma)), _f64(np.atleast_1d(beta)), _f64(E)
    p = len(g)
    ex = np.zeros(1)
    dg = np.empty(p)
    db = np.empty(p)
    _chk(lib().orc_grad(n, p, _p(g, C.c_double), _p(b, C.c_double), _p(E, C.c_double), mixer_sign,
                        _p(ex, C.c_double), _p(dg, C.c_double), _p(db, C.c_double)))
    return float(ex[0]), dg, db


def splitmix64(seed, count):
    out = np.empty(count, dtype=np.uint64)
    lib().orc_splitmix64(seed, count, _p(out, C.c_uint64))
    return out


def impact(Q, x):
    Q = _f64(Q)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    out = np.empty(Q.shape[0])
    lib().orc_impact(_p(Q, C.c_double), Q.shape[0], _p(x, C.c_uint8), _p(out, C.c_double))
    return out


RANDOM, IFD, BFS, PFS = 0, 1, 2, 3
SIGNED = 16     # or-ed with IFD / BFS / PFS: rank by the energy change, largest decrease first


def decompose(Q, x, m, k, seed, cycle=0, method=RANDOM, conditioned=True):
    Q = _f64(Q)
    N = Q.shape[0]
    xx = np.ascontiguousarray(x if x is not None else np.zeros(N), dtype=np.uint8)
    idx = np.empty((m, k), dtype=np.int32)
    qs = np.empty((m, k, k), dtype=np.float64)
    _chk(lib().orc_decompose(_p(Q, C.c_double), N, _p(xx, C.c_uint8), method, int(conditioned), m,
                             k, seed, cycle, _p(idx, C.c_int32), _p(qs, C.c_double)))
    return idx, qs


def merge(Q, x, idx, cand):
    """Returns (x', energy(x'), accepted). cand is m x K uint64 bitstrings in top-k order."""
    Q = _f64(Q)
    N = Q.shape[0]
    x = np.array(x, dtype=np.uint8, copy=True)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    cand = np.ascontiguousarray(cand, dtype=np.uint64)
    m, k = idx.shape
    K = cand.shape[1]
    e = np.zeros(1)
    acc = np.zeros(1, dtype=np.int32)
    _chk(lib().orc_merge(_p(Q, C.c_double), N, _p(x, C.c_uint8), m, k, _p(idx, C.c_int32), K,
                         _p(cand, C.c_uint64), _p(e, C.c_double), acc.ctypes.data_as(C.POINTER(C.c_int))))
    return x, float(e[0]), int(acc[0])
