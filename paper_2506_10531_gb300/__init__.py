"""Python binding of libqaoa (include/qaoa.h): batched state-vector QAOA on sub-QUBOs and the
DQAOA decompose / merge steps, for NVIDIA GB300 (sm_103a).

Every function here only marshals arguments (device pointers from torch tensors, the current
CUDA stream, ctypes structs) and calls the C entry point of the same name; all computation
happens in the CUDA library. Importing the package does not need a GPU; calling into the
library needs the built ``libqaoa.so`` (``paper_2506_10531_gb300.build.build()``) and raises
``RuntimeError`` when it is missing. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqaoa.so")

QAOA_OK, QAOA_E_INVALID, QAOA_E_NOMEM, QAOA_E_CUDA, QAOA_E_TIMEOUT, QAOA_E_UNSUPPORTED = range(6)
QAOA_INST_GRAD = 1
QAOA_TIER_AUTO, QAOA_TIER_RESIDENT, QAOA_TIER_CLUSTER, QAOA_TIER_STREAM, QAOA_TIER_CSTREAM = 0, 1, 2, 3, 4
DQAOA_RANDOM, DQAOA_IFD, DQAOA_BFS, DQAOA_PFS = 0, 1, 2, 3
DQAOA_SIGNED_IMPACT = 16   # or-ed with IFD / BFS / PFS: rank by impact ascending
DQAOA_PAPER_MIXER = 32     # session: the printed mixer H_X = -sum X (beta -> -beta)

# Every symbol include/qaoa.h declares.
EXPORTS = [
    "qaoa_create", "qaoa_destroy", "qaoa_last_error", "qaoa_reserve", "qaoa_workspace_bytes",
    "qaoa_set_tier",
    "qaoa_build_energies", "qaoa_run_layers", "qaoa_expect", "qaoa_topk", "qaoa_grad",
    "qaoa_build_energies_z", "qaoa_run_layers_z", "qaoa_expect_z", "qaoa_topk_z", "qaoa_grad_z",
    "qaoa_plan_create", "qaoa_plan_launch", "qaoa_plan_kernel_count", "qaoa_plan_check", "qaoa_plan_destroy",
    "qaoa_batch_run", "qaoa_batch_run_z", "qaoa_plain_solve",
    "dqaoa_draw_indices", "dqaoa_decompose", "dqaoa_subqubo_build", "dqaoa_merge",
    "qaoa_plan_set_timing", "qaoa_plan_kernel_times", "qaoa_plan_kernel_bytes",
    "qaoa_expect_topk_static", "qaoa_adam_step",
    "dqaoa_session_create", "dqaoa_session_cycle", "dqaoa_session_results", "dqaoa_session_plan",
    "dqaoa_session_destroy", "dqaoa_session_cycle_sampled", "dqaoa_session_shots", "dqaoa_session_solve_ms",
    "qaoa_server_create", "qaoa_server_destroy", "qaoa_server_job_bytes", "qaoa_server_submit",
    "qaoa_server_tick", "qaoa_server_poll", "qaoa_server_stats", "qaoa_server_clock",
    "qaoa_server_cancel", "qaoa_server_fail_admissions",
    "qaoa_autotune", "qaoa_tuning_get", "qaoa_tuning_save", "qaoa_tuning_load", "qaoa_plan_capture",
    "dqaoa_session_timing", "qaoa_sample",
    "qaoa_cobyla_create", "qaoa_cobyla_ask", "qaoa_cobyla_tell", "qaoa_cobyla_result", "qaoa_cobyla_destroy",
]


class QaoaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libqaoa status {status}: {msg}")
        self.status = status


class qaoa_inst(C.Structure):
    _fields_ = [("n", C.c_int32), ("p", C.c_int32), ("k", C.c_int32), ("flags", C.c_int32),
                ("q_off", C.c_int64), ("par_off", C.c_int64), ("psi_off", C.c_int64),
                ("e_off", C.c_int64)]


class qaoa_job_result(C.Structure):
    _fields_ = [("job_id", C.c_int64), ("n", C.c_int32), ("p", C.c_int32), ("steps", C.c_int32),
                ("k", C.c_int32), ("expect", C.c_double), ("topk_idx", C.c_uint64 * 16),
                ("topk_prob", C.c_double * 16), ("params", C.c_float * 128), ("t_submit", C.c_double),
                ("t_done", C.c_double)]


class qaoa_batch_io(C.Structure):
    _fields_ = [("q", C.c_void_p), ("params", C.c_void_p), ("psi", C.c_void_p), ("e", C.c_void_p),
                ("expect", C.c_void_p), ("topk_idx", C.c_void_p), ("topk_prob", C.c_void_p),
                ("k_stride", C.c_int32), ("grad", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libqaoa (ctypes.CDLL). Raises RuntimeError if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libqaoa.so not built at {LIB_PATH}: run "
                                   "paper_2506_10531_gb300.build.build() (there is no CPU path)")
            L = C.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    vp, i32, i64, u64, sz, dp = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_size_t, C.c_void_p
    st = C.c_int
    L.qaoa_create.argtypes = [C.POINTER(vp), i32]
    L.qaoa_destroy.argtypes = [vp]
    L.qaoa_destroy.restype = None
    L.qaoa_last_error.restype = C.c_char_p
    L.qaoa_reserve.argtypes = [vp, sz]
    L.qaoa_workspace_bytes.argtypes = [i32, i32]
    L.qaoa_workspace_bytes.restype = sz
    L.qaoa_set_tier.argtypes = [vp, i32, i32, i32]
    L.qaoa_adam_step.argtypes = [i32, vp, vp, vp, vp, i32, C.c_float, C.c_float, C.c_float, C.c_float,
                                 i32, vp]
    L.qaoa_expect_topk_static.argtypes = [i32, vp, vp, i32, vp, vp, vp, vp]
    for suf in ("", "_z"):
        getattr(L, "qaoa_build_energies" + suf).argtypes = [vp, i32, vp, vp, vp]
        getattr(L, "qaoa_run_layers" + suf).argtypes = [vp, i32, i32, vp, vp, vp, vp, i32, vp]
        getattr(L, "qaoa_expect" + suf).argtypes = [vp, i32, vp, vp, vp, vp]
        getattr(L, "qaoa_topk" + suf).argtypes = [vp, i32, vp, i32, vp, vp, vp]
        getattr(L, "qaoa_grad" + suf).argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp]
    L.qaoa_plan_create.argtypes = [vp, vp, i32, C.POINTER(qaoa_batch_io), i32, C.POINTER(vp)]
    L.qaoa_plan_launch.argtypes = [vp, vp]
    L.qaoa_plan_kernel_count.argtypes = [vp]
    L.qaoa_plan_kernel_count.restype = i32
    L.qaoa_plan_check.argtypes = [vp]
    L.qaoa_plan_check.restype = st
    L.qaoa_plan_destroy.argtypes = [vp]
    L.qaoa_plan_destroy.restype = None
    L.qaoa_batch_run.argtypes = [vp, vp, i32, C.POINTER(qaoa_batch_io), vp]
    L.qaoa_batch_run_z.argtypes = [vp, vp, i32, C.POINTER(qaoa_batch_io), vp]
    L.qaoa_plain_solve.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp]
    L.dqaoa_draw_indices.argtypes = [vp, i32, vp, i32, i32, i32, u64, u64, vp]
    L.dqaoa_decompose.argtypes = [vp, i32, vp, i32, i32, i32, i32, u64, u64, vp, vp]
    L.dqaoa_subqubo_build.argtypes = [vp, vp, i32, vp, i32, i32, vp, i32, vp, vp]
    L.dqaoa_merge.argtypes = [vp, i32, vp, i32, i32, vp, i32, vp, vp, vp]
    L.qaoa_plan_set_timing.argtypes = [vp, i32]
    L.qaoa_plan_kernel_times.argtypes = [vp, vp, vp, i32]
    L.qaoa_plan_kernel_times.restype = i32
    L.qaoa_plan_kernel_bytes.argtypes = [vp, vp, i32]
    L.qaoa_plan_kernel_bytes.restype = i32
    L.dqaoa_session_create.argtypes = [vp, i32, i32, i32, i32, i32, i32, i32, vp, vp, C.POINTER(vp)]
    L.dqaoa_session_cycle.argtypes = [vp, vp, i32, vp, u64, u64, vp, vp, vp]
    L.dqaoa_session_results.argtypes = [vp, vp, vp]
    L.dqaoa_session_cycle_sampled.argtypes = [vp, vp, i32, vp, u64, u64, i32, vp, vp, vp, vp]
    L.dqaoa_session_shots.argtypes = [vp, vp, vp, vp]
    L.dqaoa_session_timing.argtypes = [vp, vp]
    L.dqaoa_session_solve_ms.argtypes = [vp, vp]
    L.dqaoa_session_plan.argtypes = [vp, i32]
    L.dqaoa_session_plan.restype = vp
    L.dqaoa_session_destroy.argtypes = [vp]
    L.dqaoa_session_destroy.restype = None
    L.qaoa_server_create.argtypes = [vp, sz, i32, i32, C.POINTER(vp)]
    L.qaoa_server_destroy.argtypes = [vp]
    L.qaoa_server_destroy.restype = None
    L.qaoa_server_job_bytes.argtypes = [vp, i32, i32]
    L.qaoa_server_job_bytes.restype = sz
    L.qaoa_server_submit.argtypes = [vp, i32, i32, vp, vp, i32, C.c_float, C.POINTER(i64)]
    L.qaoa_server_tick.argtypes = [vp, vp, C.POINTER(i32), C.POINTER(i32)]
    L.qaoa_server_poll.argtypes = [vp, i32, C.POINTER(qaoa_job_result), i32]
    L.qaoa_server_poll.restype = i32
    L.qaoa_server_stats.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(sz), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    L.qaoa_server_cancel.argtypes = [vp, i64]
    L.qaoa_server_fail_admissions.argtypes = [vp, i32, C.POINTER(C.c_longlong)]
    L.qaoa_autotune.argtypes = [vp, i32, i32, i32, i32, vp, C.POINTER(C.c_double)]
    L.qaoa_tuning_get.argtypes = [vp, i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_double)]
    L.qaoa_tuning_save.argtypes = [vp, C.c_char_p]
    L.qaoa_tuning_load.argtypes = [vp, C.c_char_p]
    L.qaoa_plan_capture.argtypes = [vp, vp]
    L.qaoa_sample.argtypes = [vp, i32, vp, i64, vp, vp, vp]
    L.qaoa_cobyla_create.argtypes = [i32, vp, C.c_double, C.c_double, i32, C.POINTER(vp)]
    L.qaoa_cobyla_ask.argtypes = [vp, vp]
    L.qaoa_cobyla_ask.restype = i32
    L.qaoa_cobyla_tell.argtypes = [vp, C.c_double]
    L.qaoa_cobyla_result.argtypes = [vp, vp, vp, vp]
    L.qaoa_cobyla_destroy.argtypes = [vp]
    L.qaoa_cobyla_destroy.restype = None
    L.qaoa_server_clock.argtypes = []
    L.qaoa_server_clock.restype = C.c_double
    del st, dp


def _check(status):
    if status != QAOA_OK:
        msg = lib().qaoa_last_error()
        raise QaoaError(status, msg.decode() if msg else "")


def ptr(x):
    """Device/host address of a torch tensor or numpy array, an int, or None (NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(type(x))


def stream_ptr(stream=None):
    """cudaStream_t of a torch stream (default: the current stream)."""
    if isinstance(stream, int):
        return stream
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# ---------------------------------------------------------------------------------------------
# thin wrappers, same names as the C entry points
# ---------------------------------------------------------------------------------------------

def qaoa_create(device: int = 0):
    h = C.c_void_p()
    _check(lib().qaoa_create(C.byref(h), device))
    return h


def qaoa_destroy(ctx):
    lib().qaoa_destroy(ctx)


def qaoa_reserve(ctx, nbytes: int):
    _check(lib().qaoa_reserve(ctx, nbytes))


def qaoa_workspace_bytes(n: int, dbl: bool = False) -> int:
    return lib().qaoa_workspace_bytes(n, int(dbl))


def qaoa_build_energies(ctx, n, Q, E, stream=None, dbl=False):
    f = lib().qaoa_build_energies_z if dbl else lib().qaoa_build_energies
    _check(f(ctx, n, ptr(Q), ptr(E), stream_ptr(stream)))


def qaoa_run_layers(ctx, n, p, gamma, beta, E, psi, init_plus=True, stream=None, dbl=False):
    f = lib().qaoa_run_layers_z if dbl else lib().qaoa_run_layers
    _check(f(ctx, n, p, ptr(gamma), ptr(beta), ptr(E), ptr(psi), int(init_plus), stream_ptr(stream)))


def qaoa_expect(ctx, n, psi, E, out, stream=None, dbl=False):
    f = lib().qaoa_expect_z if dbl else lib().qaoa_expect
    _check(f(ctx, n, ptr(psi), ptr(E), ptr(out), stream_ptr(stream)))


def qaoa_sample(ctx, n, psi, shots, u, out, stream=None):
    """Inverse-CDF shots of a complex64 state with the caller's uniforms u (device doubles)."""
    _check(lib().qaoa_sample(ctx, n, ptr(psi), int(shots), ptr(u), ptr(out), stream_ptr(stream)))


def qaoa_cobyla_create(nvar, x0, rhobeg, rhoend, maxfun):
    """Handle of a new minimisation (x0: host float64 array of nvar values)."""
    h = C.c_void_p()
    _check(lib().qaoa_cobyla_create(int(nvar), ptr(x0), float(rhobeg), float(rhoend), int(maxfun),
                                    C.byref(h)))
    return h


def qaoa_cobyla_ask(h, x) -> int:
    """1: evaluate at x (written into the float64 array x); 0: finished, x = best point."""
    return lib().qaoa_cobyla_ask(h, ptr(x))


def qaoa_cobyla_tell(h, f):
    _check(lib().qaoa_cobyla_tell(h, float(f)))


def qaoa_cobyla_result(h, x):
    """Writes the best point into x; returns (best value, values told)."""
    f = C.c_double()
    n = C.c_int()
    _check(lib().qaoa_cobyla_result(h, ptr(x), C.byref(f), C.byref(n)))
    return f.value, n.value


def qaoa_cobyla_destroy(h):
    lib().qaoa_cobyla_destroy(h)


class Cobyla:
    """Reverse-communication minimiser (qaoa_cobyla_*): ask() returns the next point to evaluate
    (numpy float64) or None when finished; tell(f) reports its value; result() the best point."""

    def __init__(self, x0, rhobeg, rhoend, maxfun):
        import numpy as np
        self._h = None
        self.x = np.array(x0, dtype=np.float64).ravel()
        self._h = qaoa_cobyla_create(self.x.size, self.x, rhobeg, rhoend, maxfun)

    def ask(self):
        return self.x.copy() if qaoa_cobyla_ask(self._h, self.x) else None

    def tell(self, f):
        qaoa_cobyla_tell(self._h, f)

    def result(self):
        import numpy as np
        x = np.empty_like(self.x)
        f, n = qaoa_cobyla_result(self._h, x)
        return x, f, n

    def close(self):
        if self._h:
            qaoa_cobyla_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qaoa_topk(ctx, n, psi, k, idx, prob, stream=None, dbl=False):
    f = lib().qaoa_topk_z if dbl else lib().qaoa_topk
    _check(f(ctx, n, ptr(psi), k, ptr(idx), ptr(prob), stream_ptr(stream)))


def qaoa_grad(ctx, n, p, gamma, beta, E, expect, dgamma, dbeta, stream=None, dbl=False):
    f = lib().qaoa_grad_z if dbl else lib().qaoa_grad
    _check(f(ctx, n, p, ptr(gamma), ptr(beta), ptr(E), ptr(expect), ptr(dgamma), ptr(dbeta),
             stream_ptr(stream)))


def make_io(q, params, expect=None, topk_idx=None, topk_prob=None, k_stride=0, psi=None, e=None,
            grad=None) -> qaoa_batch_io:
    io = qaoa_batch_io(ptr(q), ptr(params), ptr(psi), ptr(e), ptr(expect), ptr(topk_idx),
                       ptr(topk_prob), k_stride, ptr(grad))
    # the descriptor holds raw addresses: keep the buffers alive as long as it is
    io._keep = (q, params, expect, topk_idx, topk_prob, psi, e, grad)
    return io


def make_insts(rows):
    """rows: iterable of (n, p, k, flags, q_off, par_off, psi_off, e_off)."""
    rows = list(rows)
    arr = (qaoa_inst * len(rows))()
    for i, r in enumerate(rows):
        arr[i] = qaoa_inst(*r)
    return arr


def qaoa_plan_create(ctx, insts, io: qaoa_batch_io, dbl=False):
    h = C.c_void_p()
    _check(lib().qaoa_plan_create(ctx, C.cast(insts, C.c_void_p), len(insts), C.byref(io), int(dbl),
                                  C.byref(h)))
    return h


def qaoa_plan_launch(plan, stream=None):
    _check(lib().qaoa_plan_launch(plan, stream_ptr(stream)))


def qaoa_plan_kernel_count(plan) -> int:
    return lib().qaoa_plan_kernel_count(plan)


def qaoa_plan_check(plan):
    """Raises QaoaError (QAOA_E_TIMEOUT) if a device-side wait of the plan's launches ran out."""
    _check(lib().qaoa_plan_check(plan))


def qaoa_plan_destroy(plan):
    lib().qaoa_plan_destroy(plan)


def qaoa_batch_run(ctx, insts, io: qaoa_batch_io, stream=None, dbl=False):
    f = lib().qaoa_batch_run_z if dbl else lib().qaoa_batch_run
    _check(f(ctx, C.cast(insts, C.c_void_p), len(insts), C.byref(io), stream_ptr(stream)))


def qaoa_plain_solve(ctx, n, p, Q, gamma, beta, E, psi, k, expect, topk_idx, topk_prob, stream=None):
    _check(lib().qaoa_plain_solve(ctx, n, p, ptr(Q), ptr(gamma), ptr(beta), ptr(E), ptr(psi), k,
                                  ptr(expect), ptr(topk_idx), ptr(topk_prob), stream_ptr(stream)))


def dqaoa_draw_indices(Q, N, x, method, m, k, seed, cycle, idx):
    _check(lib().dqaoa_draw_indices(ptr(Q), N, ptr(x), method, m, k, seed, cycle, ptr(idx)))


def dqaoa_decompose(Q, N, x, method, conditioned, m, k, seed, cycle, idx, qsub):
    _check(lib().dqaoa_decompose(ptr(Q), N, ptr(x), method, int(conditioned), m, k, seed, cycle,
                                 ptr(idx), ptr(qsub)))


def dqaoa_subqubo_build(ctx, Q_dev, N, x_dev, m, k, idx_dev, conditioned, qsub_dev, stream=None):
    _check(lib().dqaoa_subqubo_build(ctx, ptr(Q_dev), N, ptr(x_dev), m, k, ptr(idx_dev),
                                     int(conditioned), ptr(qsub_dev), stream_ptr(stream)))


def dqaoa_merge(Q, N, x, m, k, idx, K, cand):
    """Host merge; returns (energy, accepted). x (numpy uint8) is updated in place."""
    e = C.c_double()
    a = C.c_int()
    _check(lib().dqaoa_merge(ptr(Q), N, ptr(x), m, k, ptr(idx), K, ptr(cand), C.byref(e), C.byref(a)))
    return e.value, a.value


def qaoa_last_error() -> str:
    m = lib().qaoa_last_error()
    return m.decode() if m else ""


def qaoa_build_energies_z(ctx, n, Q, E, stream=None):
    qaoa_build_energies(ctx, n, Q, E, stream, dbl=True)


def qaoa_run_layers_z(ctx, n, p, gamma, beta, E, psi, init_plus=True, stream=None):
    qaoa_run_layers(ctx, n, p, gamma, beta, E, psi, init_plus, stream, dbl=True)


def qaoa_expect_z(ctx, n, psi, E, out, stream=None):
    qaoa_expect(ctx, n, psi, E, out, stream, dbl=True)


def qaoa_topk_z(ctx, n, psi, k, idx, prob, stream=None):
    qaoa_topk(ctx, n, psi, k, idx, prob, stream, dbl=True)


def qaoa_grad_z(ctx, n, p, gamma, beta, E, expect, dgamma, dbeta, stream=None):
    qaoa_grad(ctx, n, p, gamma, beta, E, expect, dgamma, dbeta, stream, dbl=True)


def qaoa_batch_run_z(ctx, insts, io: qaoa_batch_io, stream=None):
    qaoa_batch_run(ctx, insts, io, stream, dbl=True)


def qaoa_plan_set_timing(plan, on=True):
    _check(lib().qaoa_plan_set_timing(plan, int(on)))


def qaoa_plan_kernel_times(plan, max_kernels=256):
    """[(kernel family, ms)] of the last launch of a plan with timing on."""
    ms = (C.c_float * max_kernels)()
    names = (C.c_char_p * max_kernels)()
    n = lib().qaoa_plan_kernel_times(plan, ms, names, max_kernels)
    return [(names[i].decode(), float(ms[i])) for i in range(n)]


def dqaoa_session_create(ctx, N, m, k, p, K, method, conditioned, gamma, beta):
    import numpy as np
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    h = C.c_void_p()
    _check(lib().dqaoa_session_create(ctx, N, m, k, p, K, method, int(conditioned), ptr(g), ptr(b),
                                      C.byref(h)))
    return h


def dqaoa_session_cycle(sess, Q, q_changed, x, seed, cycle, stream=None):
    """One DQAOA cycle; x (host uint8) is updated in place. Returns (energy, accepted)."""
    e = C.c_double()
    a = C.c_int()
    _check(lib().dqaoa_session_cycle(sess, ptr(Q), int(q_changed), ptr(x), seed, cycle, C.byref(e),
                                     C.byref(a), stream_ptr(stream)))
    return e.value, a.value


def dqaoa_session_results(sess, m, K):
    import numpy as np
    ex = np.zeros(m, dtype=np.float64)
    tk = np.zeros((m, K), dtype=np.uint64)
    _check(lib().dqaoa_session_results(sess, ptr(ex), ptr(tk)))
    return ex, tk


def dqaoa_session_solve_ms(sess) -> float:
    """Device ms of the last cycle's chunk solves (first launch to last kernel end)."""
    v = C.c_double()
    _check(lib().dqaoa_session_solve_ms(sess, C.byref(v)))
    return v.value


def dqaoa_session_cycle_sampled(sess, Q, q_changed, x, seed, cycle, u, stream=None):
    """One DQAOA cycle with shot-based sub-solutions; u: (m, shots) host float64 uniforms in
    [0, 1). x (host uint8) is updated in place. Returns (energy, accepted)."""
    import numpy as np
    u = np.ascontiguousarray(u, dtype=np.float64)
    e = C.c_double()
    a = C.c_int()
    _check(lib().dqaoa_session_cycle_sampled(sess, ptr(Q), int(q_changed), ptr(x), seed, cycle, int(u.shape[-1]),
                                             ptr(u), C.byref(e), C.byref(a), stream_ptr(stream)))
    return e.value, a.value


def dqaoa_session_shots(sess, m, k, shots, states=False):
    """(shots (m, shots) uint64, chosen candidate (m,) uint64, states (m, 2^k) complex64 or None)
    of the last sampled cycle."""
    import numpy as np
    z = np.zeros((m, shots), dtype=np.uint64)
    best = np.zeros(m, dtype=np.uint64)
    psi = np.zeros((m, 1 << k), dtype=np.complex64) if states else None
    _check(lib().dqaoa_session_shots(sess, ptr(z), ptr(best), ptr(psi) if states else None))
    return z, best, psi


def dqaoa_session_plan(sess, i=0):
    """Plan i of the session (None past the last one)."""
    h = lib().dqaoa_session_plan(sess, i)
    return C.c_void_p(h) if h else None


def dqaoa_session_plans(sess):
    out, i = [], 0
    while True:
        h = dqaoa_session_plan(sess, i)
        if h is None:
            return out
        out.append(h)
        i += 1


def dqaoa_session_destroy(sess):
    lib().dqaoa_session_destroy(sess)


def qaoa_plan_kernel_bytes(plan, max_kernels=256):
    """Algorithmic DRAM bytes of each kernel of one launch of the plan, in launch order."""
    b = (C.c_double * max_kernels)()
    n = lib().qaoa_plan_kernel_bytes(plan, b, max_kernels)
    return [float(b[i]) for i in range(n)]


def qaoa_set_tier(ctx, n, tier, param=0):
    _check(lib().qaoa_set_tier(ctx, n, tier, param))


def qaoa_expect_topk_static(n, psi, E, k, expect, idx, prob, stream=None):
    """<C> and top-k without a context or any allocation (fixed scratch inside the library)."""
    _check(lib().qaoa_expect_topk_static(n, ptr(psi), ptr(E), k, ptr(expect), ptr(idx), ptr(prob),
                                         stream_ptr(stream)))


def qaoa_adam_step(count, theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, minimise=True,
                   stream=None):
    _check(lib().qaoa_adam_step(count, ptr(theta), ptr(grad), ptr(m), ptr(v), step, lr, beta1, beta2, eps,
                                int(minimise), stream_ptr(stream)))


# ---- serving ---------------------------------------------------------------------------------

def qaoa_server_create(ctx, scratch_bytes: int, max_jobs: int, k: int):
    h = C.c_void_p()
    _check(lib().qaoa_server_create(ctx, scratch_bytes, max_jobs, k, C.byref(h)))
    return h


def qaoa_server_destroy(srv):
    lib().qaoa_server_destroy(srv)


def qaoa_server_job_bytes(srv, n, p) -> int:
    return lib().qaoa_server_job_bytes(srv, n, p)


def qaoa_server_submit(srv, n, p, Q, params, steps, lr) -> int:
    """Q: n*n host floats, params: 2p host floats (gamma then beta). Returns the job id."""
    import numpy as np
    Qa = np.ascontiguousarray(Q, dtype=np.float32).reshape(-1)
    Pa = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
    jid = C.c_int64()
    _check(lib().qaoa_server_submit(srv, n, p, Qa.ctypes.data, Pa.ctypes.data, steps, lr, C.byref(jid)))
    return jid.value


def qaoa_server_tick(srv, stream=None):
    """Returns (active, queued) after admission."""
    a, q = C.c_int(), C.c_int()
    _check(lib().qaoa_server_tick(srv, stream_ptr(stream), C.byref(a), C.byref(q)))
    return a.value, q.value


def qaoa_server_poll(srv, wait=False, max_results=4096):
    """Finished jobs as a list of qaoa_job_result."""
    buf = (qaoa_job_result * max_results)()
    n = lib().qaoa_server_poll(srv, int(wait), buf, max_results)
    if n < 0:
        raise QaoaError(QAOA_E_INVALID, "server_poll: NULL server")
    return [buf[i] for i in range(n)]


def qaoa_server_stats(srv):
    """(queued, active, scratch bytes in use, algorithmic bytes launched, device ms harvested,
    kernel launches)."""
    q, a, u, b, t, n = C.c_int(), C.c_int(), C.c_size_t(), C.c_double(), C.c_double(), C.c_longlong()
    _check(lib().qaoa_server_stats(srv, C.byref(q), C.byref(a), C.byref(u), C.byref(b), C.byref(t),
                                   C.byref(n)))
    return q.value, a.value, u.value, b.value, t.value, n.value


def qaoa_server_cancel(srv, job_id):
    _check(lib().qaoa_server_cancel(srv, job_id))


def qaoa_server_fail_admissions(srv, count) -> int:
    """Make the next `count` admission attempts fail (host-side fault injection); returns the
    admission failures so far."""
    f = C.c_longlong()
    _check(lib().qaoa_server_fail_admissions(srv, count, C.byref(f)))
    return f.value


def qaoa_server_clock() -> float:
    return lib().qaoa_server_clock()


# ---- autotuner and graph capture -------------------------------------------------------------

def qaoa_autotune(ctx, n, p, k, count, stream=None) -> float:
    """Time the configurations for (n, p) batches and store the fastest; returns its ms."""
    ms = C.c_double()
    _check(lib().qaoa_autotune(ctx, n, p, k, count, stream_ptr(stream), C.byref(ms)))
    return ms.value


def qaoa_tuning_get(ctx, n, p):
    """(tier, param, ms) stored for (n, p); tier 0 when none."""
    t, prm, ms = C.c_int(), C.c_int(), C.c_double()
    _check(lib().qaoa_tuning_get(ctx, n, p, C.byref(t), C.byref(prm), C.byref(ms)))
    return t.value, prm.value, ms.value


def qaoa_tuning_save(ctx, path):
    _check(lib().qaoa_tuning_save(ctx, os.fsencode(path)))


def qaoa_tuning_load(ctx, path):
    _check(lib().qaoa_tuning_load(ctx, os.fsencode(path)))


def qaoa_plan_capture(plan, stream):
    """Capture the plan's launch into a CUDA graph; later launches replay it (non-legacy stream)."""
    _check(lib().qaoa_plan_capture(plan, stream_ptr(stream)))


def dqaoa_session_timing(sess):
    """{decompose_ms, device_ms, merge_ms, cycle_ms} of the session's last cycle."""
    import numpy as np
    out = np.zeros(4)
    _check(lib().dqaoa_session_timing(sess, out.ctypes.data))
    return dict(zip(("decompose_ms", "device_ms", "merge_ms", "cycle_ms"), out.tolist()))
