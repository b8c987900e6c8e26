"""Batched QAOA parameter training on the device.

A `QAOABatch` binds a fixed set of sub-QUBO instances (n_i qubits, p_i layers) to device pools
and a launch plan of libqaoa: one plan launch computes <C> (Section IV, the cost C(theta)) of every
instance and, with gradients enabled, d<C>/d(gamma, beta) by the adjoint sweep. `QAOAExpectation`
exposes that as a torch.autograd.Function; `adam_train` runs the optimise loop (plan launch, then
the library's Adam kernel) with parameters and moments kept on the device. Everything that
computes runs in libqaoa; this module only arranges buffers and calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (QAOA_INST_GRAD, Cobyla, make_insts, make_io, qaoa_adam_step, qaoa_plan_capture,
               qaoa_plan_create, qaoa_plan_destroy, qaoa_plan_kernel_count, qaoa_plan_launch)


def footprint_bytes(n: int, grad: bool = True) -> int:
    """Device bytes one instance needs beyond the pools (streaming tier: psi, lam, E)."""
    if n <= 13:
        return 0
    return (20 if grad else 12) << n


class QAOABatch:
    """Instances with QUBO matrices Qs[i] (n_i x n_i), p_i layers and initial parameters
    params[i] = (gamma[p_i], beta[p_i])."""

    def __init__(self, ctx, Qs, params, k: int = 0, grad: bool = True, device="cuda"):
        self.count = len(Qs)
        self.ns = [int(Q.shape[0]) for Q in Qs]
        self.ps = [len(g) for g, _ in params]
        qoff, poff, rows = 0, 0, []
        qflat, pflat, owner = [], [], []
        for i, (Q, (g, b)) in enumerate(zip(Qs, params)):
            n, p = self.ns[i], self.ps[i]
            rows.append((n, p, k, QAOA_INST_GRAD if grad else 0, qoff, poff, -1, -1))
            qflat.append(np.asarray(Q, dtype=np.float32).reshape(-1))
            pflat.append(np.concatenate([np.asarray(g, np.float32), np.asarray(b, np.float32)]))
            owner.append(np.full(2 * p, i, dtype=np.int64))
            qoff += n * n
            poff += 2 * p
        self.nparams = poff
        self.q = torch.as_tensor(np.concatenate(qflat)).to(device)
        self.params = torch.as_tensor(np.concatenate(pflat)).to(device)
        self.grad = torch.zeros(poff, dtype=torch.float64, device=device)
        self.expect = torch.zeros(self.count, dtype=torch.float64, device=device)
        self.owner = torch.as_tensor(np.concatenate(owner)).to(device)
        self.k = k
        self.topk_idx = torch.zeros(max(self.count * k, 1), dtype=torch.int64, device=device)
        self.topk_prob = torch.zeros(max(self.count * k, 1), dtype=torch.float64, device=device)
        io = make_io(self.q, self.params, expect=self.expect,
                     topk_idx=self.topk_idx if k else None, topk_prob=self.topk_prob if k else None,
                     k_stride=k, grad=self.grad if grad else None)
        self._insts = make_insts(rows)
        self._io = io
        self.plan = qaoa_plan_create(ctx, self._insts, io)
        self.m = torch.zeros(poff, dtype=torch.float32, device=device)
        self.v = torch.zeros(poff, dtype=torch.float32, device=device)
        self.steps_done = 0
        self.captured = False

    @property
    def kernels_per_launch(self) -> int:
        return qaoa_plan_kernel_count(self.plan)

    def run(self, stream=None):
        """<C> (and gradients) of every instance at the current parameters (async). After
        capture() this replays the captured graph: one launch for the whole batch."""
        qaoa_plan_launch(self.plan, stream)

    def capture(self, stream):
        """Record the plan's launch sequence into a CUDA graph on `stream` (not the legacy
        default stream); every later run() replays it with one graph launch. The graph reads the
        bound pools, so parameters updated in place are seen. Per-kernel timing is off for a
        captured plan."""
        qaoa_plan_capture(self.plan, stream)
        self.captured = True

    def adam_step(self, lr: float, stream=None, beta1=0.9, beta2=0.999, eps=1e-8):
        self.steps_done += 1
        qaoa_adam_step(self.nparams, self.params, self.grad, self.m, self.v, self.steps_done, lr,
                       beta1, beta2, eps, True, stream)

    def close(self):
        if self.plan is not None:
            qaoa_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class QAOAExpectation(torch.autograd.Function):
    """<C> of every instance of a QAOABatch as a differentiable function of its parameter pool.

    forward(params, batch) copies params into the batch's pool when they are not the pool itself,
    launches the plan (values and adjoint gradients in one pass) and returns <C> per instance;
    backward scales each parameter's stored gradient by the upstream gradient of its instance.
    """

    @staticmethod
    def forward(ctx, params, batch: QAOABatch):
        if params.data_ptr() != batch.params.data_ptr():
            batch.params.copy_(params.detach())
        batch.run()
        ctx.batch = batch
        return batch.expect.clone()

    @staticmethod
    def backward(ctx, grad_out):
        b = ctx.batch
        g = b.grad * grad_out.to(torch.float64)[b.owner]
        return g.to(torch.float32), None


def adam_train(batch: QAOABatch, steps: int, lr: float, stream=None):
    """`steps` Adam steps of every instance's parameters; returns <C> before each step
    (device tensor [steps, count])."""
    import contextlib
    hist = torch.zeros(steps, batch.count, dtype=torch.float64, device=batch.params.device)
    on = torch.cuda.stream(stream) if isinstance(stream, torch.cuda.Stream) else contextlib.nullcontext()
    with on:   # the history copies are ordered with the launches on the same stream
        for s in range(steps):
            batch.run(stream)
            hist[s].copy_(batch.expect)
            batch.adam_step(lr, stream)
    return hist


def waves_by_footprint(ns, budget_bytes: int, grad: bool = True):
    """Split instance indices into consecutive waves whose streaming footprint fits the budget."""
    waves, cur, used = [], [], 0
    for i, n in enumerate(ns):
        f = footprint_bytes(n, grad)
        if cur and used + f > budget_bytes:
            waves.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += f
    if cur:
        waves.append(cur)
    return waves


def cobyla_lockstep(x0s, evaluate, rhobeg: float = 0.2, rhoend: float = 1e-4, maxfun: int = 300):
    """Independent derivative-free minimisations (libqaoa's qaoa_cobyla_*, Powell's method) advanced
    together: every round asks each unfinished minimisation for its next point and evaluates all
    of them with one call evaluate(points) -> values (a list of arrays in, a sequence of floats
    out; finished minimisations contribute their best point, whose value is not used). Returns
    (best points, best values, values evaluated per minimisation, rounds)."""
    states = [Cobyla(x0, rhobeg, rhoend, maxfun) for x0 in x0s]
    points = [np.array(x0, dtype=np.float64) for x0 in x0s]
    active = [True] * len(states)
    rounds = 0
    try:
        while True:
            for i, st in enumerate(states):
                if active[i]:
                    x = st.ask()
                    if x is None:
                        active[i] = False
                        points[i] = st.result()[0]
                    else:
                        points[i] = x
            if not any(active):
                break
            values = evaluate(points)
            for i, st in enumerate(states):
                if active[i]:
                    st.tell(float(values[i]))
            rounds += 1
        res = [st.result() for st in states]
    finally:
        for st in states:
            st.close()
    return [r[0] for r in res], [r[1] for r in res], [r[2] for r in res], rounds


def cobyla_train(batch: QAOABatch, rhobeg: float = 0.2, rhoend: float = 1e-4, maxfun: int = 300,
                 stream=None):
    """Gradient-free training of every instance of `batch` (the paper's optimiser family, Section
    IV): one COBYLA-type minimisation per instance over its (gamma, beta), all advanced in
    lockstep, each round one plan launch evaluating <C> of every instance. The best parameters
    end up in the batch's parameter pool (FP32). Returns (best <C> per instance, rounds)."""
    import contextlib
    dev = batch.params.device
    # every copy into the pool and every read of <C> is ordered on the stream the plan runs on
    if dev.type == "cuda":
        s = (torch.cuda.current_stream(dev) if stream is None else
             torch.cuda.ExternalStream(stream, device=dev) if isinstance(stream, int) else stream)
        on_stream = torch.cuda.stream(s)
    else:
        s, on_stream = None, contextlib.nullcontext()
    with on_stream:
        offs = np.cumsum([0] + [2 * p for p in batch.ps])
        flat = batch.params.detach().cpu().numpy().astype(np.float64)
        x0s = [flat[offs[i]:offs[i + 1]] for i in range(batch.count)]

        def evaluate(points):
            buf = np.concatenate(points).astype(np.float32)
            batch.params.copy_(torch.from_numpy(buf).to(dev))
            batch.run(s)
            return batch.expect.detach().cpu().numpy()

        best, fbest, _, rounds = cobyla_lockstep(x0s, evaluate, rhobeg, rhoend, maxfun)
        batch.params.copy_(torch.from_numpy(np.concatenate(best).astype(np.float32)).to(dev))
        if s is not None:
            s.synchronize()
    return np.array(fbest), rounds
