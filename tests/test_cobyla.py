"""The library's derivative-free minimiser (qaoa_cobyla_*, Powell's linear-interpolation method,
unconstrained) on problems with known minima, its reverse-communication protocol, and the
lockstep driver on QAOA objectives evaluated by the FP64 oracle: the result must be a stationary
point by the oracle's adjoint gradient. Host code only, no GPU."""
import numpy as np
import pytest

import synth
import paper_2506_10531_gb300 as q
from paper_2506_10531_gb300.train import cobyla_lockstep


def minimise(f, x0, rhobeg, rhoend, maxfun):
    c = q.Cobyla(x0, rhobeg, rhoend, maxfun)
    told = []
    try:
        while True:
            x = c.ask()
            if x is None:
                break
            v = f(x)
            told.append(v)
            c.tell(v)
        x, fv, n = c.result()
    finally:
        c.close()
    return x, fv, n, told


def test_separable_quadratic():
    a = np.array([1.0, -2.0, 0.5, 3.0, 0.0, -1.0])
    w = np.arange(1.0, 7.0)
    x, fv, n, told = minimise(lambda x: float(np.sum(w * (x - a) ** 2)), np.zeros(6), 0.5, 1e-6, 2000)
    assert np.abs(x - a).max() < 1e-4 and fv < 1e-8
    assert n == len(told) <= 2000 and fv == min(told)


def test_rotated_ill_conditioned_quadratic():
    rng = np.random.default_rng(0)
    Qm, _ = np.linalg.qr(rng.normal(size=(5, 5)))
    H = Qm @ np.diag([1.0, 3.0, 10.0, 30.0, 100.0]) @ Qm.T
    x, fv, n, _ = minimise(lambda x: float((x - 1) @ H @ (x - 1)), np.zeros(5), 0.5, 1e-7, 6000)
    assert np.abs(x - 1).max() < 1e-4 and fv < 1e-8


def test_budget_and_best_point():
    # an unbounded linear function: every step lowers it, so the budget ends the run
    c = np.array([1.0, -2.0, 0.5])
    x, fv, n, told = minimise(lambda x: float(c @ x), np.zeros(3), 0.1, 1e-3, 40)
    assert n == 40 and len(told) == 40
    assert fv == min(told) and fv < -1.0


def test_non_finite_values_stay_out_of_the_model():
    # an objective that is NaN (or +inf) on part of the space, with its minimum near the edge of
    # that region: the failed evaluations are neither kept as simplex values nor allowed to stop
    # the search early
    a = np.array([1.0, -0.5])
    for bad in (np.nan, np.inf):
        def f(x, bad=bad):
            return bad if x[0] > 1.2 else float(np.sum((x - a) ** 2))
        x, fv, n, told = minimise(f, np.zeros(2), 1.0, 1e-6, 2000)
        assert any(not np.isfinite(v) for v in told)         # the bad region was hit
        assert np.isfinite(fv) and np.abs(x - a).max() < 1e-4 and fv < 1e-8
    # a start inside the bad region has nothing to work from: the run ends with no finite value
    x, fv, n, told = minimise(lambda x: np.nan, np.zeros(2), 0.5, 1e-3, 50)
    assert not np.isfinite(fv) and n == 3


def test_protocol_errors():
    with pytest.raises(q.QaoaError):
        q.Cobyla(np.zeros(3), 0.1, 0.2, 100)        # rhoend > rhobeg
    with pytest.raises(q.QaoaError):
        q.Cobyla(np.zeros(3), 0.1, 1e-3, 4)         # maxfun < n + 2
    c = q.Cobyla(np.zeros(2), 0.1, 1e-3, 4)
    while c.ask() is not None:
        c.tell(1.0)
    with pytest.raises(q.QaoaError):
        c.tell(1.0)                                  # finished
    c.close()


def oracle_objective(orc, n, p, seed):
    Q = synth.symmetric_q(n, seed=seed)
    E = orc.energies(Q)

    def f(x):
        return float(orc.expect(orc.state(n, x[:p], x[p:], E), E))
    return f, E


@pytest.mark.parametrize("n,p,seed", [(6, 1, 1), (8, 2, 2), (9, 3, 3)])
def test_qaoa_objective_reaches_a_stationary_point(orc, n, p, seed):
    f, E = oracle_objective(orc, n, p, seed)
    g0, b0 = synth.random_params(p, seed=seed + 10)
    x0 = 0.3 * np.concatenate([g0, b0])
    x, fv, nf, _ = minimise(f, x0, 0.2, 1e-6, 3000)
    assert fv < f(x0)
    _, dg, db = orc.grad(n, x[:p], x[p:], E)
    scale = np.abs(E).max()
    assert np.abs(np.concatenate([dg, db])).max() < 1e-4 * scale


def test_lockstep_equals_separate_runs(orc):
    objs = [oracle_objective(orc, 7, 2, s)[0] for s in (4, 5, 6)]
    x0s = [0.3 * np.concatenate(synth.random_params(2, seed=20 + i)) for i in range(3)]
    calls = []

    def evaluate(points):
        calls.append(len(points))
        return [objs[i](x) for i, x in enumerate(points)]
    best, fbest, nfev, rounds = cobyla_lockstep(x0s, evaluate, 0.2, 1e-5, 500)
    assert rounds == max(nfev) and all(c == 3 for c in calls)
    for i in range(3):
        x, fv, n, _ = minimise(objs[i], x0s[i], 0.2, 1e-5, 500)
        np.testing.assert_array_equal(best[i], x)
        assert fbest[i] == fv and nfev[i] == n


class _OracleBatch:
    """Stand-in with QAOABatch's pools and layout (count, ps, float32 params as gamma[p] beta[p]
    per instance, float64 expect) whose run() evaluates <C> with the oracle."""

    def __init__(self, orc, specs):
        self.orc = orc
        self.Es, self.ns, self.ps, pars = [], [], [], []
        for n, p, seed in specs:
            self.Es.append(orc.energies(synth.symmetric_q(n, seed=seed)))
            self.ns.append(n)
            self.ps.append(p)
            pars.append(0.3 * np.concatenate(synth.random_params(p, seed=seed + 50)))
        import torch
        self.count = len(specs)
        self.params = torch.as_tensor(np.concatenate(pars).astype(np.float32))
        self.expect = torch.zeros(self.count, dtype=torch.float64)
        self.runs = 0

    def run(self, stream=None):
        flat = self.params.numpy().astype(np.float64)
        o = 0
        for i in range(self.count):
            n, p, E = self.ns[i], self.ps[i], self.Es[i]
            x = flat[o:o + 2 * p]
            self.expect[i] = float(self.orc.expect(self.orc.state(n, x[:p], x[p:], E), E))
            o += 2 * p
        self.runs += 1


def test_cobyla_train_layout_and_result(orc):
    from paper_2506_10531_gb300.train import cobyla_train
    b = _OracleBatch(orc, [(6, 1, 31), (7, 2, 32), (5, 3, 33)])
    b.run()
    start = b.expect.numpy().copy()
    fbest, rounds = cobyla_train(b, rhobeg=0.2, rhoend=1e-6, maxfun=2000)
    assert rounds > 0 and b.runs == rounds + 1
    assert np.all(fbest < start)
    # the pool holds the best parameters (FP32): re-evaluating reproduces the best values
    b.run()
    np.testing.assert_allclose(b.expect.numpy(), fbest, rtol=0, atol=1e-5 * np.abs(fbest).max())
    o = 0
    for i in range(b.count):
        n, p, E = b.ns[i], b.ps[i], b.Es[i]
        x = b.params.numpy()[o:o + 2 * p].astype(np.float64)
        _, dg, db = orc.grad(n, x[:p], x[p:], E)
        assert np.abs(np.concatenate([dg, db])).max() < 1e-3 * np.abs(E).max()
        o += 2 * p
