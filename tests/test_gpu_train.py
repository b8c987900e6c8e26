"""Training on the device: the Adam kernel, the autograd wrapper and the uneven adjoint batch.

Checks (all through the C ABI):
  * qaoa_adam_step against the textbook Adam update (Kingma & Ba 2015) in FP64 on the same
    float32 inputs, over three consecutive steps (bias correction depends on the step number);
  * the adjoint gradients of an uneven batch (n 8..24 mixed with p 1..6, normal Q) against the
    FP64 oracle's adjoint (the parity tolerance of the single-instance gradient test) and
    against central finite differences of the oracle's <C> with h = 1e-3 (relative 1e-3);
  * QAOAExpectation.backward equals the plan's gradients scaled by the upstream gradient;
  * a short Adam run: <C> reported by the device at the final parameters equals the oracle's,
    and <C> went down for most instances.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_10531_gb300 import build
    build.build()
    import paper_2506_10531_gb300 as qq
    return qq


@pytest.fixture(scope="module")
def ctx(q):
    c = q.qaoa_create(0)
    yield c
    q.qaoa_destroy(c)


def adam_fp64(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def test_adam_step_matches_textbook(q):
    cnt = 1000
    rng = np.random.default_rng(11)
    th = rng.uniform(-1, 1, cnt).astype(np.float32)
    grads = [rng.normal(0, 3, cnt) for _ in range(3)]
    t_d = torch.as_tensor(th).cuda()
    m_d = torch.zeros(cnt, dtype=torch.float32, device="cuda")
    v_d = torch.zeros(cnt, dtype=torch.float32, device="cuda")
    th_r, m_r, v_r = th.astype(np.float64), np.zeros(cnt), np.zeros(cnt)
    for s, g in enumerate(grads, start=1):
        q.qaoa_adam_step(cnt, t_d, torch.as_tensor(g).cuda(), m_d, v_d, s, 0.05)
        th_r, m_r, v_r = adam_fp64(th_r, g.astype(np.float32).astype(np.float64), m_r, v_r, s, 0.05)
    torch.cuda.synchronize()
    np.testing.assert_allclose(t_d.cpu().numpy(), th_r, rtol=0, atol=2e-6)
    np.testing.assert_allclose(m_d.cpu().numpy(), m_r, rtol=1e-5, atol=1e-6)
    # maximise flips the update direction
    t2 = torch.zeros(4, dtype=torch.float32, device="cuda")
    q.qaoa_adam_step(4, t2, torch.ones(4, dtype=torch.float64, device="cuda"),
                     torch.zeros(4, device="cuda"), torch.zeros(4, device="cuda"), 1, 0.1, minimise=False)
    torch.cuda.synchronize()
    assert np.allclose(t2.cpu().numpy(), 0.1, atol=1e-6)
    with pytest.raises(q.QaoaError):
        q.qaoa_adam_step(4, t2, t2, t2, t2, 0, 0.1)


def sample_batch(count, seed, n_hi=24):
    return synth.uneven_batch(count, seed, 8, n_hi, 1, 6)


def oracle_fd(orc, n, g, b, E, h=1e-3):
    p = len(g)
    th = np.concatenate([g, b])
    out = np.zeros(2 * p)
    for j in range(2 * p):
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fp = orc.expect(orc.state(n, tp[:p], tp[p:], E), E)
        fm = orc.expect(orc.state(n, tm[:p], tm[p:], E), E)
        out[j] = (fp - fm) / (2 * h)
    return out


def test_uneven_batch_grads_vs_oracle(q, ctx, orc):
    from paper_2506_10531_gb300.train import QAOABatch
    inst = sample_batch(48, seed=31, n_hi=20)
    B = QAOABatch(ctx, [x[0] for x in inst], [(x[1], x[2]) for x in inst])
    try:
        B.run()
        torch.cuda.synchronize()
        grad = B.grad.cpu().numpy()
        expect = B.expect.cpu().numpy()
        params = B.params.cpu().numpy().astype(np.float64)
        off = 0
        checked_fd = 0
        for i, (Q, g0, _) in enumerate(inst):
            n, p = Q.shape[0], len(g0)
            Qd = Q.astype(np.float32).astype(np.float64)
            E = orc.energies(Qd)
            g, b = params[off:off + p], params[off + p:off + 2 * p]
            e_o, dg_o, db_o = orc.grad(n, g, b, E)
            ref = np.concatenate([dg_o, db_o])
            got = grad[off:off + 2 * p]
            absq = np.abs(Qd).sum()
            assert abs(expect[i] - e_o) <= 1e-5 * absq, (i, n, p)
            scale = max(np.max(np.abs(ref)), 1.0)
            assert np.max(np.abs(got - ref)) <= 1e-5 * scale * max(1.0, n / 4), (i, n, p)
            if n <= 14 and checked_fd < 8:
                fd = oracle_fd(orc, n, g, b, E)
                assert np.max(np.abs(got - fd)) <= 1e-3 * max(np.max(np.abs(fd)), 1.0), (i, n, p)
                checked_fd += 1
            off += 2 * p
        assert checked_fd >= 4
    finally:
        B.close()


def test_autograd_backward_scales_plan_grads(q, ctx, orc):
    from paper_2506_10531_gb300.train import QAOABatch, QAOAExpectation
    inst = sample_batch(12, seed=32, n_hi=16)
    B = QAOABatch(ctx, [x[0] for x in inst], [(x[1], x[2]) for x in inst])
    try:
        theta = B.params.clone().requires_grad_(True)
        w = torch.linspace(-1.0, 2.0, B.count, dtype=torch.float64, device="cuda")
        loss = (QAOAExpectation.apply(theta, B) * w).sum()
        loss.backward()
        torch.cuda.synchronize()
        ref = (B.grad * w[B.owner]).to(torch.float32)
        assert torch.equal(theta.grad, ref)
        assert loss.item() == pytest.approx(float((B.expect * w).sum()), rel=1e-12)
    finally:
        B.close()


def test_adam_training_matches_oracle_at_final_params(q, ctx, orc):
    from paper_2506_10531_gb300.train import QAOABatch, adam_train
    inst = sample_batch(24, seed=33, n_hi=18)
    B = QAOABatch(ctx, [x[0] for x in inst], [(x[1], x[2]) for x in inst])
    try:
        hist = adam_train(B, steps=8, lr=0.05)
        B.run()
        torch.cuda.synchronize()
        h = hist.cpu().numpy()
        final = B.expect.cpu().numpy()
        params = B.params.cpu().numpy().astype(np.float64)
        off = 0
        for i, (Q, g0, _) in enumerate(inst):
            n, p = Q.shape[0], len(g0)
            Qd = Q.astype(np.float32).astype(np.float64)
            E = orc.energies(Qd)
            e_o = orc.expect(orc.state(n, params[off:off + p], params[off + p:off + 2 * p], E), E)
            assert abs(final[i] - e_o) <= 1e-5 * np.abs(Qd).sum(), (i, n, p)
            off += 2 * p
        assert np.mean(final < h[0]) >= 0.75
    finally:
        B.close()


def test_training_through_a_captured_graph_is_identical(q, ctx):
    # the same Adam run with the batch plan launched kernel by kernel and replayed from one
    # captured CUDA graph per step: identical parameters and <C> history, bit for bit
    from paper_2506_10531_gb300.train import QAOABatch, adam_train
    inst = sample_batch(40, seed=34, n_hi=20)
    s = torch.cuda.Stream()
    A = QAOABatch(ctx, [x[0] for x in inst], [(x[1], x[2]) for x in inst])
    B = QAOABatch(ctx, [x[0] for x in inst], [(x[1], x[2]) for x in inst])
    try:
        ha = adam_train(A, 5, 0.05, stream=s)
        B.capture(s)
        hb = adam_train(B, 5, 0.05, stream=s)
        s.synchronize()
        assert B.captured and not A.captured
        assert torch.equal(ha, hb)
        assert torch.equal(A.params, B.params)
        assert torch.equal(A.grad, B.grad)
    finally:
        A.close()
        B.close()


def test_tma_adjoint_matches_cp_async_adjoint(q, orc):
    # the TMA adjoint passes (default) and the per-thread cp.async adjoint (streaming variant 2)
    # on the same gradient batch (n 14..24, every adjoint pass shape: kind A, kind-B chunks of
    # 1..8 high qubits): gradients and <C> agree within the parity tolerance, and both match the
    # FP64 oracle on a sample
    from paper_2506_10531_gb300.train import QAOABatch
    inst = []
    for i, (n, p) in enumerate([(14, 3), (15, 2), (16, 4), (17, 1), (19, 2), (20, 3), (21, 2), (22, 1), (24, 2)]):
        Q = synth.symmetric_q(n, seed=700 + i, dist="normal")
        g, b = synth.random_params(p, seed=800 + i)
        inst.append((Q, g, b))
    out = {}
    for variant in (0, 2):
        ctx = q.qaoa_create(0)
        try:
            for n in range(15, 25):
                q.qaoa_set_tier(ctx, n, q.QAOA_TIER_STREAM, variant)
            B = QAOABatch(ctx, [x[0] for x in inst], [(x[1], x[2]) for x in inst])
            try:
                B.run()
                torch.cuda.synchronize()
                q.qaoa_plan_check(B.plan)
                out[variant] = (B.grad.cpu().numpy(), B.expect.cpu().numpy(), B.params.cpu().numpy().astype(np.float64))
            finally:
                B.close()
        finally:
            q.qaoa_destroy(ctx)
    g0, e0, params = out[0]
    g2, e2, _ = out[2]
    off = 0
    for i, (Q, gg, _) in enumerate(inst):
        n, p = Q.shape[0], len(gg)
        Qd = Q.astype(np.float32).astype(np.float64)
        absq = np.abs(Qd).sum()
        a, b = g0[off:off + 2 * p], g2[off:off + 2 * p]
        scale = max(np.max(np.abs(b)), 1.0)
        assert np.max(np.abs(a - b)) <= 1e-5 * scale * max(1.0, n / 4), (i, n, p)
        assert abs(e0[i] - e2[i]) <= 1e-5 * absq, (i, n, p)
        if n <= 20:
            E = orc.energies(Qd)
            e_o, dg_o, db_o = orc.grad(n, params[off:off + p], params[off + p:off + 2 * p], E)
            ref = np.concatenate([dg_o, db_o])
            assert np.max(np.abs(a - ref)) <= 1e-5 * max(np.max(np.abs(ref)), 1.0) * max(1.0, n / 4), (i, n, p)
        off += 2 * p
