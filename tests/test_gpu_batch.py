"""Batched plans (mixed tiers in one plan) against the FP64 oracle and against the single-
instance path; batch invariance: an instance's results do not depend on the rest of the batch."""
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
    q.qaoa_reserve(c, q.qaoa_workspace_bytes(24))
    yield c
    q.qaoa_destroy(c)


GRAD_STATE_NMAX = 13   # the final state is returned together with a gradient up to this n


def build_batch(specs, seed):
    """specs: list of (n, p, k, grad). Returns host pools and descriptor rows."""
    qpool, ppool, rows, Qs, params = [], [], [], [], []
    qo = po = so = eo = 0
    for i, (n, p, k, grad) in enumerate(specs):
        Q = synth.symmetric_q(n, seed=seed + i).astype(np.float32)
        g, b = synth.random_params(p, seed=seed + 1000 + i)
        par = np.concatenate([g, b]).astype(np.float32)
        psi_off = so if not (grad and n > GRAD_STATE_NMAX) else -1
        rows.append((n, p, k, 1 if grad else 0, qo, po, psi_off, eo))
        qpool.append(Q.reshape(-1)); ppool.append(par)
        Qs.append(Q); params.append(par)
        qo += n * n; po += 2 * p; so += 1 << n; eo += 1 << n
    return np.concatenate(qpool), np.concatenate(ppool), rows, Qs, params, so, eo


def run_batch(q, ctx, specs, seed, order=None):
    qp, pp, rows, Qs, params, so, eo = build_batch(specs, seed)
    count = len(rows)
    qd = torch.as_tensor(qp).cuda()
    pd = torch.as_tensor(pp).cuda()
    psi = torch.zeros(2 * so, dtype=torch.float32, device="cuda")
    E = torch.zeros(eo, dtype=torch.float32, device="cuda")
    ex = torch.zeros(count, dtype=torch.float64, device="cuda")
    K = 16
    ti = torch.zeros(count * K, dtype=torch.int64, device="cuda")
    tp = torch.zeros(count * K, dtype=torch.float64, device="cuda")
    gr = torch.zeros(len(pp), dtype=torch.float64, device="cuda")
    io = q.make_io(qd, pd, expect=ex, topk_idx=ti, topk_prob=tp, k_stride=K, psi=psi, e=E, grad=gr)
    insts = q.make_insts(rows)
    q.qaoa_batch_run(ctx, insts, io)
    torch.cuda.synchronize()
    return dict(rows=rows, Qs=Qs, params=params, psi=psi.cpu().numpy(), E=E.cpu().numpy(),
                ex=ex.cpu().numpy(), ti=ti.cpu().numpy().reshape(count, K),
                tp=tp.cpu().numpy().reshape(count, K), gr=gr.cpu().numpy())


SPECS = [(3, 2, 4, True), (9, 3, 8, True), (14, 2, 8, False), (12, 1, 16, True), (15, 2, 8, False),
         (17, 3, 8, False), (14, 3, 8, False), (5, 8, 8, True), (13, 2, 1, True), (16, 1, 8, False),
         (18, 2, 8, False), (16, 3, 8, False), (14, 2, 8, True), (16, 2, 4, True)]


def test_batch_matches_oracle(q, ctx, orc):
    r = run_batch(q, ctx, SPECS, seed=900)
    for i, (n, p, k, grad, qo, po, so, eo) in enumerate(r["rows"]):
        Qd = r["Qs"][i].astype(np.float64)
        par = r["params"][i].astype(np.float64)
        g, b = par[:p], par[p:]
        E_o = orc.energies(Qd)
        absq = np.abs(Qd).sum()
        E_g = r["E"][eo:eo + (1 << n)]
        assert np.max(np.abs(E_g - E_o)) <= 1e-5 * absq, i
        psi_o = orc.state(n, g, b, E_o)
        assert abs(r["ex"][i] - orc.expect(psi_o, E_o)) <= 1e-5 * absq, i
        if so >= 0:
            ps = r["psi"][2 * so:2 * (so + (1 << n))].reshape(-1, 2)
            psi_g = ps[:, 0].astype(np.float64) + 1j * ps[:, 1]
            assert np.max(np.abs(psi_g - psi_o)) <= 1e-5, i
            oi, op = orc.topk_probs(orc.probs(psi_g), k)
            np.testing.assert_array_equal(r["ti"][i, :k].astype(np.uint64), oi)
            np.testing.assert_array_equal(r["tp"][i, :k], op)
        else:   # top-k against the FP64 state with the near-tie rule
            pr = np.abs(psi_o) ** 2
            eps = 4e-5 * np.sqrt(pr.max())
            ri, rp = orc.topk_probs(pr, k)
            for t in range(k):
                assert abs(pr[int(r["ti"][i, t])] - rp[t]) <= eps, (i, t)
        if grad:
            _, dg, db = orc.grad(n, g, b, E_o)
            ref = np.concatenate([dg, db])
            got = r["gr"][po:po + 2 * p]
            assert np.max(np.abs(got - ref)) <= 1e-5 * max(np.max(np.abs(ref)), 1.0) * max(1.0, n / 4), i


def test_batch_invariance(q, ctx):
    # the same instance alone and inside a mix gives bitwise identical results
    full = run_batch(q, ctx, SPECS, seed=900)
    for i in (1, 2, 5):
        alone = run_batch(q, ctx, [SPECS[i]], seed=900 + i)
        n = SPECS[i][0]
        so = full["rows"][i][6]
        np.testing.assert_array_equal(alone["psi"][:2 << n], full["psi"][2 * so:2 * so + (2 << n)])
        assert alone["ex"][0] == full["ex"][i]
        np.testing.assert_array_equal(alone["ti"][0], full["ti"][i])


@pytest.mark.parametrize("tier,param", [(2, 13), (2, 14), (3, 0)])
def test_tiers_agree_for_large_n(q, orc, tier, param):
    # the cluster tier (13 or 14 local qubits per CTA) and the streaming tier give the oracle's
    # results for n = 15..18
    specs = [(15, 2, 8, False), (16, 3, 8, False), (17, 1, 8, False), (18, 2, 4, False)]
    c = q.qaoa_create(0)
    try:
        for n, *_ in specs:
            if tier == 2 and n - param > 4:
                continue
            q.qaoa_set_tier(c, n, tier, param)
        r = run_batch(q, c, specs, seed=4242)
    finally:
        q.qaoa_destroy(c)
    for i, (n, p, k, grad, qo, po, so, eo) in enumerate(r["rows"]):
        Qd = r["Qs"][i].astype(np.float64)
        par = r["params"][i].astype(np.float64)
        E_o = orc.energies(Qd)
        psi_o = orc.state(n, par[:p], par[p:], E_o)
        ps = r["psi"][2 * so:2 * (so + (1 << n))].reshape(-1, 2)
        psi_g = ps[:, 0].astype(np.float64) + 1j * ps[:, 1]
        assert np.max(np.abs(psi_g - psi_o)) <= 1e-5, (n, tier, param)
        assert abs(r["ex"][i] - orc.expect(psi_o, E_o)) <= 1e-5 * np.abs(Qd).sum()
        oi, op = orc.topk_probs(orc.probs(psi_g), k)
        np.testing.assert_array_equal(r["ti"][i, :k].astype(np.uint64), oi)


def test_batch_rejects_bad_descriptors(q, ctx):
    qd = torch.zeros(16, device="cuda")
    io = q.make_io(qd, qd, expect=torch.zeros(1, dtype=torch.float64, device="cuda"))
    for row in [(0, 1, 0, 0, 0, 0, -1, -1), (31, 1, 0, 0, 0, 0, -1, -1), (4, 0, 0, 0, 0, 0, -1, -1),
                (4, 1, 17, 0, 0, 0, -1, -1), (4, 1, 2, 0, 0, 0, -1, -1)]:
        with pytest.raises(q.QaoaError) as e:
            q.qaoa_batch_run(ctx, q.make_insts([row]), io)
        assert e.value.status == q.QAOA_E_INVALID
