"""Edge cases through the C ABI: the largest depth (p = 64) on every tier, a batch of one and of
zero instances, k = 0 (no top-k requested), k = 2^n (every bitstring ranked), the DQAOA session
with one chunk and with two chunks giving the same cycle, a zero-parameter layer (γ = β = 0:
the state stays |+>), and the streaming top-k carried across runs of tiles (runs crossing states,
long runs, all-tied probabilities, FP64 states)."""
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


def solve(q, ctx, Q32, g, b, k, want_state=True):
    n = Q32.shape[0]
    qd = torch.as_tensor(Q32.reshape(-1)).cuda()
    pd = torch.as_tensor(np.concatenate([g, b]).astype(np.float32)).cuda()
    psi = torch.zeros(2 << n, dtype=torch.float32, device="cuda") if want_state else None
    ex = torch.zeros(1, dtype=torch.float64, device="cuda")
    ti = torch.zeros(max(k, 1), dtype=torch.int64, device="cuda")
    tp = torch.zeros(max(k, 1), dtype=torch.float64, device="cuda")
    io = q.make_io(qd, pd, expect=ex, topk_idx=ti if k else None, topk_prob=tp if k else None,
                   k_stride=k, psi=psi)
    q.qaoa_batch_run(ctx, q.make_insts([(n, len(g), k, 0, 0, 0, 0 if want_state else -1, -1)]), io)
    torch.cuda.synchronize()
    return psi, ex.item(), ti.cpu().numpy(), tp.cpu().numpy()


@pytest.mark.parametrize("n,tier", [(8, 0), (15, 2), (16, 3), (17, 3)])
def test_depth_64(q, orc, n, tier):
    c = q.qaoa_create(0)
    try:
        if tier:
            q.qaoa_set_tier(c, n, tier, 13 if tier == 2 else 0)
        p = 64
        Q32 = synth.symmetric_q(n, seed=600 + n).astype(np.float32)
        g, b = synth.random_params(p, seed=601 + n)
        g = (0.05 * g).astype(np.float32)      # keep the phases of a 64-layer circuit moderate
        b = b.astype(np.float32)
        psi, ex, ti, tp = solve(q, c, Q32, g, b, 4)
        Qd = Q32.astype(np.float64)
        E = orc.energies(Qd)
        psi_o = orc.state(n, g.astype(np.float64), b.astype(np.float64), E)
        ps = psi.cpu().numpy().reshape(-1, 2)
        psi_g = ps[:, 0].astype(np.float64) + 1j * ps[:, 1]
        # 64 layers of FP32 rotations: the error budget grows with the depth
        assert np.max(np.abs(psi_g - psi_o)) <= 1e-5 * 8
        assert abs(ex - orc.expect(psi_o, E)) <= 1e-5 * 8 * np.abs(Qd).sum()
    finally:
        q.qaoa_destroy(c)


def test_zero_parameters_keep_plus_state(q, ctx, orc):
    for n in (5, 14, 16, 20):
        Q32 = synth.symmetric_q(n, seed=700 + n).astype(np.float32)
        psi, ex, _, _ = solve(q, ctx, Q32, np.zeros(2, np.float32), np.zeros(2, np.float32), 0)
        amp = psi.cpu().numpy().reshape(-1, 2)
        np.testing.assert_allclose(amp[:, 0], 2.0 ** (-n / 2), rtol=0, atol=1e-7)
        np.testing.assert_allclose(amp[:, 1], 0.0, rtol=0, atol=1e-7)
        Qd = Q32.astype(np.float64)
        mean = np.trace(Qd) / 2 + (Qd.sum() - np.trace(Qd)) / 4
        assert abs(ex - mean) <= 1e-5 * np.abs(Qd).sum()


def test_k_equals_all_bitstrings(q, ctx, orc):
    n, k = 4, 16
    Q32 = synth.symmetric_q(n, seed=801).astype(np.float32)
    g, b = synth.random_params(2, seed=802)
    psi, ex, ti, tp = solve(q, ctx, Q32, g.astype(np.float32), b.astype(np.float32), k)
    ps = psi.cpu().numpy().reshape(-1, 2)
    psi_g = ps[:, 0].astype(np.float64) + 1j * ps[:, 1]
    oi, op = orc.topk_probs(orc.probs(psi_g), k)
    np.testing.assert_array_equal(ti.astype(np.uint64), oi)
    np.testing.assert_array_equal(tp, op)
    assert sorted(ti.tolist()) == list(range(16))


def test_empty_and_single_batches(q, ctx):
    qd = torch.zeros(16, device="cuda")
    io = q.make_io(qd, qd, expect=torch.zeros(1, dtype=torch.float64, device="cuda"))
    with pytest.raises(q.QaoaError):
        q.qaoa_batch_run(ctx, q.make_insts([]), io)
    # a batch of one on each tier
    for n in (6, 15, 19):
        Q32 = synth.symmetric_q(n, seed=900 + n).astype(np.float32)
        g, b = synth.random_params(1, seed=901)
        _, ex, _, _ = solve(q, ctx, Q32, g.astype(np.float32), b.astype(np.float32), 0, want_state=False)
        assert np.isfinite(ex)


def test_session_chunking_does_not_change_the_cycle(q, orc):
    # m = 127 runs in one chunk, m = 128 in two; the first 127 sub-QUBOs of the m = 128 cycle are
    # the same draws, and the merge is sequential in sub-QUBO order either way
    N, k, p, K = 300, 12, 2, 4
    Q = synth.symmetric_q(N, seed=11)
    x0 = synth.bits(12, N)
    ctx = q.qaoa_create(0)
    try:
        out = {}
        for m in (127, 128):
            s = q.dqaoa_session_create(ctx, N, m, k, p, K, q.DQAOA_RANDOM, True, (0.3, 0.5), (0.4, 0.2))
            assert len(q.dqaoa_session_plans(s)) == (1 if m < 128 else 2)
            x = x0.copy()
            e, acc = q.dqaoa_session_cycle(s, Q, 1, x, 5, 3)
            ex, cand = q.dqaoa_session_results(s, m, K)
            q.dqaoa_session_destroy(s)
            out[m] = (x, e, cand)
    finally:
        q.qaoa_destroy(ctx)
    for m in (127, 128):
        idx, _ = orc.decompose(Q, x0, m, k, 5, 3, conditioned=True)
        xo, eo, _ = orc.merge(Q, x0, idx, out[m][2])
        np.testing.assert_array_equal(out[m][0], xo)
    np.testing.assert_array_equal(out[127][2], out[128][2][:127])


def batch_states_topk(q, ctx, n, count, k, p, seed, zero=False, dbl=False):
    """One plan over `count` instances of n qubits; returns the final states and the top-k."""
    rt, tt = (np.float64, torch.float64) if dbl else (np.float32, torch.float32)
    Qs, pars = [], []
    for i in range(count):
        Qs.append(synth.symmetric_q(n, seed=seed + i).astype(rt).reshape(-1))
        g, b = synth.random_params(p, seed=seed + 1000 + i)
        if zero:
            g, b = 0.0 * g, 0.0 * b
        pars.append(np.concatenate([g, b]).astype(rt))
    qd = torch.as_tensor(np.concatenate(Qs)).cuda()
    pd = torch.as_tensor(np.concatenate(pars)).cuda()
    psi = torch.zeros(count << (n + 1), dtype=tt, device="cuda")
    ex = torch.zeros(count, dtype=torch.float64, device="cuda")
    ti = torch.zeros(count * k, dtype=torch.int64, device="cuda")
    tp = torch.zeros(count * k, dtype=torch.float64, device="cuda")
    io = q.make_io(qd, pd, expect=ex, topk_idx=ti, topk_prob=tp, k_stride=k, psi=psi)
    rows = [(n, p, k, 0, i * n * n, i * 2 * p, i << n, -1) for i in range(count)]
    plan = q.qaoa_plan_create(ctx, q.make_insts(rows), io, dbl=dbl)
    try:
        q.qaoa_plan_launch(plan)
        torch.cuda.synchronize()
    finally:
        q.qaoa_plan_destroy(plan)
    amps = psi.cpu().numpy().reshape(count, 1 << n, 2).astype(np.float64)
    return amps, ti.cpu().numpy().reshape(count, k), tp.cpu().numpy().reshape(count, k)


def host_topk(a, k):
    # |psi|^2 of the stored amplitudes as the device forms it: two rounded squares, one rounded add
    pr = a[:, 0] * a[:, 0] + a[:, 1] * a[:, 1]
    order = np.lexsort((np.arange(pr.size), -pr))[:k]
    return order, pr[order]


# The last streaming pass hands each block a run of consecutive tiles and carries one top-k list
# across the tiles of a state. These cases make the runs cross state boundaries (40 states of 32
# tiles), run long inside one state (n = 24), tie every probability (zero angles: the candidate
# buffer overflows on every tile), and use FP64 states. The list must equal the top-k of the
# returned state, bit for bit.
@pytest.mark.parametrize("n,count,k,p,zero,dbl", [
    (18, 40, 8, 2, False, False),
    (18, 40, 16, 1, False, False),
    (24, 1, 8, 2, False, False),
    (18, 40, 8, 1, True, False),
    (17, 48, 5, 2, False, True),
])
def test_stream_topk_runs(q, ctx, n, count, k, p, zero, dbl):
    amps, ti, tp = batch_states_topk(q, ctx, n, count, k, p, 1300 + n, zero=zero, dbl=dbl)
    for i in range(count):
        oi, op = host_topk(amps[i], k)
        np.testing.assert_array_equal(ti[i].astype(np.int64), oi)
        np.testing.assert_array_equal(tp[i], op)
    if zero:
        assert (ti == np.arange(k)[None, :]).all()
