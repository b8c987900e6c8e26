"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (complex64 path): max |psi_gpu - psi_oracle| <= 1e-5, |d<C>| <= 1e-5 * sum|Q_ij|,
energies within 1e-5 * sum|Q_ij|; top-k indices bit-exact when ranked on the GPU's own stored
amplitudes (both sides rank the same exact FP64 probabilities), and within the near-tie rule
against the oracle's FP64 state. complex128 path: 1e-12 on amplitudes.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5


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
    q.qaoa_reserve(c, q.qaoa_workspace_bytes(22))
    yield c
    q.qaoa_destroy(c)


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_state(q, ctx, Q32, gamma, beta, dbl=False):
    n = Q32.shape[0]
    rt = torch.float64 if dbl else torch.float32
    Qd = dev(Q32, rt)
    E = torch.empty(1 << n, dtype=rt, device="cuda")
    psi = torch.empty(2 << n, dtype=rt, device="cuda")
    g, b = dev(gamma, rt), dev(beta, rt)
    q.qaoa_build_energies(ctx, n, Qd, E, dbl=dbl)
    q.qaoa_run_layers(ctx, n, len(gamma), g, b, E, psi, True, dbl=dbl)
    torch.cuda.synchronize()
    ps = psi.cpu().numpy().reshape(-1, 2)
    return E.cpu().numpy(), ps[:, 0].astype(np.float64) + 1j * ps[:, 1], psi, E


def check_topk(orc, psi_gpu_c, psi_orc, idx, prob, k):
    # (1) exact: the oracle ranks the GPU's stored amplitudes with the same FP64 probabilities
    oi, op = orc.topk_probs(orc.probs(psi_gpu_c), k)
    np.testing.assert_array_equal(idx, oi)
    np.testing.assert_array_equal(prob, op)
    # (2) against the FP64 state: equal where the oracle's gaps exceed eps, else within eps
    pr = np.abs(psi_orc) ** 2
    eps = 4 * AMP_TOL * np.sqrt(pr.max())
    ri, rp = orc.topk_probs(pr, k)
    for j in range(k):
        gap_ok = (j == 0 or rp[j - 1] - rp[j] > eps) and (j == k - 1 or rp[j] - rp[j + 1] > eps)
        if gap_ok:
            assert int(idx[j]) == int(ri[j])
        else:
            assert abs(pr[int(idx[j])] - rp[j]) <= eps


@pytest.mark.parametrize("n,p", [(1, 1), (2, 3), (3, 2), (4, 1), (5, 3), (6, 8), (8, 2), (10, 1),
                                 (11, 4), (13, 3), (14, 2), (14, 5)])
def test_resident_layers_expect_topk(q, ctx, orc, n, p):
    Q = synth.symmetric_q(n, seed=1000 + n)
    Q32 = Q.astype(np.float32)
    Qd = Q32.astype(np.float64)
    g, b = synth.random_params(p, seed=2000 + n)
    g32, b32 = g.astype(np.float32), b.astype(np.float32)
    E_g, psi_g, psi_t, E_t = gpu_state(q, ctx, Q32, g32, b32)
    E_o = orc.energies(Qd)
    absq = np.abs(Qd).sum()
    assert np.max(np.abs(E_g - E_o)) <= 1e-5 * absq
    psi_o = orc.state(n, g32.astype(np.float64), b32.astype(np.float64), E_o)
    assert np.max(np.abs(psi_g - psi_o)) <= AMP_TOL
    # <C> and top-k through the standalone reductions
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    k = min(8, 1 << n)
    idx = torch.zeros(k, dtype=torch.int64, device="cuda")
    prob = torch.zeros(k, dtype=torch.float64, device="cuda")
    q.qaoa_expect(ctx, n, psi_t, E_t, out)
    q.qaoa_topk(ctx, n, psi_t, k, idx, prob)
    torch.cuda.synchronize()
    assert abs(out.item() - orc.expect(psi_o, E_o)) <= 1e-5 * absq
    check_topk(orc, psi_g, psi_o, idx.cpu().numpy().astype(np.uint64), prob.cpu().numpy(), k)


@pytest.mark.parametrize("n,p", [(15, 1), (16, 3), (17, 2), (19, 2), (22, 1)])
def test_streaming_layers(q, ctx, orc, n, p):
    Q = synth.symmetric_q(n, seed=3000 + n)
    Q32 = Q.astype(np.float32)
    Qd = Q32.astype(np.float64)
    g, b = synth.random_params(p, seed=4000 + n)
    g32, b32 = g.astype(np.float32), b.astype(np.float32)
    E_g, psi_g, psi_t, E_t = gpu_state(q, ctx, Q32, g32, b32)
    E_o = orc.energies(Qd)
    absq = np.abs(Qd).sum()
    assert np.max(np.abs(E_g - E_o)) <= 1e-5 * absq
    psi_o = orc.state(n, g32.astype(np.float64), b32.astype(np.float64), E_o)
    assert np.max(np.abs(psi_g - psi_o)) <= AMP_TOL
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    q.qaoa_expect(ctx, n, psi_t, E_t, out)
    torch.cuda.synchronize()
    assert abs(out.item() - orc.expect(psi_o, E_o)) <= 1e-5 * absq


@pytest.mark.parametrize("n,p", [(1, 2), (6, 3), (10, 1), (13, 2), (14, 1), (16, 2)])
def test_complex128_layers(q, ctx, orc, n, p):
    Q = synth.symmetric_q(n, seed=5000 + n)
    g, b = synth.random_params(p, seed=6000 + n)
    E_g, psi_g, psi_t, E_t = gpu_state(q, ctx, Q, g, b, dbl=True)
    E_o = orc.energies(Q)
    np.testing.assert_allclose(E_g, E_o, atol=1e-12 * np.abs(Q).sum())
    psi_o = orc.state(n, g, b, E_o)
    assert np.max(np.abs(psi_g - psi_o)) <= 1e-12
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    q.qaoa_expect(ctx, n, psi_t, E_t, out, dbl=True)
    torch.cuda.synchronize()
    assert out.item() == pytest.approx(orc.expect(psi_o, E_o), abs=1e-11 * np.abs(Q).sum())


@pytest.mark.parametrize("n,p", [(1, 1), (3, 2), (7, 3), (10, 2), (13, 4), (14, 2), (15, 3), (17, 2),
                                 (20, 1)])
def test_grad_vs_oracle(q, ctx, orc, n, p):
    Q = synth.symmetric_q(n, seed=7000 + n, dist="normal")
    Q32 = Q.astype(np.float32)
    Qd = Q32.astype(np.float64)
    g, b = synth.random_params(p, seed=8000 + n)
    g32, b32 = g.astype(np.float32), b.astype(np.float32)
    E = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    q.qaoa_build_energies(ctx, n, dev(Q32), E)
    ex = torch.zeros(1, dtype=torch.float64, device="cuda")
    dg = torch.zeros(p, dtype=torch.float64, device="cuda")
    db = torch.zeros(p, dtype=torch.float64, device="cuda")
    q.qaoa_grad(ctx, n, p, dev(g32), dev(b32), E, ex, dg, db)
    torch.cuda.synchronize()
    E_o = orc.energies(Qd)
    e_o, dg_o, db_o = orc.grad(n, g32.astype(np.float64), b32.astype(np.float64), E_o)
    absq = np.abs(Qd).sum()
    assert abs(ex.item() - e_o) <= 1e-5 * absq
    ref = np.concatenate([dg_o, db_o])
    got = np.concatenate([dg.cpu().numpy(), db.cpu().numpy()])
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(np.max(np.abs(ref)), 1.0) * max(1.0, n / 4)


@pytest.mark.parametrize("n,p", [(9, 3), (14, 2)])
def test_grad_complex128(q, ctx, orc, n, p):
    Q = synth.symmetric_q(n, seed=71)
    g, b = synth.random_params(p, seed=72)
    E = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    q.qaoa_build_energies(ctx, n, dev(Q), E, dbl=True)
    ex = torch.zeros(1, dtype=torch.float64, device="cuda")
    dg = torch.zeros(p, dtype=torch.float64, device="cuda")
    db = torch.zeros(p, dtype=torch.float64, device="cuda")
    q.qaoa_grad(ctx, n, p, dev(g), dev(b), E, ex, dg, db, dbl=True)
    torch.cuda.synchronize()
    e_o, dg_o, db_o = orc.grad(n, g, b, orc.energies(Q))
    assert ex.item() == pytest.approx(e_o, abs=1e-11)
    np.testing.assert_allclose(dg.cpu().numpy(), dg_o, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(db.cpu().numpy(), db_o, rtol=1e-10, atol=1e-11)


def test_plain_path(q, ctx, orc):
    n, p, k = 12, 2, 8
    Q32 = synth.symmetric_q(n, seed=81).astype(np.float32)
    g32, b32 = (v.astype(np.float32) for v in synth.random_params(p, seed=82))
    E = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    psi = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    ex = torch.zeros(1, dtype=torch.float64, device="cuda")
    idx = torch.zeros(k, dtype=torch.int64, device="cuda")
    prob = torch.zeros(k, dtype=torch.float64, device="cuda")
    q.qaoa_plain_solve(ctx, n, p, dev(Q32), dev(g32), dev(b32), E, psi, k, ex, idx, prob)
    torch.cuda.synchronize()
    E_o = orc.energies(Q32.astype(np.float64))
    psi_o = orc.state(n, g32.astype(np.float64), b32.astype(np.float64), E_o)
    ps = psi.cpu().numpy().reshape(-1, 2)
    psi_g = ps[:, 0].astype(np.float64) + 1j * ps[:, 1]
    assert np.max(np.abs(psi_g - psi_o)) <= AMP_TOL
    assert abs(ex.item() - orc.expect(psi_o, E_o)) <= 1e-5 * np.abs(Q32).sum()
    check_topk(orc, psi_g, psi_o, idx.cpu().numpy().astype(np.uint64), prob.cpu().numpy(), k)


@pytest.mark.parametrize("cond", [False, True])
def test_subqubo_build(q, ctx, orc, cond):
    # device FP32 sub-QUBO matrices: copied entries equal the FP32 rounding of Q exactly; the
    # conditioned diagonal lies within half an FP32 ulp of the oracle's FP64 sum plus the bound of
    # two FP64 summation orders (the device and the oracle add the same terms in different orders)
    from test_dqaoa_host import qsub_diag_bound
    N, m, k = 1000, 64, 16
    Q = synth.symmetric_q(N, seed=2)
    x = synth.bits(3, N)
    idx, qs_o = orc.decompose(Q, x, m, k, seed=2, cycle=1, conditioned=cond)
    out = torch.zeros(m * k * k, dtype=torch.float32, device="cuda")
    q.dqaoa_subqubo_build(ctx, dev(Q), N, dev(x), m, k, dev(idx), cond, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(m, k, k).astype(np.float64)
    b64 = qsub_diag_bound(Q, x, idx, cond)
    bound = np.where(b64 > 0, b64 + 0.5 * np.spacing(np.abs(qs_o + b64).astype(np.float32)).astype(np.float64), 0.0)
    want = np.where(b64 > 0, qs_o, qs_o.astype(np.float32).astype(np.float64))
    diff = np.abs(got - want)
    assert not (diff > bound).any(), f"{int((diff > bound).sum())} entries beyond the FP32 rounding bound"
    differ = int((got != qs_o.astype(np.float32)).sum())
    print(f"conditioned={cond}: {differ} of {got.size} FP32 entries differ from fl32(oracle)")


@pytest.mark.parametrize("n", [1, 2, 3, 7, 12, 14, 17, 21])
def test_energies_nonsymmetric_q(q, ctx, orc, n):
    # E(z) = z^T Q z uses Q_ij and Q_ji as separate terms (Section IV): a non-symmetric Q
    rng = np.random.default_rng(900 + n)
    Q32 = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    E = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    q.qaoa_build_energies(ctx, n, dev(Q32), E)
    Ed = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    q.qaoa_build_energies(ctx, n, dev(Q32, torch.float64), Ed, dbl=True)
    torch.cuda.synchronize()
    E_o = orc.energies(Q32.astype(np.float64))
    absq = np.abs(Q32).sum()
    assert np.max(np.abs(E.cpu().numpy() - E_o)) <= 1e-5 * absq
    assert np.max(np.abs(Ed.cpu().numpy() - E_o)) <= 1e-12 * absq


def test_energies_unaligned_pointer(q, ctx, orc):
    # an energy array that is 8- but not 16-byte aligned takes the narrow stores
    n = 16
    Q32 = synth.symmetric_q(n, seed=77).astype(np.float32)
    buf = torch.zeros((1 << n) + 2, dtype=torch.float32, device="cuda")
    q.qaoa_build_energies(ctx, n, dev(Q32), buf[2:])
    torch.cuda.synchronize()
    E_o = orc.energies(Q32.astype(np.float64))
    assert np.max(np.abs(buf[2:].cpu().numpy() - E_o)) <= 1e-5 * np.abs(Q32).sum()
    assert buf[0].item() == 0.0 and buf[1].item() == 0.0
