"""The measured configurations end to end through the C ABI, against the FP64 oracle.

* Plain n = 10 grid (complex128): 256 (gamma, beta) points of a 16 x 16 grid as one batch of
  resident instances that share Q; <C>, top-8 and the energies against the oracle, the argmin of
  the energies against brute force over all 1024 bitstrings.
* Large instance: the n = 30, p = 2 streaming configuration, checked where the oracle cannot
  follow by properties that hold at any size (energies sampled one by one against x^T Q x, norm,
  top-k consistent with the returned state, the uniform mean at gamma = 0, the closed-form p = 1
  Ising expectation), and its n = 26 twin (same generator, same seed) against the full FP64
  oracle state.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_oracle_pins import closed_form_p1  # noqa: E402


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


def run_single_plan(q, ctx, Q32, gamma, beta, k, want_state=True, dbl=False):
    """One instance through a batch plan (the fused streaming path); returns device buffers."""
    n = Q32.shape[0]
    rt = torch.float64 if dbl else torch.float32
    qd = torch.as_tensor(np.ascontiguousarray(Q32)).to(rt).cuda().reshape(-1)
    pd = torch.as_tensor(np.concatenate([gamma, beta])).to(rt).cuda()
    psi = torch.empty(2 << n, dtype=rt, device="cuda") if want_state else None
    E = torch.empty(1 << n, dtype=rt, device="cuda")
    ex = torch.zeros(1, dtype=torch.float64, device="cuda")
    ti = torch.zeros(max(k, 1), dtype=torch.int64, device="cuda")
    tp = torch.zeros(max(k, 1), dtype=torch.float64, device="cuda")
    io = q.make_io(qd, pd, expect=ex, topk_idx=ti, topk_prob=tp, k_stride=k, psi=psi, e=E)
    insts = q.make_insts([(n, len(gamma), k, 0, 0, 0, 0 if want_state else -1, 0)])
    q.qaoa_batch_run(ctx, insts, io, dbl=dbl)
    torch.cuda.synchronize()
    return psi, E, ex, ti, tp


# ---------------------------------------------------------------------------------------------
# Plain n = 10, complex128, 16 x 16 grid
# ---------------------------------------------------------------------------------------------

def test_plain_grid_complex128(q, ctx, orc):
    n, k = 10, 8
    Q = synth.symmetric_q(n, seed=1)
    gg, bb = synth.grid_params(16)
    count = gg.size
    qd = torch.as_tensor(Q.reshape(-1)).cuda()
    pd = torch.as_tensor(np.stack([gg, bb], axis=1).reshape(-1)).cuda()
    E = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    ex = torch.zeros(count, dtype=torch.float64, device="cuda")
    ti = torch.zeros(count * k, dtype=torch.int64, device="cuda")
    tp = torch.zeros(count * k, dtype=torch.float64, device="cuda")
    io = q.make_io(qd, pd, expect=ex, topk_idx=ti, topk_prob=tp, k_stride=k, e=E)
    # every grid point shares Q (q_off 0); the first instance also returns the energies
    rows = [(n, 1, k, 0, 0, 2 * i, -1, 0 if i == 0 else -1) for i in range(count)]
    q.qaoa_batch_run(ctx, q.make_insts(rows), io, dbl=True)
    torch.cuda.synchronize()
    E_o = orc.energies(Q)
    absq = np.abs(Q).sum()
    np.testing.assert_allclose(E.cpu().numpy(), E_o, rtol=0, atol=1e-12 * absq)
    # brute force over all 2^10 bitstrings: the minimum and where it is
    z = np.arange(1 << n)
    brute = np.array([orc.qubo_energy(Q, ((int(v) >> np.arange(n)) & 1).astype(np.uint8)) for v in z])
    assert int(np.argmin(E.cpu().numpy())) == int(np.argmin(brute))
    assert E.cpu().numpy().min() == pytest.approx(brute.min(), abs=1e-12 * absq)
    exh, tih, tph = ex.cpu().numpy(), ti.cpu().numpy().reshape(count, k), tp.cpu().numpy().reshape(count, k)
    for i in range(count):
        psi_o = orc.state(n, [gg[i]], [bb[i]], E_o)
        assert exh[i] == pytest.approx(orc.expect(psi_o, E_o), abs=1e-11 * absq), i
        pr = orc.probs(psi_o)
        ri, rp = orc.topk_probs(pr, k)
        np.testing.assert_allclose(tph[i], rp, rtol=0, atol=1e-12)
        for j in range(k):
            # indices equal unless the FP64 probabilities are within rounding of a neighbour
            tie = (j > 0 and rp[j - 1] - rp[j] <= 1e-12) or (j < k - 1 and rp[j] - rp[j + 1] <= 1e-12)
            if not tie:
                assert int(tih[i, j]) == int(ri[j]), (i, j)
            else:
                assert abs(pr[int(tih[i, j])] - rp[j]) <= 1e-12


# ---------------------------------------------------------------------------------------------
# Large instance (streaming): n = 30 properties and the n = 26 twin
# ---------------------------------------------------------------------------------------------

LARGE = dict(seed=5, p=2, gamma=(0.4, 0.7), beta=(0.6, 0.3), k=8)


def test_large_twin_n26_vs_oracle(q, ctx, orc):
    n = 26
    Q = synth.symmetric_q(n, seed=LARGE["seed"])
    Q32 = Q.astype(np.float32)
    g = np.array(LARGE["gamma"], dtype=np.float32)
    b = np.array(LARGE["beta"], dtype=np.float32)
    psi, E, ex, ti, tp = run_single_plan(q, ctx, Q32, g, b, LARGE["k"])
    Qd = Q32.astype(np.float64)
    E_o = orc.energies(Qd)
    absq = np.abs(Qd).sum()
    assert np.max(np.abs(E.cpu().numpy() - E_o)) <= 1e-5 * absq
    psi_o = orc.state(n, g.astype(np.float64), b.astype(np.float64), E_o)
    ps = psi.cpu().numpy().reshape(-1, 2)
    psi_g = ps[:, 0].astype(np.float64) + 1j * ps[:, 1]
    assert np.max(np.abs(psi_g - psi_o)) <= 1e-5
    assert abs(ex.item() - orc.expect(psi_o, E_o)) <= 1e-5 * absq
    # top-k: exact against the oracle's ranking of the GPU's own amplitudes
    oi, op = orc.topk_probs(orc.probs(psi_g), LARGE["k"])
    np.testing.assert_array_equal(ti.cpu().numpy().astype(np.uint64), oi)
    np.testing.assert_array_equal(tp.cpu().numpy(), op)
    # the single-instance entry points agree with the fused plan
    ex2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    psi2 = torch.empty_like(psi)
    E2 = torch.empty_like(E)
    q.qaoa_build_energies(ctx, n, torch.as_tensor(Q32).cuda(), E2)
    q.qaoa_reserve(ctx, q.qaoa_workspace_bytes(n))
    q.qaoa_run_layers(ctx, n, 2, torch.as_tensor(g).cuda(), torch.as_tensor(b).cuda(), E2, psi2, True)
    q.qaoa_expect(ctx, n, psi2, E2, ex2)
    torch.cuda.synchronize()
    assert torch.equal(E2, E)
    assert torch.max(torch.abs(psi2 - psi)).item() <= 1e-6
    assert abs(ex2.item() - ex.item()) <= 1e-6 * absq


def test_large_n30_properties(q, ctx, orc):
    n = 30
    Q = synth.symmetric_q(n, seed=LARGE["seed"])
    Q32 = Q.astype(np.float32)
    Qd = Q32.astype(np.float64)
    absq = np.abs(Qd).sum()
    g = np.array(LARGE["gamma"], dtype=np.float32)
    b = np.array(LARGE["beta"], dtype=np.float32)
    k = LARGE["k"]
    psi, E, ex, ti, tp = run_single_plan(q, ctx, Q32, g, b, k)
    # energies, sampled one by one against x^T Q x in FP64
    zs = (synth.splitmix64(55, 4096) >> np.uint64(34)).astype(np.int64)
    Eh = E[torch.as_tensor(zs).cuda()].cpu().numpy()
    for z, e in zip(zs, Eh):
        x = ((int(z) >> np.arange(n)) & 1).astype(np.uint8)
        assert abs(e - orc.qubo_energy(Qd, x)) <= 1e-5 * absq
    # norm (FP64 sum of the squared components, in chunks)
    v = psi.view(-1)
    tot = 0.0
    for c0 in range(0, v.numel(), 1 << 28):
        tot += float(torch.sum(v[c0:c0 + (1 << 28)].double() ** 2).item())
    assert tot == pytest.approx(1.0, abs=1e-4)
    # top-k consistent with the returned state: probabilities are those of the returned
    # amplitudes and no amplitude outside the list is more probable than the last entry
    idx = ti.cpu().numpy()
    pv = psi.view(-1, 2)
    pr_sel = (pv[torch.as_tensor(idx).cuda()].double() ** 2).sum(dim=1).cpu().numpy()
    np.testing.assert_array_equal(pr_sel, tp.cpu().numpy())
    assert np.all(np.diff(tp.cpu().numpy()) <= 0)
    worse = 0
    for c0 in range(0, pv.shape[0], 1 << 27):
        chunk = (pv[c0:c0 + (1 << 27)].double() ** 2).sum(dim=1)
        mask = torch.ones_like(chunk, dtype=torch.bool)
        sel = [int(i) - c0 for i in idx if c0 <= int(i) < c0 + chunk.numel()]
        if sel:
            mask[torch.as_tensor(sel).cuda()] = False
        worse += int((chunk[mask] > tp[-1]).sum().item())
    assert worse == 0
    del psi, E
    torch.cuda.empty_cache()
    # gamma = 0: uniform probabilities, <C> = tr(Q)/2 + sum_{i != j} Q_ij / 4
    _, _, ex0, _, _ = run_single_plan(q, ctx, Q32, np.zeros(2, np.float32), b, 0, want_state=False)
    mean = np.trace(Qd) / 2 + (Qd.sum() - np.trace(Qd)) / 4
    assert abs(ex0.item() - mean) <= 1e-5 * absq
    # closed-form p = 1 expectation of a field-free Ising cost at n = 30
    Qm = synth.maxcut_form_q(n, seed=6, edge_prob=0.3).astype(np.float32)
    Qmd = Qm.astype(np.float64)
    gm, bm = np.float32(0.37), np.float32(0.21)
    _, _, exm, _, _ = run_single_plan(q, ctx, Qm, np.array([gm]), np.array([bm]), 0, want_state=False)
    ref = closed_form_p1(Qmd, float(gm), float(bm))
    assert abs(exm.item() - ref) <= 1e-5 * np.abs(Qmd).sum()
