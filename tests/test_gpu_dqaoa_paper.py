"""Paper-literal pieces of the DQAOA session (Section IV), against the FP64 oracle:

* DQAOA_PAPER_MIXER: the ansatz with the printed mixer H_X = -sum X. Every sub-QUBO's <C> and
  top-K match the oracle's state with mixer_sign = -1 (and the default session matches
  mixer_sign = +1); the merged solution equals the oracle's merge of the session's candidates.
* dqaoa_session_cycle_sampled: sub-solutions read from measured shots. The shots equal the
  oracle's inverse-CDF sampling of the session's own final states for the same uniforms (a shot
  may differ only where the target sits within rounding of a CDF boundary), the states match the
  oracle's, the chosen candidate is the shot of lowest FP64 sub-QUBO energy (the oracle's
  conditioned sub-QUBO), and the merged solution equals the oracle's merge of those candidates
  bit for bit.
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


def f32(v):
    return np.array(v, dtype=np.float32).astype(np.float64)


def check_topk(orc, psi_o, cand_row, K, j):
    pr = orc.probs(psi_o)
    eps = 4e-5 * np.sqrt(pr.max())
    ri, rp = orc.topk_probs(pr, K)
    for t in range(K):
        clear = (t == 0 or rp[t - 1] - rp[t] > eps) and (t == K - 1 or rp[t] - rp[t + 1] > eps)
        if clear:
            assert int(cand_row[t]) == int(ri[t]), (j, t)
        else:
            assert abs(pr[int(cand_row[t])] - rp[t]) <= eps, (j, t)


def test_session_paper_mixer_sign(q, orc):
    N, m, k, p, K = 200, 16, 12, 2, 4
    Q = synth.symmetric_q(N, seed=41)
    x0 = synth.bits(42, N)
    g, b = [0.3, 0.7], [0.5, 0.2]
    res = {}
    ctx = q.qaoa_create(0)
    try:
        for flag in (0, q.DQAOA_PAPER_MIXER):
            s = q.dqaoa_session_create(ctx, N, m, k, p, K, q.DQAOA_RANDOM | flag, True, g, b)
            x = x0.copy()
            e, acc = q.dqaoa_session_cycle(s, Q, 1, x, 9, 0)
            ex, cand = q.dqaoa_session_results(s, m, K)
            q.dqaoa_session_destroy(s)
            res[flag] = (x, e, acc, ex, cand)
    finally:
        q.qaoa_destroy(ctx)
    idx, qs = orc.decompose(Q, x0, m, k, 9, 0, conditioned=True)
    for flag, sign in ((0, 1), (q.DQAOA_PAPER_MIXER, -1)):
        x, e, acc, ex, cand = res[flag]
        for j in range(m):
            E = orc.energies(qs[j])
            psi = orc.state(k, f32(g), f32(b), E, mixer_sign=sign)
            assert abs(ex[j] - orc.expect(psi, E)) <= 1e-5 * np.abs(qs[j]).sum(), (sign, j)
            check_topk(orc, psi, cand[j], K, j)
        xo, eo, ao = orc.merge(Q, x0, idx, cand)
        np.testing.assert_array_equal(x, xo)
        assert acc == ao
    # the two mixers are different circuits: <C> moves for most sub-QUBOs
    d = np.abs(res[0][3] - res[q.DQAOA_PAPER_MIXER][3])
    assert np.mean(d > 1e-3) > 0.5, d


def sub_energy(Qs, y, k):
    b = ((int(y) >> np.arange(k)) & 1).astype(np.float64)
    return float(b @ Qs @ b)


@pytest.mark.parametrize("N,m,k,p,shots", [(300, 24, 12, 2, 64), (1000, 40, 16, 3, 200)])
def test_session_sampled_cycle(q, orc, N, m, k, p, shots):
    seed = 77 + k
    Q = synth.symmetric_q(N, seed=seed)
    x0 = synth.bits(seed + 1, N)
    g, b = [0.2, 0.4, 0.6][:p], [0.6, 0.4, 0.2][:p]
    u = synth.uniform01(seed + 2, m * shots).reshape(m, shots)
    ctx = q.qaoa_create(0)
    try:
        s = q.dqaoa_session_create(ctx, N, m, k, p, 4, q.DQAOA_RANDOM, True, g, b)
        x = x0.copy()
        e, acc = q.dqaoa_session_cycle_sampled(s, Q, 1, x, seed, 3, u)
        z, best, psi = q.dqaoa_session_shots(s, m, k, shots, states=True)
        ex, _ = q.dqaoa_session_results(s, m, 4)
        # a second cycle from the merged solution (cached h = Qx) against a fresh oracle merge
        x2 = x.copy()
        u2 = synth.uniform01(seed + 3, m * shots).reshape(m, shots)
        e2, acc2 = q.dqaoa_session_cycle_sampled(s, Q, 0, x2, seed, 4, u2)
        z2, best2, _ = q.dqaoa_session_shots(s, m, k, shots)
        q.dqaoa_session_destroy(s)
    finally:
        q.qaoa_destroy(ctx)
    idx, qs = orc.decompose(Q, x0, m, k, seed, 3, conditioned=True)
    boundary, near_ties = 0, 0
    for j in range(m):
        E = orc.energies(qs[j])
        psi_o = orc.state(k, f32(g), f32(b), E)
        assert np.max(np.abs(psi[j].astype(np.complex128) - psi_o)) <= 1e-5, j
        assert abs(ex[j] - orc.expect(psi_o, E)) <= 1e-5 * np.abs(qs[j]).sum(), j
        # shots: the oracle's sampling of the session's own state
        pr = orc.probs(psi[j].astype(np.complex128))
        zo = orc.sample_probs(pr, u[j])
        cdf = np.cumsum(pr)
        tol = 1e-12 * cdf[-1]
        for i in np.nonzero(z[j] != zo)[0]:
            t = u[j, i] * cdf[-1]
            assert np.min(np.abs(cdf - t)) <= tol, (j, i)
            boundary += 1
        # the candidate: lowest sub-QUBO energy among the shots (ties: smaller bitstring)
        ys = np.unique(z[j])
        es = np.array([sub_energy(qs[j], y, k) for y in ys])
        order = np.lexsort((ys, es))
        bo = ys[order[0]]
        if len(ys) > 1 and es[order[1]] - es[order[0]] <= 1e-9 * np.abs(qs[j]).sum():
            near_ties += 1
            assert abs(sub_energy(qs[j], best[j], k) - es[order[0]]) <= 1e-9 * np.abs(qs[j]).sum(), j
        else:
            assert int(best[j]) == int(bo), (j, int(best[j]), int(bo))
    print(f"shots at CDF boundaries: {boundary}; candidate near-ties: {near_ties}")
    xo, eo, ao = orc.merge(Q, x0, idx, best.reshape(m, 1))
    np.testing.assert_array_equal(x, xo)
    assert acc == ao
    assert e == pytest.approx(eo, abs=1e-9 * np.abs(Q).sum())
    assert e <= orc.qubo_energy(Q, x0)
    idx2, _ = orc.decompose(Q, xo, m, k, seed, 4, conditioned=True)
    xo2, eo2, ao2 = orc.merge(Q, xo, idx2, best2.reshape(m, 1))
    np.testing.assert_array_equal(x2, xo2)
    assert acc2 == ao2
    assert e2 == pytest.approx(eo2, abs=1e-9 * np.abs(Q).sum())


def test_sampled_cycle_edges(q, orc):
    # one shot per sub-QUBO (the shot is the candidate), a single-chunk session (m < 128) with
    # the IFD decomposition and the paper's mixer sign, and a call with more shots than before
    # (the shot buffers grow): merged x bit-exact with the oracle's merge of the chosen shots
    N, m, k, p = 200, 20, 10, 2
    Q = synth.symmetric_q(N, seed=91)
    x0 = synth.bits(92, N)
    g, b = [0.35, 0.6], [0.45, 0.3]
    ctx = q.qaoa_create(0)
    try:
        s = q.dqaoa_session_create(ctx, N, m, k, p, 4, q.DQAOA_IFD | q.DQAOA_PAPER_MIXER, True, g, b)
        x = x0.copy()
        u1 = synth.uniform01(93, m).reshape(m, 1)
        e1, a1 = q.dqaoa_session_cycle_sampled(s, Q, 1, x, 0, 0, u1)
        z1, best1, psi1 = q.dqaoa_session_shots(s, m, k, 1, states=True)
        x_after1 = x.copy()
        u2 = synth.uniform01(94, m * 300).reshape(m, 300)
        e2, a2 = q.dqaoa_session_cycle_sampled(s, Q, 0, x, 0, 1, u2)
        z2, best2, _ = q.dqaoa_session_shots(s, m, k, 300)
        q.dqaoa_session_destroy(s)
    finally:
        q.qaoa_destroy(ctx)
    np.testing.assert_array_equal(best1, z1[:, 0])          # one shot: it is the candidate
    idx1, qs1 = orc.decompose(Q, x0, m, k, 0, 0, method=orc.IFD, conditioned=True)
    for j in range(m):                                      # the paper's mixer: mixer_sign = -1
        E = orc.energies(qs1[j])
        psi_o = orc.state(k, f32(g), f32(b), E, mixer_sign=-1)
        assert np.max(np.abs(psi1[j].astype(np.complex128) - psi_o)) <= 1e-5, j
    xo1, eo1, ao1 = orc.merge(Q, x0, idx1, best1.reshape(m, 1))
    np.testing.assert_array_equal(x_after1, xo1)
    assert a1 == ao1 and e1 == pytest.approx(eo1, abs=1e-9 * np.abs(Q).sum())
    idx2, qs2 = orc.decompose(Q, xo1, m, k, 0, 1, method=orc.IFD, conditioned=True)
    for j in range(m):
        ys = np.unique(z2[j])
        es = np.array([sub_energy(qs2[j], y, k) for y in ys])
        order = np.lexsort((ys, es))
        if len(ys) == 1 or es[order[1]] - es[order[0]] > 1e-9 * np.abs(qs2[j]).sum():
            assert int(best2[j]) == int(ys[order[0]]), j
    xo2, eo2, ao2 = orc.merge(Q, xo1, idx2, best2.reshape(m, 1))
    np.testing.assert_array_equal(x, xo2)
    assert a2 == ao2 and e2 == pytest.approx(eo2, abs=1e-9 * np.abs(Q).sum())
