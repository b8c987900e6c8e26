"""Host DQAOA steps of libqaoa (index draws, sub-QUBO matrices, merge) against the FP64 oracle:
bit-exact on integer results and on the copied entries of the sub-QUBO matrices; the conditioned
diagonal (a sum of up to N FP64 terms, whose order the paper does not fix) within the rounding
bound of two summation orders. Host code only, no GPU."""
import numpy as np
import pytest

import synth
import paper_2506_10531_gb300 as q


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_10531_gb300 import build
    build.build()


U64 = 2.0 ** -53


def qsub_diag_bound(Q, x, idx, conditioned):
    """Per-entry bound on |Qsub_lib - Qsub_oracle| for m x k x k sub-QUBO matrices.

    Off-diagonal entries are copies of Q (bound 0). A conditioned diagonal entry is
    Q_aa + 2 sum_{l not in S, x_l = 1} Q[S_a][l]: two FP64 summation orders of the same A terms
    (absolute sum T) each lie within (A-1) u T of the exact sum (Higham, Accuracy and Stability,
    eq. 4.4), and the final doubling and addition round once more."""
    m, k = idx.shape
    bound = np.zeros((m, k, k))
    if not conditioned:
        return bound
    N = Q.shape[0]
    xs = np.asarray(x, dtype=bool)
    for j in range(m):
        out = xs.copy()
        out[idx[j]] = False
        for a in range(k):
            T = float(np.abs(Q[idx[j][a], out]).sum())
            A = int(out.sum())
            bound[j, a, a] = 2.0 * (2.0 * A * U64 * T) + 4.0 * U64 * (abs(Q[idx[j][a], idx[j][a]]) + 2.0 * T)
    return bound


def assert_qsub_close(got, want, bound, what=""):
    """Element-wise |got - want| <= bound; copies (bound 0) must be equal. Returns how many
    entries differ at all (reported by the callers)."""
    diff = np.abs(got - want)
    bad = diff > bound
    assert not bad.any(), f"{what}: {int(bad.sum())} entries beyond the rounding bound, max excess " \
                          f"{float((diff - bound)[bad].max())}"
    return int((diff > 0).sum())


def lib_decompose(Q, x, m, k, seed, cycle, method, conditioned):
    N = Q.shape[0]
    idx = np.zeros((m, k), dtype=np.int32)
    qs = np.zeros((m, k, k))
    q.dqaoa_decompose(np.ascontiguousarray(Q), N, None if x is None else np.ascontiguousarray(x),
                      method, conditioned, m, k, seed, cycle, idx, qs)
    return idx, qs


@pytest.mark.parametrize("N,m,k,seed,cycle", [(1000, 256, 16, 2, 0), (300, 160, 20, 7, 5),
                                               (17, 40, 17, 1, 1), (50, 3, 1, 9, 2)])
def test_random_decompose_bit_exact(orc, N, m, k, seed, cycle):
    Q = synth.symmetric_q(N, seed=seed)
    x = synth.bits(seed + 100, N)
    for cond in (False, True):
        i_l, q_l = lib_decompose(Q, x, m, k, seed, cycle, q.DQAOA_RANDOM, cond)
        i_o, q_o = orc.decompose(Q, x, m, k, seed, cycle, method=orc.RANDOM, conditioned=cond)
        np.testing.assert_array_equal(i_l, i_o)
        nd = assert_qsub_close(q_l, q_o, qsub_diag_bound(Q, x, i_o, cond), f"cond={cond}")
        print(f"N={N} m={m} k={k} conditioned={cond}: {nd} of {q_o.size} entries differ by rounding")


def test_ifd_decompose_bit_exact(orc):
    N, m, k = 300, 45, 20
    Q = synth.symmetric_q(N, seed=4)
    x = synth.bits(5, N)
    for flag, oflag in ((0, 0), (q.DQAOA_SIGNED_IMPACT, orc.SIGNED)):
        i_l, q_l = lib_decompose(Q, x, m, k, 0, 0, q.DQAOA_IFD | flag, True)
        i_o, q_o = orc.decompose(Q, x, m, k, 0, 0, method=orc.IFD | oflag, conditioned=True)
        np.testing.assert_array_equal(i_l, i_o)
        assert_qsub_close(q_l, q_o, qsub_diag_bound(Q, x, i_o, True), "IFD")


@pytest.mark.parametrize("kind,N,m,k", [("maxcut", 400, 200, 12), ("dense", 300, 300, 20),
                                         ("sparse", 120, 120, 12), ("maxcut", 60, 60, 2)])
def test_bfs_pfs_decompose_bit_exact(orc, kind, N, m, k):
    if kind == "maxcut":
        Q = synth.maxcut_graph_q(N, seed=21)
    elif kind == "sparse":
        Q = synth.maxcut_graph_q(N, seed=22, edges=N // 2)     # many components: restarts
    else:
        Q = synth.symmetric_q(N, seed=23)
    x = synth.bits(24, N)
    for flag, oflag in ((0, 0), (q.DQAOA_SIGNED_IMPACT, orc.SIGNED)):
        for lm, om in ((q.DQAOA_BFS, orc.BFS), (q.DQAOA_PFS, orc.PFS)):
            i_l, q_l = lib_decompose(Q, x, m, k, 0, 0, lm | flag, True)
            i_o, q_o = orc.decompose(Q, x, m, k, 0, 0, method=om | oflag, conditioned=True)
            np.testing.assert_array_equal(i_l, i_o)
            assert_qsub_close(q_l, q_o, qsub_diag_bound(Q, x, i_o, True), f"{kind} method {lm}")


def test_draw_indices_worked_examples():
    # the library's draw against the index sets worked by hand from published SplitMix64
    # outputs (tests/golden/random_draw.json; Section V-A random selection, reading O5)
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "random_draw.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        N, k, j = c["N"], c["k"], c["j"]
        idx = np.zeros((j + 1, k), dtype=np.int32)
        q.dqaoa_draw_indices(None, N, None, q.DQAOA_RANDOM, j + 1, k, int(c["seed"]), c["cycle"], idx)
        assert list(idx[j]) == c["S_sorted"], c["note"]


def test_draw_indices_matches_decompose(orc):
    N, m, k = 1000, 64, 16
    idx = np.zeros((m, k), dtype=np.int32)
    q.dqaoa_draw_indices(None, N, None, q.DQAOA_RANDOM, m, k, 11, 3, idx)
    i_o, _ = orc.decompose(np.zeros((N, N)), None, m, k, 11, 3, conditioned=False)
    np.testing.assert_array_equal(idx, i_o)


@pytest.mark.parametrize("N,m,k,K,seed", [(1000, 256, 16, 8, 2), (200, 60, 12, 16, 3), (16, 4, 16, 8, 5)])
def test_merge_bit_exact(orc, N, m, k, K, seed):
    Q = synth.symmetric_q(N, seed=seed)
    x0 = synth.bits(seed + 1, N)
    idx, _ = orc.decompose(Q, x0, m, k, seed, 0)
    cand = (synth.splitmix64(seed + 2, m * K) & np.uint64((1 << k) - 1)).reshape(m, K)
    xo, eo, ao = orc.merge(Q, x0, idx, cand)
    xl = x0.copy()
    el, al = q.dqaoa_merge(np.ascontiguousarray(Q), N, xl, m, k, np.ascontiguousarray(idx), K,
                           np.ascontiguousarray(cand))
    np.testing.assert_array_equal(xl, xo)
    assert al == ao
    assert el == pytest.approx(eo, abs=1e-9 * np.abs(Q).sum())
    assert el == pytest.approx(orc.qubo_energy(Q, xl), abs=1e-9 * np.abs(Q).sum())


def test_host_argument_errors():
    with pytest.raises(q.QaoaError) as e:
        q.dqaoa_draw_indices(None, 10, None, q.DQAOA_RANDOM, 4, 11, 0, 0, np.zeros(44, np.int32))
    assert e.value.status == q.QAOA_E_INVALID
    with pytest.raises(q.QaoaError):
        q.dqaoa_draw_indices(None, 10, None, q.DQAOA_IFD, 4, 3, 0, 0, np.zeros(12, np.int32))
    Qz, xz = np.zeros((10, 10)), np.zeros(10, np.uint8)
    for meth in (q.DQAOA_BFS, q.DQAOA_PFS):
        with pytest.raises(q.QaoaError):          # m > N
            q.dqaoa_draw_indices(Qz, 10, xz, meth, 11, 3, 0, 0, np.zeros(33, np.int32))
        with pytest.raises(q.QaoaError):          # needs Q and x
            q.dqaoa_draw_indices(None, 10, None, meth, 4, 3, 0, 0, np.zeros(12, np.int32))
    with pytest.raises(q.QaoaError):
        q.dqaoa_draw_indices(Qz, 10, xz, 4, 4, 3, 0, 0, np.zeros(12, np.int32))
    for bad in (q.DQAOA_RANDOM | q.DQAOA_SIGNED_IMPACT, q.DQAOA_IFD | 32, 4 | q.DQAOA_SIGNED_IMPACT):
        with pytest.raises(q.QaoaError):
            q.dqaoa_draw_indices(Qz, 10, xz, bad, 4, 3, 0, 0, np.zeros(12, np.int32))
    idx = np.array([[0, 12]], dtype=np.int32)
    with pytest.raises(q.QaoaError):
        q.dqaoa_merge(np.zeros((10, 10)), 10, np.zeros(10, np.uint8), 1, 2, idx, 1,
                      np.zeros(1, np.uint64))
