"""Host DQAOA steps of libqaoa (index draws, sub-QUBO matrices, merge) against the FP64 oracle:
bit-exact on integer results and on the FP64 sub-QUBO matrices. Host code only, no GPU."""
import numpy as np
import pytest

import synth
import paper_2506_10531_gb300 as q


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_10531_gb300 import build
    build.build()


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
        np.testing.assert_array_equal(q_l, q_o)          # same FP64 sums in the same order


def test_ifd_decompose_bit_exact(orc):
    N, m, k = 300, 45, 20
    Q = synth.symmetric_q(N, seed=4)
    x = synth.bits(5, N)
    for flag, oflag in ((0, 0), (q.DQAOA_SIGNED_IMPACT, orc.SIGNED)):
        i_l, q_l = lib_decompose(Q, x, m, k, 0, 0, q.DQAOA_IFD | flag, True)
        i_o, q_o = orc.decompose(Q, x, m, k, 0, 0, method=orc.IFD | oflag, conditioned=True)
        np.testing.assert_array_equal(i_l, i_o)
        np.testing.assert_array_equal(q_l, q_o)


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
            np.testing.assert_array_equal(q_l, q_o)


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
