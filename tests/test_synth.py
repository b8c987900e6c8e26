"""The seeded input generators shared by the oracle and the CUDA path: their definitions checked
against properties that do not depend on the generator's own code (distribution moments, exact
edge counts, the Max-Cut energy identity, grid endpoints, ranges, reproducibility)."""
import itertools

import numpy as np

import synth


def test_reproducible_and_stream_offsets():
    a = synth.splitmix64(99, 10)
    np.testing.assert_array_equal(a, synth.splitmix64(99, 10))
    np.testing.assert_array_equal(a[4:], synth.splitmix64(99, 6, start=4))     # counter-based
    assert not np.array_equal(a, synth.splitmix64(100, 10))


def test_uniform_and_normal_moments():
    u = synth.uniform01(5, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    z = synth.normal(6, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_symmetric_q():
    Q = synth.symmetric_q(50, seed=7)
    np.testing.assert_array_equal(Q, Q.T)
    assert Q.min() >= -1.0 and Q.max() < 1.0
    # the stream fills the upper triangle row-major: entry (0, 0) is the first draw
    assert Q[0, 0] == synth.uniform_pm1(7, 1)[0]


def test_maxcut_graph_q_definition():
    for n, seed in ((40, 1), (101, 2)):
        Q = synth.maxcut_graph_q(n, seed)
        off = Q - np.diag(np.diag(Q))
        np.testing.assert_array_equal(Q, Q.T)
        assert set(np.unique(off)) <= {0.0, 1.0}
        assert int(np.triu(off, 1).sum()) == n * (n - 1) // 8            # exact edge count
        np.testing.assert_array_equal(np.diag(Q), -off.sum(axis=1))       # Q_ii = -deg(i)
    # x^T Q x = -cut(x) for every x of a small graph (brute force over all 2^10 cuts)
    Q = synth.maxcut_graph_q(10, 3)
    for bits in itertools.product((0, 1), repeat=10):
        x = np.array(bits, dtype=np.float64)
        assert x @ Q @ x == -synth.cut_value(Q, x)


def test_params_grid_and_mixes():
    g, b = synth.grid_params(16)                     # the 16 x 16 grid, gamma-major
    assert len(g) == 256 and len(b) == 256
    pts = {(round(x, 12), round(y, 12)) for x, y in zip(g, b)}
    assert len(pts) == 256                              # every (gamma_i, beta_j) once
    np.testing.assert_allclose(np.unique(g), np.arange(16) * np.pi / 15)
    np.testing.assert_allclose(np.unique(b), np.arange(16) * (np.pi / 2) / 15)
    gam, bet = synth.random_params(64, seed=8)
    assert gam.min() >= 0 and gam.max() <= np.pi and bet.min() >= 0 and bet.max() <= np.pi / 2
    ns, ps = synth.uneven_mix(5000, 9, 8, 24, 1, 6)
    assert ns.min() == 8 and ns.max() == 24 and ps.min() == 1 and ps.max() == 6
    t = synth.poisson_arrivals(100.0, 20000, 10)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps >= 0) and abs(gaps.mean() - 0.01) < 0.0005
