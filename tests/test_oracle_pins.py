"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the fact it uses: closed forms of the p = 1 QAOA expectation, exact special
cases of the mixer (beta = pi/2, pi), single-qubit algebra, invariants (norm, conjugation),
identities of the QUBO energy, published SplitMix64 outputs, and brute force on tiny inputs.
A plausible slip in the oracle (a dropped factor 2, a wrong sign of a phase or of the mixer, a
swapped layer order, a transposed index, a wrong tie rule) fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------------------------
# Random source
# ---------------------------------------------------------------------------------------------

def _golden_ints(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return [int(l) for l in f if l.strip() and not l.startswith("#")]


def test_splitmix64_published_vector(orc):
    want = _golden_ints("splitmix64_seed1234567.txt")
    assert [int(v) for v in orc.splitmix64(1234567, 5)] == want
    # the input generators' counter-based form is the same sequence
    assert [int(v) for v in synth.splitmix64(1234567, 5)] == want


def test_random_draw_worked_examples(orc):
    # Section V-A random selection, pinned by index sets worked by hand from published SplitMix64
    # outputs and Lemire's bounded draw (tests/golden/random_draw.json): the row state is
    # seed ^ (cycle * golden gamma) ^ j, step i swaps positions i and i + r, and a draw whose low
    # word is below (2^64 - range) mod range is redrawn. The cases include a rejected draw, a draw
    # accepted with the low word exactly at the threshold, and rows / cycles reached only by xor.
    import json
    with open(os.path.join(HERE, "golden", "random_draw.json")) as f:
        gold = json.load(f)
    pub = {k: [int(v) for v in vals] for k, vals in gold["published_outputs"].items() if not k.startswith("_")}
    assert pub["1234567"][:len(_golden_ints("splitmix64_seed1234567.txt"))] == \
        _golden_ints("splitmix64_seed1234567.txt")[:len(pub["1234567"])]
    M64, PHI = (1 << 64) - 1, 0x9E3779B97F4A7C15
    saw_reject = saw_boundary = False
    for c in gold["cases"]:
        N, k, j, cyc, seed = c["N"], c["k"], c["j"], c["cycle"], int(c["seed"])
        state = seed ^ ((cyc * PHI) & M64) ^ j
        assert state == int(c["state"]), c["note"]
        xs = [int(d["x"]) for st in c["steps"] for d in st["draws"]]
        # the worked draws are the generator's stream from that state ...
        assert [int(v) for v in orc.splitmix64(state, len(xs))] == xs, c["note"]
        # ... which is a published stream where the case says so
        if c["stream_seed"] in pub:
            ref = pub[c["stream_seed"]]
            tail = xs[len(xs) - len(ref):] if c["stream_seed"] == "0" else xs[:len(ref)]
            assert tail[:len(ref)] == ref[:len(tail)], c["note"]
        # the worked arithmetic is self-consistent (a check of the golden file, not of the oracle)
        perm = list(range(N))
        for st in c["steps"]:
            rng = N - st["i"]
            assert st["range"] == rng
            for d in st["draws"]:
                prod = int(d["x"]) * rng
                assert int(d["x_times_range_hi"]) == prod >> 64 and int(d["x_times_range_lo"]) == prod & M64
                assert int(d["threshold"]) == ((1 << 64) - rng) % rng
                assert d["rejected"] == (int(d["x_times_range_lo"]) < int(d["threshold"]))
                saw_reject |= d["rejected"]
                saw_boundary |= int(d["x_times_range_lo"]) == int(d["threshold"])
            assert not st["draws"][-1]["rejected"] and st["r"] == int(st["draws"][-1]["x_times_range_hi"])
            i, r = st["i"], st["r"]
            perm[i], perm[i + r] = perm[i + r], perm[i]
            assert perm[:i + 1] == st["perm_prefix"]
        assert sorted(perm[:k]) == c["S_sorted"]
        # the oracle's decomposition reproduces the worked index set in row j
        idx, _ = orc.decompose(np.zeros((N, N)), None, j + 1, k, seed, cyc, conditioned=False)
        assert list(idx[j]) == c["S_sorted"], c["note"]
    assert saw_reject and saw_boundary


# ---------------------------------------------------------------------------------------------
# QUBO energies: E(z) = z^T Q z
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_energy_identities(orc, n):
    Q = synth.symmetric_q(n, seed=100 + n)
    E = orc.energies(Q)
    assert E[0] == 0.0
    for i in range(n):
        assert E[1 << i] == pytest.approx(Q[i, i], abs=1e-14)           # single variable
    for i in range(n):
        for j in range(i + 1, n):
            pair = E[(1 << i) | (1 << j)] - E[1 << i] - E[1 << j]
            assert pair == pytest.approx(2.0 * Q[i, j], abs=1e-13)      # coupling counted twice
    assert E[-1] == pytest.approx(Q.sum(), abs=1e-12)                   # all ones
    mean = 0.5 * np.trace(Q) + 0.25 * (Q.sum() - np.trace(Q))           # E[z_i]=1/2, E[z_i z_j]=1/4
    assert E.mean() == pytest.approx(mean, abs=1e-12)


def test_energy_brute_force_minimum(orc):
    n = 10
    Q = synth.symmetric_q(n, seed=1)
    E = orc.energies(Q)
    best = min(itertools.product((0, 1), repeat=n), key=lambda b: np.array(b) @ Q @ np.array(b))
    zb = sum(b << i for i, b in enumerate(best))
    assert int(np.argmin(E)) == zb


def test_energy_asymmetric_input_reads_q_as_given(orc):
    # Q_ij and Q_ji enter as separate terms (z^T Q z, not 2 * upper triangle)
    Q = np.array([[0.5, 2.0], [-1.0, 0.25]])
    E = orc.energies(Q)
    np.testing.assert_allclose(E, [0.0, 0.5, 0.25, 0.5 + 0.25 + 2.0 - 1.0], atol=0)


# ---------------------------------------------------------------------------------------------
# State vector (Eq. 2): special cases with exact answers
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("sign", [1, -1])
def test_single_qubit_closed_form(orc, sign):
    # n = 1, E(z) = q z. After e^{-i g H}: (1, e^{-i g q})/sqrt2; after [[c, -i s sb],[-i s sb, c]]
    # with s = sign: P(1) = (1 + s sin(2b) sin(g q)) / 2.
    q = 0.8
    E = orc.energies(np.array([[q]]))
    for g, b in [(0.3, 0.2), (1.1, -0.7), (2.5, 1.3)]:
        psi = orc.state(1, [g], [b], E, mixer_sign=sign)
        p1 = 0.5 * (1.0 + sign * np.sin(2 * b) * np.sin(g * q))
        assert abs(psi[1]) ** 2 == pytest.approx(p1, abs=1e-15)
        assert orc.expect(psi, E) == pytest.approx(q * p1, abs=1e-15)
        # amplitude itself: psi0 = (cos b - i s sin b e^{-igq}) / sqrt2
        a0 = (np.cos(b) - 1j * sign * np.sin(b) * np.exp(-1j * g * q)) / np.sqrt(2)
        assert psi[0] == pytest.approx(a0, abs=1e-15)


@pytest.mark.parametrize("n", [3, 8])
def test_uniform_when_gamma_or_beta_zero(orc, n):
    Q = synth.symmetric_q(n, seed=7)
    E = orc.energies(Q)
    mean = 0.5 * np.trace(Q) + 0.25 * (Q.sum() - np.trace(Q))
    for g, b in [(0.0, 0.9), (1.3, 0.0), (0.0, 0.0)]:
        psi = orc.state(n, [g], [b], E)
        np.testing.assert_allclose(np.abs(psi) ** 2, 2.0 ** -n, rtol=1e-12)
        assert orc.expect(psi, E) == pytest.approx(mean, abs=1e-12)


@pytest.mark.parametrize("n", [2, 5, 10])
def test_beta_half_pi_flips_all_bits(orc, n):
    # e^{-i (pi/2) X} = -i X on every qubit: psi(z) = (-i)^n e^{-i g E(~z)} 2^{-n/2}
    Q = synth.symmetric_q(n, seed=11)
    E = orc.energies(Q)
    g = 0.77
    psi = orc.state(n, [g], [np.pi / 2], E)
    z = np.arange(1 << n)
    want = (-1j) ** n * np.exp(-1j * g * E[z ^ ((1 << n) - 1)]) * 2.0 ** (-n / 2)
    np.testing.assert_allclose(psi, want, atol=1e-13)


@pytest.mark.parametrize("n", [3, 6])
def test_beta_pi_is_minus_identity(orc, n):
    # e^{-i pi X} = -I on every qubit: psi = (-1)^n e^{-i g E} 2^{-n/2}
    Q = synth.symmetric_q(n, seed=12)
    E = orc.energies(Q)
    psi = orc.state(n, [0.4], [np.pi], E)
    np.testing.assert_allclose(psi, (-1) ** n * np.exp(-0.4j * E) * 2.0 ** (-n / 2), atol=1e-13)


@pytest.mark.parametrize("n,p", [(4, 1), (9, 3), (12, 2)])
def test_norm_and_conjugation(orc, n, p):
    Q = synth.symmetric_q(n, seed=13)
    E = orc.energies(Q)
    g, b = synth.random_params(p, seed=5)
    psi = orc.state(n, g, b, E)
    assert np.sum(np.abs(psi) ** 2) == pytest.approx(1.0, abs=1e-12)
    # (-gamma, -beta) conjugates every factor of Eq. 2 and |+> is real
    psim = orc.state(n, -g, -b, E)
    np.testing.assert_allclose(psim, np.conj(psi), atol=1e-14)


def test_layers_compose_in_order(orc):
    # layer 1 acts first: state(p=2) == apply layer 2 to state(p=1); a zero second layer is identity
    n = 7
    Q = synth.symmetric_q(n, seed=14)
    E = orc.energies(Q)
    ps2 = orc.state(n, [0.3, 0.9], [0.5, 0.2], E)
    ps1 = orc.state(n, [0.3], [0.5], E)
    np.testing.assert_allclose(orc.apply_layers(ps1, [0.9], [0.2], E), ps2, atol=1e-14)
    np.testing.assert_allclose(orc.state(n, [0.3, 0.0], [0.5, 0.0], E), ps1, atol=1e-14)
    # the other order gives a different state (the test would notice swapped layers)
    assert np.max(np.abs(orc.state(n, [0.9, 0.3], [0.2, 0.5], E) - ps2)) > 1e-3


# ---------------------------------------------------------------------------------------------
# Closed-form p = 1 expectation for field-free Ising costs (Wang, Hadfield, Jiang & Rieffel 2018;
# Ozaeta, van Dam & McMahon 2022). With s = 1 - 2z, E = c + sum_{u<v} J_uv s_u s_v,
# J = offdiag(Q) / 2 and mixer e^{-i b sum X}:
#   <Z_u Z_v> = 1/2 sin(4b) sin(2g J_uv) [prod_{w!=u,v} cos(2g J_uw) + prod_{w!=u,v} cos(2g J_vw)]
#             - 1/2 sin^2(2b) [prod_{w!=u,v} cos(2g (J_uw + J_vw)) - prod cos(2g (J_uw - J_vw))]
# ---------------------------------------------------------------------------------------------

def closed_form_p1(Q, g, b):
    n = Q.shape[0]
    J = (Q - np.diag(np.diag(Q))) / 2.0
    c = -(Q.sum() - np.trace(Q)) / 4.0
    tot = c
    for u in range(n):
        for v in range(u + 1, n):
            if J[u, v] == 0.0:
                continue
            w = [x for x in range(n) if x not in (u, v)]
            t1 = np.prod(np.cos(2 * g * J[u, w])) + np.prod(np.cos(2 * g * J[v, w]))
            t2 = np.prod(np.cos(2 * g * (J[u, w] + J[v, w]))) - np.prod(np.cos(2 * g * (J[u, w] - J[v, w])))
            zz = 0.5 * np.sin(4 * b) * np.sin(2 * g * J[u, v]) * t1 - 0.5 * np.sin(2 * b) ** 2 * t2
            tot += J[u, v] * zz
    return tot


@pytest.mark.parametrize("n,seed,dens", [(6, 1, 1.0), (10, 2, 0.5), (14, 3, 0.3)])
def test_closed_form_p1_ising(orc, n, seed, dens):
    Q = synth.maxcut_form_q(n, seed=seed, edge_prob=dens)
    E = orc.energies(Q)
    for g, b in [(0.31, 0.17), (0.9, 0.6), (-0.4, 1.2)]:
        psi = orc.state(n, [g], [b], E)
        assert orc.expect(psi, E) == pytest.approx(closed_form_p1(Q, g, b), abs=1e-10)
    # the paper's printed mixer sign (H_X = -sum X) mirrors beta
    psi = orc.state(n, [0.31], [0.17], E, mixer_sign=-1)
    assert orc.expect(psi, E) == pytest.approx(closed_form_p1(Q, 0.31, -0.17), abs=1e-10)


def test_two_layers_reduce_to_one_via_bit_flip(orc):
    # Field-free E satisfies E(~z) = E(z). With beta_1 = pi/2 the first mixer only flips all bits,
    # so two layers (g1, pi/2), (g2, b2) equal one layer (g1 + g2, b2) up to the phase (-i)^n.
    n = 9
    Q = synth.maxcut_form_q(n, seed=4, edge_prob=0.6)
    E = orc.energies(Q)
    psi2 = orc.state(n, [0.3, 0.5], [np.pi / 2, 0.35], E)
    psi1 = orc.state(n, [0.8], [0.35], E)
    np.testing.assert_allclose(psi2, (-1j) ** n * psi1, atol=1e-13)
    assert orc.expect(psi2, E) == pytest.approx(closed_form_p1(Q, 0.8, 0.35), abs=1e-10)


# ---------------------------------------------------------------------------------------------
# Top-k: probability descending, ties to the smaller index
# ---------------------------------------------------------------------------------------------

def test_topk_tie_rule_uniform(orc):
    n = 6
    E = orc.energies(synth.symmetric_q(n, seed=3))
    psi = orc.state(n, [0.0], [0.0], E)
    idx, pk = orc.topk(psi, 8)
    assert list(idx) == list(range(8))
    np.testing.assert_allclose(pk, 2.0 ** -n)


def test_topk_against_lexsort(orc):
    rng = np.random.default_rng(0)
    for D, k in [(64, 5), (1000, 16), (4096, 1)]:
        prob = rng.integers(0, 40, size=D).astype(np.float64) / 40.0     # many exact ties
        idx, pk = orc.topk_probs(prob, k)
        order = np.lexsort((np.arange(D), -prob))[:k]
        assert list(idx) == list(order)
        np.testing.assert_array_equal(pk, prob[order])


def test_topk_of_bitflip_state_is_argmin_of_flipped_energy(orc):
    # at beta = pi/2 the probabilities are uniform, so the tie rule alone decides
    n = 5
    E = orc.energies(synth.symmetric_q(n, seed=8))
    psi = orc.state(n, [0.3], [np.pi / 4], E)
    prob = np.abs(psi) ** 2
    idx, _ = orc.topk(psi, 3)
    assert int(idx[0]) == int(np.argmax(prob))


# ---------------------------------------------------------------------------------------------
# Adjoint gradient
# ---------------------------------------------------------------------------------------------

def test_grad_single_qubit_closed_form(orc):
    # <C> = q (1 + sin 2b sin g q) / 2 -> d/dg = q^2 sin 2b cos(g q) / 2, d/db = q cos 2b sin(g q)
    q = 1.3
    E = orc.energies(np.array([[q]]))
    for g, b in [(0.4, 0.3), (2.0, -0.9)]:
        ex, dg, db = orc.grad(1, [g], [b], E)
        assert ex == pytest.approx(q * (1 + np.sin(2 * b) * np.sin(g * q)) / 2, abs=1e-15)
        assert dg[0] == pytest.approx(q * q * np.sin(2 * b) * np.cos(g * q) / 2, abs=1e-14)
        assert db[0] == pytest.approx(q * np.cos(2 * b) * np.sin(g * q), abs=1e-14)


def test_grad_vs_closed_form_derivative(orc):
    n = 8
    Q = synth.maxcut_form_q(n, seed=9, edge_prob=0.7)
    E = orc.energies(Q)
    g, b, h = 0.37, 0.21, 1e-5
    ex, dg, db = orc.grad(n, [g], [b], E)
    fg = (closed_form_p1(Q, g + h, b) - closed_form_p1(Q, g - h, b)) / (2 * h)
    fb = (closed_form_p1(Q, g, b + h) - closed_form_p1(Q, g, b - h)) / (2 * h)
    assert dg[0] == pytest.approx(fg, rel=1e-7, abs=1e-9)
    assert db[0] == pytest.approx(fb, rel=1e-7, abs=1e-9)
    assert ex == pytest.approx(closed_form_p1(Q, g, b), abs=1e-10)


@pytest.mark.parametrize("sign", [1, -1])
def test_grad_vs_central_differences_deep(orc, sign):
    # dense Q, p = 3: central differences with h = 1e-3 (rel <= 1e-3) on the pinned <C>
    n, p = 7, 3
    Q = synth.symmetric_q(n, seed=21, dist="normal")
    E = orc.energies(Q)
    g, b = synth.random_params(p, seed=22)
    ex, dg, db = orc.grad(n, g, b, E, mixer_sign=sign)
    h = 1e-3

    def f(gg, bb):
        return orc.expect(orc.state(n, gg, bb, E, mixer_sign=sign), E)

    for l in range(p):
        e = np.zeros(p)
        e[l] = h
        fd_g = (f(g + e, b) - f(g - e, b)) / (2 * h)
        fd_b = (f(g, b + e) - f(g, b - e)) / (2 * h)
        assert dg[l] == pytest.approx(fd_g, rel=1e-3, abs=1e-6)
        assert db[l] == pytest.approx(fd_b, rel=1e-3, abs=1e-6)


# ---------------------------------------------------------------------------------------------
# Decomposition (Section V-A) and aggregation (Section V step 3)
# ---------------------------------------------------------------------------------------------

def test_decompose_random_invariants(orc):
    N, m, k = 300, 64, 12
    Q = synth.symmetric_q(N, seed=2)
    x = synth.bits(99, N)
    idx, qs = orc.decompose(Q, x, m, k, seed=5, cycle=3, conditioned=False)
    for j in range(m):
        s = idx[j]
        assert np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < N       # sorted, distinct, in range
        np.testing.assert_array_equal(qs[j], Q[np.ix_(s, s)])          # full symmetric Q[S,S]
    idx2, _ = orc.decompose(Q, x, m, k, seed=5, cycle=3, conditioned=False)
    np.testing.assert_array_equal(idx, idx2)                           # deterministic
    idx3, _ = orc.decompose(Q, x, m, k, seed=5, cycle=4, conditioned=False)
    assert not np.array_equal(idx, idx3)                               # cycle changes the draw


def test_decompose_random_is_uniform(orc):
    # each variable is chosen with probability k/N; chi-square over 4000 sub-QUBOs
    N, m, k = 40, 4000, 5
    Q = np.zeros((N, N))
    idx, _ = orc.decompose(Q, None, m, k, seed=17, conditioned=False)
    counts = np.bincount(idx.reshape(-1), minlength=N)
    expct = m * k / N
    chi2 = float(np.sum((counts - expct) ** 2 / expct))
    assert chi2 < 80.0          # 39 dof: mean 39, sd ~8.8
    # pairs are uniform too: no variable is favoured as the first pick
    first = np.bincount(idx[:, 0], minlength=N)
    assert first[N - 1] == 0 or k == 1   # sorted: the largest index can only come first if k == 1


def test_conditioned_subqubo_equals_global_energy(orc):
    # E_sub(y) + const = E(x with x_S = y) for every y: brute force over all 2^k sub-solutions
    N, m, k = 60, 3, 6
    Q = synth.symmetric_q(N, seed=31)
    x = synth.bits(32, N)
    idx, qs = orc.decompose(Q, x, m, k, seed=33, conditioned=True)
    for j in range(m):
        S = idx[j]
        diffs = []
        for yb in range(1 << k):
            y = np.array([(yb >> q) & 1 for q in range(k)], dtype=np.float64)
            xx = x.astype(np.float64).copy()
            xx[S] = y
            diffs.append(xx @ Q @ xx - y @ qs[j] @ y)
        np.testing.assert_allclose(diffs, diffs[0], atol=1e-10)


def test_signed_ifd_windows_and_invalid_flags(orc):
    N, m, k = 40, 8, 5
    Q = synth.symmetric_q(N, seed=43)
    x = synth.bits(44, N)
    dE = orc.impact(Q, x)
    assert (dE < 0).any() and (dE > 0).any()              # both signs occur
    rank = sorted(range(N), key=lambda i: (dE[i], i))      # largest decrease first
    idx, _ = orc.decompose(Q, x, m, k, seed=0, method=orc.IFD | orc.SIGNED, conditioned=False)
    for j in range(m):
        np.testing.assert_array_equal(idx[j], np.sort(rank[j:j + k]))
    with pytest.raises(RuntimeError):
        orc.decompose(Q, x, m, k, seed=0, method=orc.RANDOM | orc.SIGNED)
    with pytest.raises(RuntimeError):
        orc.decompose(Q, x, m, k, seed=0, method=orc.IFD | 32)


def test_ifd_windows_follow_impact_ranking(orc):
    N, m, k = 50, 6, 5
    Q = synth.symmetric_q(N, seed=41)
    x = synth.bits(42, N)
    dE = orc.impact(Q, x)
    e0 = x.astype(float) @ Q @ x.astype(float)
    for i in range(N):                         # impact = energy change of flipping x_i
        xx = x.astype(float).copy()
        xx[i] = 1 - xx[i]
        assert dE[i] == pytest.approx(xx @ Q @ xx - e0, abs=1e-10)
    rank = sorted(range(N), key=lambda i: (-abs(dE[i]), i))
    idx, qs = orc.decompose(Q, x, m, k, seed=0, method=orc.IFD, conditioned=False)
    for j in range(m):
        np.testing.assert_array_equal(idx[j], np.sort(rank[j:j + k]))   # stride-1 window
        np.testing.assert_array_equal(qs[j], Q[np.ix_(idx[j], idx[j])])


def _figure_case():
    import json
    with open(os.path.join(HERE, "golden", "bfs_pfs_figure.json")) as f:
        g = json.load(f)
    Q = np.diag(np.array(g["diag"]))
    for a, b in g["strong_pairs"]:
        Q[a, b] = Q[b, a] = g["coupling"]
    return g, Q


def test_bfs_pfs_paper_figure(orc):
    # Fig. bfs-pfs: BFS reaches x2 first, PFS x4 (higher impact); the fixture's index sets are
    # derived by hand from the traversal rules
    g, Q = _figure_case()
    x = np.zeros(Q.shape[0], dtype=np.uint8)
    assert sorted(range(7), key=lambda i: (-abs(orc.impact(Q, x)[i]), i)) == g["impact_rank"]
    for c in g["cases"]:
        for name, method in (("bfs", orc.BFS), ("pfs", orc.PFS)):
            idx, qs = orc.decompose(Q, x, c["j"] + 1, c["k"], seed=0, method=method, conditioned=False)
            assert idx[c["j"]].tolist() == c[name], (c, name)
            np.testing.assert_array_equal(qs[c["j"]], Q[np.ix_(idx[c["j"]], idx[c["j"]])])


def _strong_sets(Q, k):
    # strong neighbours by the reading: |Q_ij| >= the d-th largest off-diagonal magnitude of row i
    N = Q.shape[0]
    out = []
    for i in range(N):
        mags = sorted((abs(Q[i, j]) for j in range(N) if j != i and Q[i, j] != 0.0), reverse=True)
        d = min(k - 1, len(mags))
        thr = mags[d - 1] if d >= 1 else float("inf")
        out.append([j for j in range(N) if j != i and Q[i, j] != 0.0 and abs(Q[i, j]) >= thr])
    return out


def _traverse_py(strong, rank, root, k, bfs):
    # the traversals written out directly over Python lists (BFS: deque of discovered variables;
    # PFS: frontier set, best by rank position)
    from collections import deque
    pos = {v: t for t, v in enumerate(rank)}
    sel, order = set(), []
    frontier = set()
    nxt = root
    q = deque()
    while len(order) < k:
        if nxt is None:
            nxt = next(v for v in rank if v not in sel)
        v, nxt = nxt, None
        sel.add(v)
        order.append(v)
        if bfs:
            q.append(v)
            while len(order) < k and q:
                w = q.popleft()
                for u in strong[w]:
                    if len(order) < k and u not in sel:
                        sel.add(u)
                        order.append(u)
                        q.append(u)
        else:
            frontier.update(strong[v])
            cand = [u for u in frontier if u not in sel]
            nxt = min(cand, key=lambda u: pos[u]) if cand else None
    return sorted(order)


@pytest.mark.parametrize("signed", [False, True])
@pytest.mark.parametrize("kind", ["dense", "maxcut", "sparse"])
@pytest.mark.parametrize("k", [2, 4, 7])
def test_bfs_pfs_against_direct_traversal(orc, kind, k, signed):
    N = 30
    if kind == "dense":
        Q = synth.symmetric_q(N, seed=71)
    elif kind == "maxcut":
        Q = synth.maxcut_graph_q(N, seed=72, edges=40)        # unit weights: ties everywhere
    else:
        Q = synth.maxcut_graph_q(N, seed=73, edges=12)        # isolated vertices force restarts
    x = synth.bits(74, N)
    dE = orc.impact(Q, x)
    # default ranking |dE| descending; signed ranking dE ascending (largest decrease first)
    rank = sorted(range(N), key=(lambda i: (dE[i], i)) if signed else (lambda i: (-abs(dE[i]), i)))
    strong = _strong_sets(Q, k)
    flag = orc.SIGNED if signed else 0
    for method, bfs in ((orc.BFS, True), (orc.PFS, False)):
        idx, _ = orc.decompose(Q, x, N, k, seed=0, method=method | flag, conditioned=False)
        for j in range(N):
            assert idx[j].tolist() == _traverse_py(strong, rank, rank[j], k, bfs), (kind, k, j, bfs)


def test_sample_two_level_and_basis_states(orc):
    # inverse CDF on a hand-made distribution: P = (0, 0.25, 0, 0.75) -> u < 0.25 gives 1, else 3
    pr = np.array([0.0, 0.25, 0.0, 0.75])
    u = np.array([0.0, 0.1, 0.2499, 0.25, 0.5, 0.9999])
    assert orc.sample_probs(pr, u).tolist() == [1, 1, 1, 3, 3, 3]
    # a basis state returns its index for every uniform; scaling the distribution changes nothing
    for z in (0, 5, 15):
        e = np.zeros(16)
        e[z] = 1.0
        assert set(orc.sample_probs(e, synth.uniform01(3, 64)).tolist()) == {z}
        assert set(orc.sample_probs(3.5 * e, synth.uniform01(4, 64)).tolist()) == {z}


def test_sample_frequencies_match_probabilities(orc):
    # shots of a p=2 QAOA state follow |psi|^2: Pearson chi-square over the 2^6 outcomes
    n, shots = 6, 200000
    Q = synth.symmetric_q(n, seed=81)
    psi = orc.state(n, [0.4, 0.7], [0.6, 0.3], orc.energies(Q))
    pr = np.abs(psi) ** 2
    z = orc.sample(psi, synth.uniform01(82, shots))
    counts = np.bincount(z.astype(np.int64), minlength=1 << n)
    expect = shots * pr
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    assert chi2 < 63 + 6 * np.sqrt(2 * 63)          # 63 degrees of freedom, six sigma
    # and the order statistics: sorted uniforms give non-decreasing indices
    us = np.sort(synth.uniform01(83, 1000))
    assert np.all(np.diff(orc.sample(psi, us).astype(np.int64)) >= 0)


def test_merge_single_subqubo_takes_best(orc):
    # N = k: every candidate fixes the whole solution, so sequential "accept if lower" ends at
    # the minimum of the starting energy and all candidate energies
    k = 8
    Q = synth.symmetric_q(k, seed=51)
    x0 = synth.bits(52, k)
    idx = np.arange(k, dtype=np.int32)[None, :]
    cand = synth.splitmix64(53, 6).reshape(1, 6) & np.uint64(0xFF)
    x1, e1, acc = orc.merge(Q, x0, idx, cand)
    allx = [x0] + [np.array([(int(c) >> q) & 1 for q in range(k)], dtype=np.uint8) for c in cand[0]]
    es = [float(v.astype(float) @ Q @ v.astype(float)) for v in allx]
    assert e1 == pytest.approx(min(es), abs=1e-12)
    np.testing.assert_array_equal(x1, allx[int(np.argmin(es))])


def test_merge_monotone_and_consistent(orc):
    N, m, k, K = 200, 30, 10, 4
    Q = synth.symmetric_q(N, seed=61)
    x = synth.bits(62, N)
    idx, _ = orc.decompose(Q, x, m, k, seed=63)
    cand = (synth.splitmix64(64, m * K) & np.uint64((1 << k) - 1)).reshape(m, K)
    e_prev = orc.qubo_energy(Q, x)
    x1, e1, acc = orc.merge(Q, x, idx, cand)
    assert e1 <= e_prev
    assert e1 == pytest.approx(orc.qubo_energy(Q, x1), abs=1e-9 * np.abs(Q).sum())
    assert 0 < acc <= m * K
    # replaying the accepted decisions one by one with direct energies gives the same path
    xr = x.copy()
    for j in range(m):
        for c in range(K):
            y = int(cand[j, c])
            xt = xr.copy()
            xt[idx[j]] = [(y >> q) & 1 for q in range(k)]
            if orc.qubo_energy(Q, xt) < orc.qubo_energy(Q, xr) - 1e-9:
                xr = xt
    np.testing.assert_array_equal(xr, x1)


def test_merge_rejects_non_improving_updates(orc):
    # "only updates that lead to lower energy are accepted": re-proposing the current fragment,
    # or a fragment of equal energy, changes nothing and counts as no acceptance
    N, k = 30, 4
    Q = synth.symmetric_q(N, seed=71)
    x = synth.bits(72, N)
    idx = np.array([[2, 5, 11, 20]], dtype=np.int32)
    cur = sum(int(x[s]) << q for q, s in enumerate(idx[0]))
    x1, e1, acc = orc.merge(Q, x, idx, np.array([[cur, cur]], dtype=np.uint64))
    assert acc == 0 and np.array_equal(x1, x)
    assert e1 == pytest.approx(orc.qubo_energy(Q, x), abs=1e-12)
    Z = np.zeros((N, N))                      # all energies equal: nothing is accepted
    _, _, acc0 = orc.merge(Z, x, idx, np.array([[cur ^ 1, cur ^ 15]], dtype=np.uint64))
    assert acc0 == 0
