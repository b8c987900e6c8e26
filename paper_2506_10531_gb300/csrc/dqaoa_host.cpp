// dqaoa_host.cpp -- host side of the DQAOA cycle (arXiv 2506.10531, Section V): the index
// sets of the random and impact-factor-directed decompositions (Section V-A, Algorithm 1),
// the sub-QUBO matrices, and the aggregation of sub-solutions (Section V step 3).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <vector>

#include "qaoa_host.h"

namespace qaoa {

namespace {

// SplitMix64 (Steele, Lea & Flood 2014): advance by the golden gamma, then the finaliser.
struct SplitMix64 {
    uint64_t s;
    uint64_t next() {
        s += 0x9E3779B97F4A7C15ULL;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    // Uniform in [0, range): Lemire (2019) multiply-shift, rejecting low words below
    // 2^64 mod range.
    uint64_t below(uint64_t range) {
        __uint128_t m = (__uint128_t)next() * range;
        uint64_t lo = (uint64_t)m;
        if (lo < range) {
            const uint64_t t = (0 - range) % range;
            while (lo < t) {
                m = (__uint128_t)next() * range;
                lo = (uint64_t)m;
            }
        }
        return (uint64_t)(m >> 64);
    }
};

}  // namespace

// Random index sets: a partial Fisher-Yates shuffle of 0..N-1 per row, with only the touched
// positions stored, which draws the same sets as a shuffle of the full array: positions
// 0..k-1 in a direct array, positions >= k (at most k of them) in a short list.
int draw_random(int N, int m, int k, uint64_t seed, uint64_t cycle, int32_t* idx) {
    std::vector<int32_t> pre((size_t)k), pos((size_t)k), val((size_t)k);
    for (int j = 0; j < m; ++j) {
        SplitMix64 g{seed ^ (cycle * 0x9E3779B97F4A7C15ULL) ^ (uint64_t)j};
        for (int i = 0; i < k; ++i) pre[i] = i;
        int used = 0;
        int32_t* S = idx + (int64_t)j * k;
        for (int i = 0; i < k; ++i) {
            const int32_t r = i + (int32_t)g.below((uint64_t)(N - i));
            const int32_t vi = pre[i];
            int32_t vr;
            if (r < k) {
                vr = pre[r];
                pre[r] = vi;
            } else {
                int e = 0;
                while (e < used && pos[e] != r) ++e;
                vr = (e < used) ? val[e] : r;
                if (e == used) { pos[used] = r; ++used; }
                val[e] = vi;
            }
            pre[i] = vr;
            S[i] = vr;
        }
        std::sort(S, S + k);
    }
    return 0;
}

// Impact factor of each variable (the energy change of flipping it) and the ranking by
// |impact| descending, ties to the smaller index.
static std::vector<int32_t> impact_order(const double* Q, int N, const uint8_t* x, bool signed_rank) {
    std::vector<double> imp(N);
    // h_i = sum over j != i with x_j = 1, ascending j. Eight rows advance together (independent
    // sums, each in its own order); a skipped term adds +0.0, which leaves every sum unchanged.
    int i0 = 0;
    for (; i0 + 8 <= N; i0 += 8) {
        double h[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        const double* rows = Q + (int64_t)i0 * N;
        for (int j = 0; j < N; ++j) {
            const bool xj = x[j] != 0;
            for (int r = 0; r < 8; ++r) {
                const double q = rows[(int64_t)r * N + j];
                h[r] += (xj && j != i0 + r) ? q : 0.0;
            }
        }
        for (int r = 0; r < 8; ++r) {
            const int i = i0 + r;
            imp[i] = (1.0 - 2.0 * (double)x[i]) * (Q[(int64_t)i * N + i] + 2.0 * h[r]);
        }
    }
    for (int i = i0; i < N; ++i) {
        const double* row = Q + (int64_t)i * N;
        double h = 0.0;
        for (int j = 0; j < N; ++j)
            if (j != i && x[j]) h += row[j];
        imp[i] = (1.0 - 2.0 * (double)x[i]) * (row[i] + 2.0 * h);
    }
    std::vector<int32_t> order(N);
    for (int i = 0; i < N; ++i) order[i] = i;
    // default: |impact| descending; signed: impact ascending (largest energy decrease first)
    if (signed_rank)
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return imp[a] < imp[b]; });
    else
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return std::fabs(imp[a]) > std::fabs(imp[b]); });
    return order;
}

// IFD (Algorithm 1): row j is the window ranking[j .. j+k-1].
int draw_ifd(const double* Q, int N, const uint8_t* x, int m, int k, int32_t* idx, bool signed_rank) {
    const std::vector<int32_t> order = impact_order(Q, N, x, signed_rank);
    for (int j = 0; j < m; ++j) {
        int32_t* S = idx + (int64_t)j * k;
        std::copy(order.begin() + j, order.begin() + j + k, S);
        std::sort(S, S + k);
    }
    return 0;
}

// BFS / PFS traversals (Section V-A). Strong neighbours of i: j != i with Q_ij != 0 and |Q_ij| at
// least the d-th largest off-diagonal magnitude of row i, d = min(k - 1, off-diagonal nonzeros),
// ties included; kept as ascending lists in CSR form (they depend on Q and k only).
void build_strong_graph(const double* Q, int N, int k, StrongGraph* g) {
    g->N = N;
    g->k = k;
    g->off.assign((size_t)N + 1, 0);
    g->nbr.clear();
    std::vector<double> mag;
    for (int i = 0; i < N; ++i) {
        const double* row = Q + (int64_t)i * N;
        mag.clear();
        for (int j = 0; j < N; ++j)
            if (j != i && row[j] != 0.0) mag.push_back(std::fabs(row[j]));
        const int d = std::min<int>(k - 1, (int)mag.size());
        if (d >= 1) {
            std::nth_element(mag.begin(), mag.begin() + (d - 1), mag.end(), std::greater<double>());
            const double thr = mag[d - 1];
            for (int j = 0; j < N; ++j)
                if (j != i && row[j] != 0.0 && std::fabs(row[j]) >= thr) g->nbr.push_back(j);
        }
        g->off[i + 1] = (int64_t)g->nbr.size();
    }
    // dense graphs (at least 32 strong neighbours per row on average, N <= 16384) also get bitset
    // rows, so that PFS unites frontiers a word at a time instead of marking every neighbour
    g->words = 0;
    g->bits.clear();
    if (N <= 16384 && (int64_t)g->nbr.size() >= 32 * (int64_t)N) {
        g->words = (N + 63) / 64;
        g->bits.assign((size_t)N * g->words, 0ull);
        for (int i = 0; i < N; ++i)
            for (int64_t e = g->off[i]; e < g->off[i + 1]; ++e)
                g->bits[(size_t)i * g->words + (g->nbr[e] >> 6)] |= 1ull << (g->nbr[e] & 63);
    }
}

// Row j starts at ranking[j]; BFS takes the strong neighbours of the queue's front in ascending
// index order, PFS the best-ranked unselected strong neighbour of any selected variable; an
// exhausted traversal restarts at the best-ranked unselected variable. g: the strong graph of
// (Q, k), built here when null.
int draw_graph(const double* Q, int N, const uint8_t* x, int method, int m, int k, int32_t* idx,
               const StrongGraph* g, bool signed_rank) {
    StrongGraph local;
    if (!g) {
        build_strong_graph(Q, N, k, &local);
        g = &local;
    }
    const std::vector<int32_t> order = impact_order(Q, N, x, signed_rank);
    const int64_t* off = g->off.data();
    const int32_t* nbr = g->nbr.data();
    std::vector<uint8_t> inS(N), inF(N);
    std::vector<int32_t> queue(N);
    const int W = (method != 2) ? g->words : 0;
    std::vector<uint64_t> fbits((size_t)W, 0ull);
    for (int j = 0; j < m; ++j) {
        int32_t* S = idx + (int64_t)j * k;
        int size = 0, head = 0, tail = 0, scan = 0;   // scan: restart cursor into the ranking
        int32_t next = order[j];
        while (size < k) {
            if (next < 0) {
                while (inS[order[scan]]) ++scan;
                next = order[scan];
            }
            const int32_t v = next;
            next = -1;
            S[size++] = v;
            inS[v] = 1;
            if (method == 2) {          // BFS
                queue[tail++] = v;
                while (size < k && head < tail) {
                    const int32_t w = queue[head++];
                    for (int64_t e = off[w]; e < off[w + 1] && size < k; ++e) {
                        const int32_t u = nbr[e];
                        if (!inS[u]) { S[size++] = u; inS[u] = 1; queue[tail++] = u; }
                    }
                }
            } else if (W) {             // PFS, bitset rows: frontier |= row v
                const uint64_t* rb = g->bits.data() + (size_t)v * W;
                for (int w = 0; w < W; ++w) fbits[w] |= rb[w];
                for (int t = 0; t < N; ++t) {
                    const int32_t u = order[t];
                    if (((fbits[u >> 6] >> (u & 63)) & 1ull) && !inS[u]) { next = u; break; }
                }
            } else {                    // PFS: first frontier variable in ranking order
                for (int64_t e = off[v]; e < off[v + 1]; ++e) inF[nbr[e]] = 1;
                for (int t = 0; t < N; ++t) {
                    const int32_t u = order[t];
                    if (inF[u] && !inS[u]) { next = u; break; }
                }
            }
        }
        // clear the marks of this row only
        for (int a = 0; a < k; ++a) inS[S[a]] = 0;
        if (W)
            std::fill(fbits.begin(), fbits.end(), 0ull);
        else if (method != 2)
            for (int a = 0; a < k; ++a)
                for (int64_t e = off[S[a]]; e < off[S[a] + 1]; ++e) inF[nbr[e]] = 0;
        std::sort(S, S + k);
    }
    return 0;
}

void build_subqubos(const double* Q, int N, const uint8_t* x, int m, int k, const int32_t* idx,
                    int conditioned, double* Qsub) {
    std::vector<uint8_t> inS(N, 0);
    for (int j = 0; j < m; ++j) {
        const int32_t* S = idx + (int64_t)j * k;
        double* Qs = Qsub + (int64_t)j * k * k;
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b) Qs[a * k + b] = Q[(int64_t)S[a] * N + S[b]];
        if (!conditioned) continue;
        for (int a = 0; a < k; ++a) inS[S[a]] = 1;
        // conditioning sum in 32 interleaved partial sums (l = r mod 32, ascending), combined by
        // the xor tree v_r <- v_r + v_{r^d}, d = 16, 8, 4, 2, 1: the device kernel's order
        for (int a = 0; a < k; ++a) {
            const double* row = Q + (int64_t)S[a] * N;
            double sr[32], nv[32];
            for (int r = 0; r < 32; ++r) {
                sr[r] = 0.0;
                for (int l = r; l < N; l += 32)
                    if (!inS[l] && x[l]) sr[r] += row[l];
            }
            for (int d = 16; d >= 1; d >>= 1) {
                for (int r = 0; r < 32; ++r) nv[r] = sr[r] + sr[r ^ d];
                for (int r = 0; r < 32; ++r) sr[r] = nv[r];
            }
            Qs[a * k + a] = Q[(int64_t)S[a] * N + S[a]] + 2.0 * sr[0];
        }
        for (int a = 0; a < k; ++a) inS[S[a]] = 0;
    }
}

// Aggregation: h = Qx is kept up to date (O(N) per flipped variable), so each candidate costs
// O(|d|^2) with d = x' - x. With a cache (h, energy, tau of the same Q and x from the previous
// call) the O(N^2) set-up is skipped.
// The sequential candidate loop of merge (one instantiation with the FP64 blocks at hand, one
// that gathers the entries from Q). KC > 0 fixes the sub-QUBO size at compile time (the common
// sizes; the arithmetic is the same, only the loops are unrolled). Returns the accepted count;
// energy is updated in place.
template <bool BLK, int KC>
static int merge_loop(const double* Q, int N, uint8_t* x, int m, int k_rt, const int32_t* idx, int K,
                      const uint64_t* cand, const double* qblk, double tau, double* hq_in,
                      double& energy, const double* pair, uint8_t* chg) {
    const int k = KC > 0 ? KC : k_rt;
    int accepted = 0;
    int nz[64];
    double d[64], h2[64];
    const uint64_t kmask = k >= 64 ? ~0ull : (1ull << k) - 1ull;
    double* __restrict__ hq = hq_in;
    for (int j = 0; j < m; ++j) {
        const int32_t* S = idx + (int64_t)j * k;
        const double* blk = BLK ? qblk + (int64_t)j * k * k : nullptr;
        // x on S_j packed like a candidate: the changed positions of a candidate are then the set
        // bits of y ^ xs, visited in ascending order without a data-dependent branch per position;
        // h2 = 2 h on S_j (exact doubling), refreshed whenever a candidate is accepted
        uint64_t xs = 0;
        bool fresh = pair != nullptr;   // no variable of S_j has flipped this cycle
        for (int a = 0; a < k; ++a) {
            xs |= (uint64_t)(x[S[a]] != 0) << a;
            h2[a] = 2.0 * hq[S[a]];
            if (pair && chg[S[a]]) fresh = false;
        }
        for (int c = 0; c < K; ++c) {
            const uint64_t y = cand[(int64_t)j * K + c];
            int cnt = 0;
            for (uint64_t diff = (y ^ xs) & kmask; diff; diff &= diff - 1) {
                const int a = __builtin_ctzll(diff);
                nz[cnt] = a;
                d[cnt] = ((y >> a) & 1u) ? 1.0 : -1.0;   // x'_a - x_a
                ++cnt;
            }
            if (!cnt) continue;
            // inner[u] = sum over v (ascending) of Q[S_u][S_v] d_v; the u sums are independent,
            // so they advance together (each keeps its own order)
            double inner[64];
            double dE = 0.0;
            if (fresh) {
                // the device's pair term for this d, plus the linear term for the current h
                double lin = 0.0;
                for (int u = 0; u < cnt; ++u) lin += d[u] * h2[nz[u]];
                dE = lin + pair[(int64_t)j * K + c];
            } else if constexpr (BLK) {
                // with the block at hand, every row a of it advances (contiguous, vectorisable:
                // Q[S_a][S_v] = Q[S_v][S_a] is row v of the symmetric block) and the changed
                // rows are read at the end; the sums of the changed rows are the same sums
                for (int a = 0; a < k; ++a) inner[a] = 0.0;
                for (int v = 0; v < cnt; ++v) {
                    const double dv = d[v];
                    const double* col = blk + (int64_t)nz[v] * k;
                    for (int a = 0; a < k; ++a) inner[a] += col[a] * dv;
                }
                for (int u = 0; u < cnt; ++u) dE += d[u] * (h2[nz[u]] + inner[nz[u]]);
            } else {
                for (int u = 0; u < cnt; ++u) inner[u] = 0.0;
                for (int v = 0; v < cnt; ++v) {
                    const double dv = d[v];
                    const int64_t cv = S[nz[v]];
                    for (int u = 0; u < cnt; ++u) inner[u] += Q[(int64_t)S[nz[u]] * N + cv] * dv;
                }
                for (int u = 0; u < cnt; ++u) dE += d[u] * (h2[nz[u]] + inner[u]);
            }
            if (dE < -tau) {
                fresh = false;
                for (int u = 0; u < cnt; ++u) {
                    const int var = S[nz[u]];
                    x[var] = (uint8_t)(d[u] > 0.0);
                    if (chg) chg[var] = 1;
                }
                // h += d_u * (column S[nz[u]] of the symmetric Q == its row) for u ascending:
                // every h[l] takes the same adds in the same order as one row at a time, with
                // eight, then four rows per sweep over h
                int u = 0;
                for (; u + 8 <= cnt; u += 8) {
                    const double* __restrict__ r0 = Q + (int64_t)S[nz[u]] * N;
                    const double* __restrict__ r1 = Q + (int64_t)S[nz[u + 1]] * N;
                    const double* __restrict__ r2 = Q + (int64_t)S[nz[u + 2]] * N;
                    const double* __restrict__ r3 = Q + (int64_t)S[nz[u + 3]] * N;
                    const double* __restrict__ r4 = Q + (int64_t)S[nz[u + 4]] * N;
                    const double* __restrict__ r5 = Q + (int64_t)S[nz[u + 5]] * N;
                    const double* __restrict__ r6 = Q + (int64_t)S[nz[u + 6]] * N;
                    const double* __restrict__ r7 = Q + (int64_t)S[nz[u + 7]] * N;
                    const double d0 = d[u], d1 = d[u + 1], d2 = d[u + 2], d3 = d[u + 3];
                    const double d4 = d[u + 4], d5 = d[u + 5], d6 = d[u + 6], d7 = d[u + 7];
                    for (int l = 0; l < N; ++l)
                        hq[l] = (((((((hq[l] + d0 * r0[l]) + d1 * r1[l]) + d2 * r2[l]) + d3 * r3[l]) + d4 * r4[l]) +
                                  d5 * r5[l]) + d6 * r6[l]) + d7 * r7[l];
                }
                for (; u + 4 <= cnt; u += 4) {
                    const double* __restrict__ r0 = Q + (int64_t)S[nz[u]] * N;
                    const double* __restrict__ r1 = Q + (int64_t)S[nz[u + 1]] * N;
                    const double* __restrict__ r2 = Q + (int64_t)S[nz[u + 2]] * N;
                    const double* __restrict__ r3 = Q + (int64_t)S[nz[u + 3]] * N;
                    const double d0 = d[u], d1 = d[u + 1], d2 = d[u + 2], d3 = d[u + 3];
                    for (int l = 0; l < N; ++l) hq[l] = (((hq[l] + d0 * r0[l]) + d1 * r1[l]) + d2 * r2[l]) + d3 * r3[l];
                }
                for (; u < cnt; ++u) {
                    const double* __restrict__ row = Q + (int64_t)S[nz[u]] * N;
                    const double du = d[u];
                    for (int l = 0; l < N; ++l) hq[l] += du * row[l];
                }
                energy += dE;
                ++accepted;
                xs = 0;
                for (int a = 0; a < k; ++a) {
                    xs |= (uint64_t)(x[S[a]] != 0) << a;
                    h2[a] = 2.0 * hq[S[a]];
                }
            }
        }
    }
    return accepted;
}

void merge_setup_from(int N, const uint8_t* x, const double* h, const double* colabs, MergeCache* cache) {
    double absq = 0.0;
    for (int l = 0; l < N; ++l) absq += colabs[l];
    cache->tau = 1e-12 * absq;
    cache->h.assign(h, h + N);
    double energy = 0.0;
    for (int i = 0; i < N; ++i)
        if (x[i]) energy += h[i];
    cache->energy = energy;
    cache->valid = true;
}

void merge_setup_host(const double* Q, int N, const uint8_t* x, MergeCache* cache) {
    constexpr int RB = MERGE_RB;   // rows per block, as in the device set-up
    std::vector<double> h(N, 0.0), a(N, 0.0), hb(N), ab(N);
    for (int i0 = 0; i0 < N; i0 += RB) {
        std::fill(hb.begin(), hb.end(), 0.0);
        std::fill(ab.begin(), ab.end(), 0.0);
        const int i1 = std::min(N, i0 + RB);
        double* __restrict__ hp = hb.data();
        double* __restrict__ ap = ab.data();
        for (int i = i0; i < i1; ++i) {
            const double* __restrict__ row = Q + (int64_t)i * N;
            for (int l = 0; l < N; ++l) ap[l] += std::fabs(row[l]);
            if (x[i])
                for (int l = 0; l < N; ++l) hp[l] += row[l];
        }
        for (int l = 0; l < N; ++l) {
            h[l] += hb[l];
            a[l] += ab[l];
        }
    }
    merge_setup_from(N, x, h.data(), a.data(), cache);
}

int merge(const double* Q, int N, uint8_t* x, int m, int k, const int32_t* idx, int K,
          const uint64_t* cand, double* energy_out, int* accepted_out, MergeCache* cache,
          const double* qblk, const double* pair) {
    MergeCache local;
    MergeCache* mc = cache ? cache : &local;
    if (!mc->valid) merge_setup_host(Q, N, x, mc);
    double energy = mc->energy;
    const double tau = mc->tau;
    uint8_t* chg = nullptr;
    if (pair) {
        if (mc->chg.size() != (size_t)N) mc->chg.assign(N, 0);
        chg = mc->chg.data();
    } else {
        pair = nullptr;
    }
    int accepted;
    double* hp0 = mc->h.data();
    if (!qblk) accepted = merge_loop<false, 0>(Q, N, x, m, k, idx, K, cand, qblk, tau, hp0, energy, pair, chg);
    else if (k == 16) accepted = merge_loop<true, 16>(Q, N, x, m, k, idx, K, cand, qblk, tau, hp0, energy, pair, chg);
    else if (k == 12) accepted = merge_loop<true, 12>(Q, N, x, m, k, idx, K, cand, qblk, tau, hp0, energy, pair, chg);
    else if (k == 20) accepted = merge_loop<true, 20>(Q, N, x, m, k, idx, K, cand, qblk, tau, hp0, energy, pair, chg);
    else accepted = merge_loop<true, 0>(Q, N, x, m, k, idx, K, cand, qblk, tau, hp0, energy, pair, chg);
    if (energy_out) *energy_out = energy;
    if (accepted_out) *accepted_out = accepted;
    mc->energy = energy;
    return 0;
}

}  // namespace qaoa
