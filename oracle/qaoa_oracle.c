/*
 * qaoa_oracle.c -- plain FP64 CPU oracle for the QAOA state-vector hot path and the DQAOA
 * decompose / merge steps (arXiv 2506.10531, "GPU-Accelerated Distributed QAOA on Large-scale
 * HPC Ecosystems").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or calls this file; only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark use it. It shares no
 * code with the CUDA library: every formula below is written from the paper's definitions,
 * directly and slowly, in FP64 / complex128, so that a reader can check it against the paper
 * by eye.
 *
 * Conventions (the paper is silent on these; the readings are listed with the design notes):
 *   - QUBO energy E(z) = z^T Q z with Q symmetric (off-diagonal pairs count twice);
 *   - bit q of the basis index z is qubit q, which is sub-QUBO variable S[q];
 *   - ansatz (Section IV, Eq. 2): |psi> = prod_{l=1..p} e^{-i beta_l B_s} e^{-i gamma_l H} |+>,
 *     layer 1 acting first, H|z> = E(z)|z>, B_s = s * sum_q X_q with s = +1 for the
 *     e^{-i beta sum X} mixer and s = -1 for the paper's printed H_X = -sum_q X_q;
 *   - top-k: probability descending, ties broken by the smaller index z.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (see oracle/__init__.py).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------------------------------ */
/* QUBO energies (Section IV, Eq. 1 and the mapping of a QUBO to the diagonal problem          */
/* Hamiltonian H|z> = E(z)|z>).                                                                 */
/* ------------------------------------------------------------------------------------------ */

/* E(z) = sum_i sum_j Q_ij z_i z_j, evaluated directly for every z (O(n^2) each). */
int orc_energies(int n, const double* Q, double* E)
{
    if (n < 1 || n > 34 || !Q || !E) return ORC_EINVAL;
    const int64_t D = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < D; ++z) {
        double e = 0.0;
        for (int i = 0; i < n; ++i) {
            const double zi = (double)((z >> i) & 1);
            for (int j = 0; j < n; ++j) {
                const double zj = (double)((z >> j) & 1);
                e += Q[(int64_t)i * n + j] * zi * zj;
            }
        }
        E[z] = e;
    }
    return ORC_OK;
}

/* x^T Q x for one bitstring x of length N (bytes 0/1), summed row by row, ascending. */
double orc_qubo_energy(const double* Q, int N, const uint8_t* x)
{
    double e = 0.0;
    for (int i = 0; i < N; ++i) {
        if (!x[i]) continue;
        for (int j = 0; j < N; ++j)
            if (x[j]) e += Q[(int64_t)i * N + j];
    }
    return e;
}

/* ------------------------------------------------------------------------------------------ */
/* State-vector simulation (Section IV, Eq. 2).                                                 */
/* ------------------------------------------------------------------------------------------ */

/* psi(z) <- e^{-i gamma E(z)} psi(z): the cost layer e^{-i gamma H}. */
static void cost_layer(int64_t D, const double* E, double gamma, cplx* psi)
{
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < D; ++z) {
        const double th = gamma * E[z];
        psi[z] *= cos(th) - I * sin(th);
    }
}

/* psi <- prod_q e^{-i beta s X_q} psi. Each factor is the 2x2 matrix
 * [[cos b, -i s sin b], [-i s sin b, cos b]] on the amplitude pair (z, z | 2^q), bit q of z clear.
 * The factors commute, so the qubit order does not matter. */
static void mixer_layer(int n, double beta, int s, cplx* psi)
{
    const int64_t D = (int64_t)1 << n;
    const double c = cos(beta), sn = (double)s * sin(beta);
    for (int q = 0; q < n; ++q) {
        const int64_t bit = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < D; ++z) {
            if (z & bit) continue;
            const cplx a = psi[z], b = psi[z | bit];
            psi[z] = c * a - I * sn * b;
            psi[z | bit] = -I * sn * a + c * b;
        }
    }
}

/* Full ansatz from |+> = 2^{-n/2} sum_z |z>; layer l applies cost(gamma_l) then mixer(beta_l). */
int orc_state(int n, int p, const double* gamma, const double* beta, const double* E,
              int mixer_sign, cplx* psi)
{
    if (n < 1 || n > 34 || p < 0 || !E || !psi || (p > 0 && (!gamma || !beta))) return ORC_EINVAL;
    if (mixer_sign != 1 && mixer_sign != -1) return ORC_EINVAL;
    const int64_t D = (int64_t)1 << n;
    const double amp = pow(2.0, -0.5 * n);
    for (int64_t z = 0; z < D; ++z) psi[z] = amp;
    for (int l = 0; l < p; ++l) {
        cost_layer(D, E, gamma[l], psi);
        mixer_layer(n, beta[l], mixer_sign, psi);
    }
    return ORC_OK;
}

/* Apply layers to a given state (no |+> initialisation). */
int orc_apply_layers(int n, int p, const double* gamma, const double* beta, const double* E,
                     int mixer_sign, cplx* psi)
{
    if (n < 1 || n > 34 || p < 0 || !E || !psi) return ORC_EINVAL;
    const int64_t D = (int64_t)1 << n;
    for (int l = 0; l < p; ++l) {
        cost_layer(D, E, gamma[l], psi);
        mixer_layer(n, beta[l], mixer_sign, psi);
    }
    return ORC_OK;
}

/* <C> = sum_z |psi(z)|^2 E(z), a plain ascending FP64 sum. */
double orc_expect(int n, const cplx* psi, const double* E)
{
    const int64_t D = (int64_t)1 << n;
    double acc = 0.0;
    for (int64_t z = 0; z < D; ++z) {
        const double pr = creal(psi[z]) * creal(psi[z]) + cimag(psi[z]) * cimag(psi[z]);
        acc += pr * E[z];
    }
    return acc;
}

/* |psi(z)|^2 = re^2 + im^2 (no fused multiply-add: the file is built with fp-contract off). */
void orc_probs(int64_t D, const cplx* psi, double* prob)
{
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < D; ++z)
        prob[z] = creal(psi[z]) * creal(psi[z]) + cimag(psi[z]) * cimag(psi[z]);
}

/* Measurement shots (Section IV: the sub-solution is read from measurements of the final state;
 * the paper's simulators sample shots). Shot s returns the smallest z whose cumulative
 * probability C(z) = sum_{y <= z} prob[y] (FP64, ascending y) exceeds u[s] * C(D - 1), i.e.
 * inverse-CDF sampling with the caller's uniforms u[s] in [0, 1). A target that no cumulative
 * sum exceeds (only possible through rounding) returns the largest z with nonzero probability. */
int orc_sample_probs(int64_t D, const double* prob, int64_t shots, const double* u, uint64_t* out)
{
    if (D < 1 || shots < 0 || !prob || (shots > 0 && (!u || !out))) return ORC_EINVAL;
    double* cdf = (double*)malloc(sizeof(double) * (size_t)D);
    if (!cdf) return ORC_ENOMEM;
    double acc = 0.0;
    int64_t last = 0;
    for (int64_t z = 0; z < D; ++z) {
        acc += prob[z];
        cdf[z] = acc;
        if (prob[z] > 0.0) last = z;
    }
    for (int64_t s = 0; s < shots; ++s) {
        const double t = u[s] * acc;
        /* binary search for the first cdf[z] > t */
        int64_t lo = 0, hi = D;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        out[s] = (uint64_t)(lo < D ? lo : last);
    }
    free(cdf);
    return ORC_OK;
}

/* k most probable indices: probability descending, ties to the smaller z. Plain insertion into
 * a sorted list of length k over one ascending scan; prob_out may be NULL. */
int orc_topk_probs(int64_t D, const double* prob, int k, uint64_t* idx, double* prob_out)
{
    if (k < 1 || (int64_t)k > D || !prob || !idx) return ORC_EINVAL;
    int cnt = 0;
    double* bp = (double*)malloc(sizeof(double) * (size_t)k);
    uint64_t* bz = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)k);
    if (!bp || !bz) { free(bp); free(bz); return ORC_ENOMEM; }
    for (int64_t z = 0; z < D; ++z) {
        const double v = prob[z];
        /* a later z never beats an equal earlier one, so strictly greater is required */
        if (cnt == k && !(v > bp[k - 1])) continue;
        int pos = (cnt < k) ? cnt : k - 1;
        while (pos > 0 && v > bp[pos - 1]) {
            bp[pos] = bp[pos - 1];
            bz[pos] = bz[pos - 1];
            --pos;
        }
        bp[pos] = v;
        bz[pos] = (uint64_t)z;
        if (cnt < k) ++cnt;
    }
    for (int i = 0; i < k; ++i) {
        idx[i] = bz[i];
        if (prob_out) prob_out[i] = bp[i];
    }
    free(bp);
    free(bz);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Adjoint gradient of <C> with respect to (gamma, beta): the reverse state-vector sweep of    */
/* Jones & Gacon (2020). With lambda = E psi_p, for l = p..1:                                   */
/*   dC/dbeta_l  = 2 s Im <lambda| sum_q X_q |psi>,  then psi, lambda <- mixer_l^dagger,        */
/*   dC/dgamma_l = 2 Im <lambda| E |psi>,            then psi, lambda <- cost_l^dagger.         */
/* ------------------------------------------------------------------------------------------ */
int orc_grad(int n, int p, const double* gamma, const double* beta, const double* E,
             int mixer_sign, double* expect, double* dgamma, double* dbeta)
{
    if (n < 1 || n > 32 || p < 1 || !gamma || !beta || !E || !dgamma || !dbeta) return ORC_EINVAL;
    const int64_t D = (int64_t)1 << n;
    cplx* psi = (cplx*)malloc(sizeof(cplx) * (size_t)D);
    cplx* lam = (cplx*)malloc(sizeof(cplx) * (size_t)D);
    if (!psi || !lam) { free(psi); free(lam); return ORC_ENOMEM; }
    orc_state(n, p, gamma, beta, E, mixer_sign, psi);
    if (expect) *expect = orc_expect(n, psi, E);
    for (int64_t z = 0; z < D; ++z) lam[z] = E[z] * psi[z];
    for (int l = p - 1; l >= 0; --l) {
        cplx acc = 0.0;
        for (int q = 0; q < n; ++q) {
            const int64_t bit = (int64_t)1 << q;
            for (int64_t z = 0; z < D; ++z) acc += conj(lam[z]) * psi[z ^ bit];
        }
        dbeta[l] = 2.0 * (double)mixer_sign * cimag(acc);
        mixer_layer(n, -beta[l], mixer_sign, psi);
        mixer_layer(n, -beta[l], mixer_sign, lam);
        acc = 0.0;
        for (int64_t z = 0; z < D; ++z) acc += conj(lam[z]) * E[z] * psi[z];
        dgamma[l] = 2.0 * cimag(acc);
        cost_layer(D, E, -gamma[l], psi);
        cost_layer(D, E, -gamma[l], lam);
    }
    free(psi);
    free(lam);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* DQAOA decomposition (Section V-A).                                                          */
/* ------------------------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood 2014): state += golden gamma, then the 64-bit finaliser. */
static uint64_t sm64_next(uint64_t* state)
{
    *state += 0x9E3779B97F4A7C15ULL;
    uint64_t z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Exported for the test-vector pin. */
void orc_splitmix64(uint64_t seed, int count, uint64_t* out)
{
    uint64_t s = seed;
    for (int i = 0; i < count; ++i) out[i] = sm64_next(&s);
}

/* Uniform integer in [0, range) by Lemire's multiply-shift with rejection ("Fast random integer
 * generation in an interval", ACM TOMACS 2019): take the high 64 bits of x * range, rejecting
 * draws whose low 64 bits fall below 2^64 mod range. */
static uint64_t bounded_draw(uint64_t* state, uint64_t range)
{
    uint64_t x = sm64_next(state);
    __uint128_t m = (__uint128_t)x * range;
    uint64_t low = (uint64_t)m;
    if (low < range) {
        const uint64_t threshold = (0 - range) % range;
        while (low < threshold) {
            x = sm64_next(state);
            m = (__uint128_t)x * range;
            low = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

static int cmp_i32(const void* a, const void* b)
{
    const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Impact factor of variable i: the change of x^T Q x when x_i is flipped in the current solution
 * (Section V-A, IFD): dE_i = (1 - 2 x_i) (Q_ii + 2 sum_{j != i} Q_ij x_j). */
void orc_impact(const double* Q, int N, const uint8_t* x, double* dE)
{
    for (int i = 0; i < N; ++i) {
        double h = 0.0;
        for (int j = 0; j < N; ++j)
            if (j != i && x[j]) h += Q[(int64_t)i * N + j];
        dE[i] = (1.0 - 2.0 * (double)x[i]) * (Q[(int64_t)i * N + i] + 2.0 * h);
    }
}

/* Ranking of Algorithm 1's impact_analysis, ties to the smaller index. Section V-A ranks by the
 * impact factor without saying whether a large energy increase counts as a high impact: the
 * default reading ranks by |dE_i| descending; with `signed` the ranking is dE_i ascending (the
 * largest energy decrease first). */
static void impact_ranking(const double* Q, int N, const uint8_t* x, int32_t* order, int signed_rank)
{
    double* dE = (double*)malloc(sizeof(double) * (size_t)N);
    orc_impact(Q, N, x, dE);
    double* key = (double*)malloc(sizeof(double) * (size_t)N);
    /* key descending = rank order */
    for (int i = 0; i < N; ++i) key[i] = signed_rank ? -dE[i] : fabs(dE[i]);
    for (int i = 0; i < N; ++i) order[i] = i;
    /* insertion sort: plain and stable */
    for (int i = 1; i < N; ++i) {
        const int32_t v = order[i];
        int j = i;
        while (j > 0 && key[order[j - 1]] < key[v]) {
            order[j] = order[j - 1];
            --j;
        }
        order[j] = v;
    }
    free(key);
    free(dE);
}

/* Strong interactions (Section V-A, BFS/PFS; the paper leaves "strongly interacted" open). Read
 * here as: j is a strong neighbour of i when j != i, Q_ij != 0 and |Q_ij| is at least the d-th
 * largest off-diagonal magnitude of row i, d = min(k - 1, nonzeros of the row off the diagonal);
 * ties at the threshold are all strong (every edge of an unweighted graph is strong). thr[i] is
 * that threshold, or +inf for a row without off-diagonal nonzeros. */
static void strong_thresholds(const double* Q, int N, int k, double* thr)
{
    double* mag = (double*)malloc(sizeof(double) * (size_t)N);
    for (int i = 0; i < N; ++i) {
        int nz = 0;
        for (int j = 0; j < N; ++j)
            if (j != i && Q[(int64_t)i * N + j] != 0.0) mag[nz++] = fabs(Q[(int64_t)i * N + j]);
        const int d = (k - 1 < nz) ? k - 1 : nz;
        if (d < 1) { thr[i] = INFINITY; continue; }
        /* selection by repeated maximum: the d-th largest value */
        double t = INFINITY;
        for (int r = 0; r < d; ++r) {
            int best = -1;
            for (int a = 0; a < nz; ++a)
                if (mag[a] <= t && (best < 0 || mag[a] > mag[best])) best = a;
            /* remove one copy of the maximum so that equal values count once each */
            t = mag[best];
            mag[best] = -1.0;
        }
        thr[i] = t;
    }
    free(mag);
}

static int strong(const double* Q, int N, const double* thr, int i, int j)
{
    const double q = Q[(int64_t)i * N + j];
    return j != i && q != 0.0 && fabs(q) >= thr[i];
}

/* Sub-QUBO j of the graph traversals (Section V-A, BFS / PFS), rooted at rank[j] (the j-th
 * variable by impact, as Algorithm 1's windows start at rank[j]):
 *   BFS: a FIFO queue; the front variable's strong neighbours join in ascending index order;
 *   PFS: the next variable is the unselected one of highest impact (rank order) among the
 *        strong neighbours of the selected variables.
 * When the traversal runs out before k variables, it restarts from the best-ranked unselected
 * variable. S receives the k variables in selection order. */
static void traverse(const double* Q, int N, const double* thr, const int32_t* rank, int method,
                     int j, int k, int32_t* S, uint8_t* inS, uint8_t* inF, int32_t* queue)
{
    memset(inS, 0, (size_t)N);
    memset(inF, 0, (size_t)N);
    int size = 0, head = 0, tail = 0;
    int32_t next = rank[j];
    while (size < k) {
        if (next < 0) {
            /* restart: best-ranked unselected variable */
            for (int t = 0; t < N; ++t)
                if (!inS[rank[t]]) { next = rank[t]; break; }
        }
        const int32_t v = next;
        next = -1;
        S[size++] = v;
        inS[v] = 1;
        if (method == 2) {
            queue[tail++] = v;
            /* expand queued variables until one neighbour is found or the queue empties */
            while (size < k && head < tail) {
                const int32_t w = queue[head++];
                for (int u = 0; u < N && size < k; ++u)
                    if (!inS[u] && strong(Q, N, thr, w, u)) {
                        S[size++] = u;
                        inS[u] = 1;
                        queue[tail++] = u;
                    }
            }
        } else {
            for (int u = 0; u < N; ++u)
                if (strong(Q, N, thr, v, u)) inF[u] = 1;
            for (int t = 0; t < N; ++t)
                if (inF[rank[t]] && !inS[rank[t]]) { next = rank[t]; break; }
        }
    }
}

/*
 * Decompose the N-variable QUBO into m sub-QUBOs of k variables.
 *   method 0 (random, Section V-A): sub-QUBO j draws k distinct variables uniformly without
 *     replacement with SplitMix64 seeded by seed ^ (cycle * 0x9E3779B97F4A7C15) ^ j, by a partial
 *     Fisher-Yates shuffle of 0..N-1 (swap position i with i + draw(N - i)), then sorts them.
 *   method 1 (IFD, Algorithm 1): variables ranked by impact; sub-QUBO j takes the window
 *     ranking[j .. j+k-1] and sorts it (requires m + k - 1 <= N).
 *   methods 2 (BFS) and 3 (PFS): the traversals above from rank[j], sorted (requires m <= N).
 *   methods 1-3 plus 16: the same with the signed impact ranking (see impact_ranking).
 * Qsub[j] = Q[S_j, S_j] as a full symmetric k x k matrix. With conditioned != 0 the couplings to
 * the fixed variables outside S_j are folded into the diagonal:
 *   Qsub[a][a] += 2 sum_{l not in S_j} Q[S_a][l] x_l,
 * so that the sub-QUBO energy of y equals E(x with x_S = y) minus a constant. The sum is the plain
 * FP64 sum over l = 0..N-1 in ascending order.
 */
int orc_decompose(const double* Q, int N, const uint8_t* x, int method_flags, int conditioned, int m,
                  int k, uint64_t seed, uint64_t cycle, int32_t* idx, double* Qsub)
{
    /* method_flags: the method in the low four bits, bit 4 (16) selects the signed ranking */
    const int method = method_flags & 15, signed_rank = (method_flags >> 4) & 1;
    if ((method_flags & ~31) || (signed_rank && method == 0)) return ORC_EINVAL;
    if (!Q || N < 1 || m < 1 || k < 1 || k > N || !idx || !Qsub) return ORC_EINVAL;
    if ((conditioned || method == 1) && !x) return ORC_EINVAL;
    if (method == 1 && m + k - 1 > N) return ORC_EINVAL;
    if ((method == 2 || method == 3) && m > N) return ORC_EINVAL;
    if (method < 0 || method > 3) return ORC_EINVAL;
    if (method >= 1 && !x) return ORC_EINVAL;
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    uint8_t* inS = (uint8_t*)malloc((size_t)N);
    uint8_t* inF = (uint8_t*)malloc((size_t)N);
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    double* thr = (double*)malloc(sizeof(double) * (size_t)N);
    if (!perm || !inS || !inF || !queue || !thr) {
        free(perm); free(inS); free(inF); free(queue); free(thr);
        return ORC_ENOMEM;
    }
    if (method >= 1) impact_ranking(Q, N, x, perm, signed_rank);
    if (method >= 2) strong_thresholds(Q, N, k, thr);
    for (int j = 0; j < m; ++j) {
        int32_t* S = idx + (int64_t)j * k;
        if (method == 0) {
            uint64_t state = seed ^ (cycle * 0x9E3779B97F4A7C15ULL) ^ (uint64_t)j;
            for (int i = 0; i < N; ++i) perm[i] = i;
            for (int i = 0; i < k; ++i) {
                const int r = (int)bounded_draw(&state, (uint64_t)(N - i));
                const int32_t t = perm[i];
                perm[i] = perm[i + r];
                perm[i + r] = t;
            }
            memcpy(S, perm, sizeof(int32_t) * (size_t)k);
        } else if (method == 1) {
            memcpy(S, perm + j, sizeof(int32_t) * (size_t)k);
        } else {
            traverse(Q, N, thr, perm, method, j, k, S, inS, inF, queue);
        }
        qsort(S, (size_t)k, sizeof(int32_t), cmp_i32);
        double* Qs = Qsub + (int64_t)j * k * k;
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b) Qs[a * k + b] = Q[(int64_t)S[a] * N + S[b]];
        if (conditioned) {
            memset(inS, 0, (size_t)N);
            for (int a = 0; a < k; ++a) inS[S[a]] = 1;
            for (int a = 0; a < k; ++a) {
                double h = 0.0;
                for (int l = 0; l < N; ++l)
                    if (!inS[l] && x[l]) h += Q[(int64_t)S[a] * N + l];
                Qs[a * k + a] += 2.0 * h;
            }
        }
    }
    free(perm);
    free(inS);
    free(inF);
    free(queue);
    free(thr);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* DQAOA aggregation (Section V, step 3): fragments of the global solution are replaced by the */
/* sub-solutions, and only updates that lower the energy are accepted.                          */
/* Sequential over j = 0..m-1 and, within j, over the K candidates in their given (top-k)       */
/* order. Candidate bit q sets variable S_j[q]. With d = x' - x:                                */
/*   dE = sum_{a: d_a != 0} d_a (2 sum_l Q[S_a][l] x_l + sum_{b: d_b != 0} Q[S_a][S_b] d_b)     */
/* (a, b ascending over the sub-QUBO, l ascending over 0..N-1). Accepted iff dE < -tau with    */
/* tau = 1e-12 sum |Q_ij|.                                                                      */
/* ------------------------------------------------------------------------------------------ */
int orc_merge(const double* Q, int N, uint8_t* x, int m, int k, const int32_t* idx, int K,
              const uint64_t* cand, double* energy_out, int* accepted_out)
{
    if (!Q || N < 1 || !x || m < 1 || k < 1 || k > 64 || K < 1 || !idx || !cand) return ORC_EINVAL;
    double absq = 0.0;
    for (int64_t t = 0; t < (int64_t)N * N; ++t) absq += fabs(Q[t]);
    const double tau = 1e-12 * absq;
    double energy = orc_qubo_energy(Q, N, x);
    int accepted = 0;
    double d[64];
    for (int j = 0; j < m; ++j) {
        const int32_t* S = idx + (int64_t)j * k;
        for (int c = 0; c < K; ++c) {
            const uint64_t y = cand[(int64_t)j * K + c];
            for (int a = 0; a < k; ++a) d[a] = (double)((y >> a) & 1) - (double)x[S[a]];
            double dE = 0.0;
            for (int a = 0; a < k; ++a) {
                if (d[a] == 0.0) continue;
                double h = 0.0;
                for (int l = 0; l < N; ++l)
                    if (x[l]) h += Q[(int64_t)S[a] * N + l];
                double inner = 0.0;
                for (int b = 0; b < k; ++b)
                    if (d[b] != 0.0) inner += Q[(int64_t)S[a] * N + S[b]] * d[b];
                dE += d[a] * (2.0 * h + inner);
            }
            if (dE < -tau) {
                for (int a = 0; a < k; ++a) x[S[a]] = (uint8_t)((y >> a) & 1);
                energy += dE;
                ++accepted;
            }
        }
    }
    if (energy_out) *energy_out = energy;
    if (accepted_out) *accepted_out = accepted;
    return ORC_OK;
}
