// k_dqaoa.cu -- device construction of the sub-QUBO matrices of one DQAOA cycle
// (Section V-A): Qsub[j] = Q[S_j, S_j], optionally conditioned on the current global solution
// by folding 2 sum_{l not in S_j} Q[S_a][l] x_l into the diagonal.
#include <cuda_runtime.h>
#include <stdint.h>

#include "qaoa_host.h"

namespace qaoa {

namespace {

// One CTA per sub-QUBO, one warp per row. The conditioning term of row a is the FP64 sum over
// l not in S with x_l = 1 of Q[S_a][l], taken as 32 partial sums over l = r (mod 32) (lane r,
// ascending l; a warp's loads cover 256 contiguous bytes) combined by the xor tree
// v_r <- v_r + v_{r^d} for d = 16, 8, 4, 2, 1 (addition is commutative, so every lane ends with
// the same bits; build_subqubos adds in the same order). The partial sums are short (N / 32
// terms): a long dependent chain of FP64 adds is slow on this GPU. All threads first write the
// k*k FP32 entries and, when qblk is given, the raw FP64 block Q[S, S] (the merge evaluates its
// candidates on it); when qdiag is given, the FP64 diagonal of the sub-QUBO before its rounding
// to FP32 (Q[S_a][S_a], plus the conditioning term).
__global__ void __launch_bounds__(1024) k_subqubo(const double* __restrict__ Q, int N,
                                                  const uint8_t* __restrict__ x, int k,
                                                  const int32_t* __restrict__ idx, int conditioned,
                                                  float* __restrict__ qsub, double* __restrict__ qblk,
                                                  double* __restrict__ qdiag) {
    extern __shared__ __align__(8) unsigned char sq_smem[];
    int32_t* S = reinterpret_cast<int32_t*>(sq_smem);
    uint8_t* xm = reinterpret_cast<uint8_t*>(S + 32);
    const int j = blockIdx.x;
    for (int a = threadIdx.x; a < k; a += blockDim.x) S[a] = idx[(int64_t)j * k + a];
    if (conditioned)
        for (int l = threadIdx.x; l < N; l += blockDim.x) xm[l] = x[l];
    __syncthreads();
    if (conditioned) {
        for (int a = threadIdx.x; a < k; a += blockDim.x) xm[S[a]] = 0;
    }
    __syncthreads();
    float* out = qsub + (int64_t)j * k * k;
    const int ra = threadIdx.x >> 5, rr = threadIdx.x & 31;   // row and residue of this lane
    const bool rowlane = conditioned && ra < k;               // whole warps
    const double* row = rowlane ? Q + (int64_t)S[ra] * N : nullptr;
    // the first 16 terms of this lane's partial sum are loaded before the element copies, so
    // that both sets of global reads are in flight together
    constexpr int NB = 16;
    double v[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int l = rr + 32 * u;
        v[u] = (rowlane && l < N && xm[l]) ? __ldg(row + l) : 0.0;
    }
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int a = e / k, b = e % k;
        const double q = Q[(int64_t)S[a] * N + S[b]];
        if (a != b || !conditioned) out[e] = (float)q;
        if (qblk) qblk[(int64_t)j * k * k + e] = q;
        if (qdiag && a == b && !conditioned) qdiag[(int64_t)j * k + a] = q;
    }
    if (!rowlane) return;
    double h = 0.0;
#pragma unroll
    for (int u = 0; u < NB; ++u)
        if (rr + 32 * u < N && xm[rr + 32 * u]) h += v[u];
    for (int l0 = rr + 32 * NB; l0 < N; l0 += 256) {
        double w[8];
        bool on[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int l = l0 + 32 * u;
            on[u] = l < N && xm[l];
            w[u] = on[u] ? __ldg(row + l) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (on[u]) h += w[u];
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) h = h + __shfl_xor_sync(0xffffffffu, h, d);
    if (rr == 0) {
        const double d = Q[(int64_t)S[ra] * N + S[ra]] + 2.0 * h;
        out[ra * k + ra] = (float)d;
        if (qdiag) qdiag[(int64_t)j * k + ra] = d;
    }
}

// One CTA per sub-QUBO: E(y) = sum_a y_a (D_a + sum_{b != a} y_b Q_ab), a and b ascending, in
// FP64, for each of its shots; the block keeps the lowest (E, y) pair (ties: smaller y).
__global__ void __launch_bounds__(256) k_best_shot(int k, int shots, const double* __restrict__ qblk,
                                                   const double* __restrict__ qdiag,
                                                   const uint64_t* __restrict__ z, uint64_t* __restrict__ best) {
    __shared__ double sq[32 * 32];
    __shared__ double be[256];
    __shared__ uint64_t bz[256];
    const int j = blockIdx.x;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x)
        sq[e] = (e / k == e % k) ? qdiag[(int64_t)j * k + e / k] : qblk[(int64_t)j * k * k + e];
    __syncthreads();
    double myE = 0.0;
    uint64_t myz = ~0ull;
    bool have = false;
    for (int s = threadIdx.x; s < shots; s += blockDim.x) {
        const uint64_t y = z[(int64_t)j * shots + s];
        double E = 0.0;
        for (int a = 0; a < k; ++a) {
            if (!((y >> a) & 1u)) continue;
            double r = sq[a * k + a];
            for (int b = 0; b < k; ++b)
                if (b != a && ((y >> b) & 1u)) r += sq[a * k + b];
            E += r;
        }
        if (!have || E < myE || (E == myE && y < myz)) { myE = E; myz = y; have = true; }
    }
    be[threadIdx.x] = have ? myE : 0.0;
    bz[threadIdx.x] = have ? myz : ~0ull;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const int o = threadIdx.x + w;
            // an empty slot (no shot) has y = ~0 and loses to every real shot
            const bool take = bz[o] != ~0ull &&
                              (bz[threadIdx.x] == ~0ull || be[o] < be[threadIdx.x] ||
                               (be[o] == be[threadIdx.x] && bz[o] < bz[threadIdx.x]));
            if (take) { be[threadIdx.x] = be[o]; bz[threadIdx.x] = bz[o]; }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) best[j] = bz[0];
}

// Aggregation set-up on the device (Section V step 3), for a merge that starts without a cached
// h = Qx: with rows taken in blocks of MS_RB (short FP64 chains), block b of the grid's y dimension adds, for each
// column l of its x dimension, the rows i of row block b in ascending order, h_b[l] over the
// rows with x_i = 1 and a_b[l] = sum |Q[i][l]| over all of them; k_merge_setup_sum then adds the
// row blocks in ascending order: h[l] = (Q x)_l (Q symmetric: column l = row l) and the column
// sums of |Q| whose total scales the acceptance threshold. merge_setup_host adds in the same
// order, so both give the same bits.
constexpr int MS_RB = MERGE_RB;

__global__ void __launch_bounds__(256) k_merge_setup(const double* __restrict__ Q, int N,
                                                     const uint8_t* __restrict__ x, double* __restrict__ hp,
                                                     double* __restrict__ ap) {
    __shared__ uint8_t xs[MS_RB];
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int i0 = blockIdx.y * MS_RB;
    const int rows = min(MS_RB, N - i0);
    for (int r = threadIdx.x; r < rows; r += blockDim.x) xs[r] = x[i0 + r];
    __syncthreads();
    if (l >= N) return;
    double h = 0.0, a = 0.0;
    const double* q = Q + (int64_t)i0 * N + l;
#pragma unroll 8
    for (int r = 0; r < rows; ++r) {
        const double v = __ldg(q + (int64_t)r * N);
        a += fabs(v);
        if (xs[r]) h += v;
    }
    hp[(int64_t)blockIdx.y * N + l] = h;
    ap[(int64_t)blockIdx.y * N + l] = a;
}

__global__ void __launch_bounds__(256) k_merge_setup_sum(int N, int blocks, const double* __restrict__ hp,
                                                         const double* __restrict__ ap, double* __restrict__ h,
                                                         double* __restrict__ colabs) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= N) return;
    double hs = 0.0, as = 0.0;
    for (int b = 0; b < blocks; ++b) {
        hs += hp[(int64_t)b * N + l];
        as += ap[(int64_t)b * N + l];
    }
    h[l] = hs;
    colabs[l] = as;
}

// The pair term of each candidate's energy change against the solution x the cycle started
// with: d = y - x_S, P = sum_u d_u sum_v Q_{S_u S_v} d_v over the changed positions, FP64, from
// the raw block Q[S, S]. One warp per candidate: lane u sums its row over v ascending, and the
// lanes' terms d_u * inner_u (zero for unchanged u) are added by the xor tree (d = 16 .. 1).
// The merge adds the linear term 2 sum_u d_u (Qx)_{S_u} for the x it has reached.
// With `packed`, the kernel also gathers what the host reads of the chunk into one block (the
// pair terms at `pair`, then the candidates, the <C> values and the plan's status word), so
// that one copy brings them back.
__global__ void __launch_bounds__(256) k_cand_pair(int m, int k, int K, const int32_t* __restrict__ idx,
                                                   const uint8_t* __restrict__ x, const double* __restrict__ qblk,
                                                   const uint64_t* __restrict__ cand, double* __restrict__ pair,
                                                   const double* __restrict__ expect, const unsigned* __restrict__ status,
                                                   int packed) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= (int64_t)m * K) return;   // warp-uniform
    if (packed && lane == 0) {
        uint64_t* cand_out = reinterpret_cast<uint64_t*>(pair + (int64_t)m * K);
        double* expect_out = reinterpret_cast<double*>(cand_out + (int64_t)m * K);
        cand_out[t] = cand[t];
        if (t % K == 0) expect_out[t / K] = expect[t / K];
        if (t == 0) *reinterpret_cast<unsigned*>(expect_out + m) = *status;
    }
    const int64_t j = t / K;
    const int32_t* S = idx + j * k;
    const bool xa = lane < k && x[S[lane]] != 0;
    const uint64_t xs = (uint64_t)__ballot_sync(0xffffffffu, xa);   // k <= 30: one ballot holds x_S
    const uint64_t kmask = (1ull << k) - 1ull;
    const uint64_t y = cand[t], diff = (y ^ xs) & kmask;
    double term = 0.0;
    if (lane < k && ((diff >> lane) & 1u)) {
        const double* row = qblk + j * k * k + (int64_t)lane * k;
        double inner = 0.0;
        for (uint64_t dv = diff; dv; dv &= dv - 1) {
            const int v = __ffsll((long long)dv) - 1;
            const double q = row[v];
            inner = inner + (((y >> v) & 1u) ? q : -q);
        }
        term = ((y >> lane) & 1u) ? inner : -inner;
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) term = term + __shfl_xor_sync(0xffffffffu, term, d);
    if (lane == 0) pair[t] = term;
}

}  // namespace

cudaError_t launch_subqubo(const double* Q, int N, const uint8_t* x, int m, int k,
                           const int32_t* idx, int conditioned, float* qsub, cudaStream_t st,
                           double* qblk, double* qdiag) {
    const size_t sm = 32 * sizeof(int32_t) + (size_t)N;
    if (sm > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_subqubo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    // a warp per row (k <= 30)
    k_subqubo<<<m, 32 * k, sm, st>>>(Q, N, x, k, idx, conditioned, qsub, qblk, qdiag);
    return cudaGetLastError();
}

cudaError_t launch_best_shot(int m, int k, int shots, const double* qblk, const double* qdiag,
                             const uint64_t* z, uint64_t* best, cudaStream_t st) {
    if (k < 1 || k > 32 || shots < 1) return cudaErrorInvalidValue;
    k_best_shot<<<m, 256, 0, st>>>(k, shots, qblk, qdiag, z, best);
    return cudaGetLastError();
}

int merge_setup_blocks(int N) { return (N + MS_RB - 1) / MS_RB; }

cudaError_t launch_merge_setup(const double* Q, int N, const uint8_t* x, double* scratch, double* h,
                               double* colabs, cudaStream_t st) {
    const int rb = merge_setup_blocks(N);
    if (rb > 65535) return cudaErrorInvalidValue;
    double* hp = scratch;
    double* ap = scratch + (size_t)rb * N;
    const unsigned cols = (unsigned)((N + 255) / 256);
    k_merge_setup<<<dim3(cols, (unsigned)rb), 256, 0, st>>>(Q, N, x, hp, ap);
    k_merge_setup_sum<<<cols, 256, 0, st>>>(N, rb, hp, ap, h, colabs);
    return cudaGetLastError();
}

cudaError_t launch_cand_pair(int m, int k, int K, const int32_t* idx, const uint8_t* x, const double* qblk,
                             const uint64_t* cand, double* pair, cudaStream_t st, const double* expect,
                             const unsigned* status) {
    if (m < 1 || k < 1 || k > 30 || K < 1) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)m * K;   // candidates, one warp each
    k_cand_pair<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(m, k, K, idx, x, qblk, cand, pair, expect, status,
                                                          expect && status ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace qaoa
