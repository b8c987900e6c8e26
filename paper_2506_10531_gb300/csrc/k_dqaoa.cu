// k_dqaoa.cu -- device construction of the sub-QUBO matrices of one DQAOA cycle
// (Section V-A): Qsub[j] = Q[S_j, S_j], optionally conditioned on the current global solution
// by folding 2 sum_{l not in S_j} Q[S_a][l] x_l into the diagonal.
#include <cuda_runtime.h>
#include <stdint.h>

namespace qaoa {

namespace {

// One CTA per sub-QUBO. The conditioning term of row a is the FP64 sum over l not in S with
// x_l = 1 of Q[S_a][l], taken as eight partial sums over l = r (mod 8) (thread 8a + r, ascending
// l) combined pairwise ((s0+s1)+(s2+s3))+((s4+s5)+(s6+s7)) by xor-shuffles within the row's eight
// lanes (addition is commutative, so every lane ends with the same bits). The rows are staged
// through shared memory in chunks of SQ_CHUNK columns, loaded by all warps with coalesced reads.
// All threads then write the k*k FP32 entries and, when qblk is given, the raw FP64 block
// Q[S, S] (the merge evaluates its candidates on it).
constexpr int SQ_CHUNK = 128;

__global__ void __launch_bounds__(256) k_subqubo(const double* __restrict__ Q, int N,
                                                 const uint8_t* __restrict__ x, int k,
                                                 const int32_t* __restrict__ idx, int conditioned,
                                                 float* __restrict__ qsub, double* __restrict__ qblk) {
    extern __shared__ __align__(8) unsigned char sq_smem[];
    double* rows = reinterpret_cast<double*>(sq_smem);                    // k x (SQ_CHUNK + 1)
    int32_t* S = reinterpret_cast<int32_t*>(rows + (size_t)k * (SQ_CHUNK + 1));
    uint8_t* xm = reinterpret_cast<uint8_t*>(S + k);
    const int j = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a = threadIdx.x; a < k; a += blockDim.x) S[a] = idx[(int64_t)j * k + a];
    if (conditioned)
        for (int l = threadIdx.x; l < N; l += blockDim.x) xm[l] = x[l];
    __syncthreads();
    if (conditioned) {
        for (int a = threadIdx.x; a < k; a += blockDim.x) xm[S[a]] = 0;
    }
    __syncthreads();
    float* out = qsub + (int64_t)j * k * k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int a = e / k, b = e % k;
        const double q = Q[(int64_t)S[a] * N + S[b]];
        if (a != b || !conditioned) out[e] = (float)q;
        if (qblk) qblk[(int64_t)j * k * k + e] = q;
    }
    if (!conditioned) return;
    const int ra = threadIdx.x >> 3, rr = threadIdx.x & 7;   // row and residue of this thread
    double h = 0.0;
    for (int c0 = 0; c0 < N; c0 += SQ_CHUNK) {
        const int len = min(SQ_CHUNK, N - c0);
        for (int a = warp; a < k; a += nw) {
            const double* row = Q + (int64_t)S[a] * N + c0;
            for (int l = lane; l < len; l += 32) rows[a * (SQ_CHUNK + 1) + l] = row[l];
        }
        __syncthreads();
        if (ra < k) {
            const double* r = rows + ra * (SQ_CHUNK + 1);
            // c0 is a multiple of 8, so column c0 + l has residue l mod 8
            for (int l = rr; l < len; l += 8)
                if (xm[c0 + l]) h += r[l];
        }
        __syncthreads();
    }
    h = h + __shfl_xor_sync(0xffffffffu, h, 1);
    h = h + __shfl_xor_sync(0xffffffffu, h, 2);
    h = h + __shfl_xor_sync(0xffffffffu, h, 4);
    if (ra < k && rr == 0) out[ra * k + ra] = (float)(Q[(int64_t)S[ra] * N + S[ra]] + 2.0 * h);
}

}  // namespace

cudaError_t launch_subqubo(const double* Q, int N, const uint8_t* x, int m, int k,
                           const int32_t* idx, int conditioned, float* qsub, cudaStream_t st,
                           double* qblk) {
    const size_t sm = (size_t)k * (SQ_CHUNK + 1) * sizeof(double) + k * sizeof(int32_t) + (size_t)N;
    if (sm > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_subqubo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    // eight threads per row (k <= 30): 256 threads cover every row
    k_subqubo<<<m, 256, sm, st>>>(Q, N, x, k, idx, conditioned, qsub, qblk);
    return cudaGetLastError();
}

}  // namespace qaoa
