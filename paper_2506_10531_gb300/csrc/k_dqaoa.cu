// k_dqaoa.cu -- device construction of the sub-QUBO matrices of one DQAOA cycle
// (Section V-A): Qsub[j] = Q[S_j, S_j], optionally conditioned on the current global solution
// by folding 2 sum_{l not in S_j} Q[S_a][l] x_l into the diagonal.
#include <cuda_runtime.h>
#include <stdint.h>

namespace qaoa {

namespace {

// One CTA per sub-QUBO; thread a < k sums the conditioning term of row a sequentially in
// ascending l (FP64, additions only), then all threads write the k*k FP32 entries.
__global__ void k_subqubo(const double* __restrict__ Q, int N, const uint8_t* __restrict__ x,
                          int k, const int32_t* __restrict__ idx, int conditioned,
                          float* __restrict__ qsub) {
    extern __shared__ int32_t S[];
    const int j = blockIdx.x;
    for (int a = threadIdx.x; a < k; a += blockDim.x) S[a] = idx[(int64_t)j * k + a];
    __syncthreads();
    float* out = qsub + (int64_t)j * k * k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int a = e / k, b = e % k;
        if (a != b || !conditioned) out[e] = (float)Q[(int64_t)S[a] * N + S[b]];
    }
    if (conditioned) {
        for (int a = threadIdx.x; a < k; a += blockDim.x) {
            const double* row = Q + (int64_t)S[a] * N;
            double h = 0.0;
            int sp = 0;
            for (int l = 0; l < N; ++l) {
                if (sp < k && S[sp] == l) { ++sp; continue; }
                if (x[l]) h += row[l];
            }
            out[a * k + a] = (float)(row[S[a]] + 2.0 * h);
        }
    }
}

}  // namespace

cudaError_t launch_subqubo(const double* Q, int N, const uint8_t* x, int m, int k,
                           const int32_t* idx, int conditioned, float* qsub, cudaStream_t st) {
    k_subqubo<<<m, 64, k * sizeof(int32_t), st>>>(Q, N, x, k, idx, conditioned, qsub);
    return cudaGetLastError();
}

}  // namespace qaoa
