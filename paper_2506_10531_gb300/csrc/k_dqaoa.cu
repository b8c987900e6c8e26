// k_dqaoa.cu -- device construction of the sub-QUBO matrices of one DQAOA cycle
// (Section V-A): Qsub[j] = Q[S_j, S_j], optionally conditioned on the current global solution
// by folding 2 sum_{l not in S_j} Q[S_a][l] x_l into the diagonal.
#include <cuda_runtime.h>
#include <stdint.h>

namespace qaoa {

namespace {

// One CTA per sub-QUBO; thread a < k sums the conditioning term of row a sequentially in
// ascending l (FP64, additions only), then all threads write the k*k FP32 entries. The
// solution x is staged in shared memory as a 0/1 mask with the sub-QUBO's own variables
// cleared, and the row is read 8 values at a time so the loads overlap the dependent adds.
__global__ void k_subqubo(const double* __restrict__ Q, int N, const uint8_t* __restrict__ x,
                          int k, const int32_t* __restrict__ idx, int conditioned,
                          float* __restrict__ qsub) {
    extern __shared__ int32_t S[];
    uint8_t* xm = reinterpret_cast<uint8_t*>(S + k);
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
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int a = e / k, b = e % k;
        if (a != b || !conditioned) out[e] = (float)Q[(int64_t)S[a] * N + S[b]];
    }
    if (conditioned) {
        for (int a = threadIdx.x; a < k; a += blockDim.x) {
            const double* row = Q + (int64_t)S[a] * N;
            double h = 0.0;
            int l = 0;
            for (; l + 8 <= N; l += 8) {
                double v[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) v[t] = row[l + t];
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (xm[l + t]) h += v[t];
            }
            for (; l < N; ++l)
                if (xm[l]) h += row[l];
            out[a * k + a] = (float)(row[S[a]] + 2.0 * h);
        }
    }
}

}  // namespace

cudaError_t launch_subqubo(const double* Q, int N, const uint8_t* x, int m, int k,
                           const int32_t* idx, int conditioned, float* qsub, cudaStream_t st) {
    const size_t sm = k * sizeof(int32_t) + (size_t)N;
    k_subqubo<<<m, 64, sm, st>>>(Q, N, x, k, idx, conditioned, qsub);
    return cudaGetLastError();
}

}  // namespace qaoa
