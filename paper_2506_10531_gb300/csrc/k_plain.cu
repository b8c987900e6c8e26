// k_plain.cu -- the plain one-instance, one-kernel-per-gate GPU path: the straightforward way
// to run Eq. 2 (Section IV) on a GPU, kept as the comparison point of the batched tiers.
// Per instance: an energy kernel, then per layer one cost-phase kernel and one kernel per
// qubit for the mixer, then the standalone reductions. Every kernel streams the whole state.
#include "qaoa_common.cuh"
#include "qaoa_stream.h"

namespace qaoa {

namespace {

__global__ void k_plain_init(uint64_t D, float amp, float2* psi) {
    const uint64_t z = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (z < D) psi[z] = make_float2(amp, 0.0f);
}

__global__ void k_plain_phase(uint64_t D, const float* __restrict__ E, const float* __restrict__ gamma,
                              int l, float2* __restrict__ psi) {
    const uint64_t z = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= D) return;
    float s, c;
    sincos_phase(gamma[l] / 3.14159265358979323846f, E[z], s, c);
    float2 v = psi[z];
    rot_neg(v, s, c);
    psi[z] = v;
}

__global__ void k_plain_rx(uint64_t half, int q, const float* __restrict__ beta, int l,
                           float2* __restrict__ psi) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= half) return;
    const uint64_t lo = t & ((1ull << q) - 1ull);
    const uint64_t z = ((t >> q) << (q + 1)) | lo;
    float s, c;
    sincosf(beta[l], &s, &c);
    // exp(-i beta X): a' = c a - i s b, b' = -i s a + c b
    const float2 a = psi[z], b = psi[z | (1ull << q)];
    psi[z] = make_float2(c * a.x + s * b.y, c * a.y - s * b.x);
    psi[z | (1ull << q)] = make_float2(c * b.x + s * a.y, c * b.y - s * a.x);
}

}  // namespace

cudaError_t launch_plain_layers(int n, int p, const float* gamma, const float* beta,
                                const float* E, float2* psi, int init_plus, cudaStream_t st,
                                int* kernels) {
    const uint64_t D = 1ull << n;
    const int B = 256;
    const unsigned gD = (unsigned)((D + B - 1) / B), gH = (unsigned)((D / 2 + B - 1) / B);
    int cnt = 0;
    if (init_plus) {
        k_plain_init<<<gD, B, 0, st>>>(D, (float)exp2(-0.5 * n), psi);
        ++cnt;
    }
    for (int l = 0; l < p; ++l) {
        k_plain_phase<<<gD, B, 0, st>>>(D, E, gamma, l, psi);
        ++cnt;
        for (int q = 0; q < n; ++q) {
            k_plain_rx<<<gH, B, 0, st>>>(D / 2, q, beta, l, psi);
            ++cnt;
        }
    }
    if (kernels) *kernels = cnt;
    return cudaGetLastError();
}

}  // namespace qaoa

// ---- Adam update of QAOA parameters (Kingma & Ba 2015) --------------------------------------
namespace qaoa {
namespace {
__global__ void k_adam(int count, float* __restrict__ theta, const double* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, int step, float lr, float b1,
                       float b2, float eps, int minimise) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    adam_update(theta[i], m[i], v[i], grad[i], step, lr, b1, b2, eps, minimise);
}
}  // namespace

cudaError_t launch_adam(int count, float* theta, const double* grad, float* m, float* v, int step,
                        float lr, float b1, float b2, float eps, int minimise, cudaStream_t st) {
    k_adam<<<(count + 255) / 256, 256, 0, st>>>(count, theta, grad, m, v, step, lr, b1, b2, eps, minimise);
    return cudaGetLastError();
}
}  // namespace qaoa
