// k_sample.cu -- measurement shots of a complex64 state: inverse-CDF sampling over |psi|^2 with
// uniforms supplied by the caller (Section IV reads the sub-solution from measured shots; the
// default path of this library takes the top-k bitstrings instead).
//
// The 2^n probabilities are cut into P = 2^(n - pb) contiguous parts of 2^pb amplitudes
// (pb = max(n - 12, 0), so P <= 4096):
//   1. k_sample_parts: FP64 sum of each part (one block per part, fixed reduction order);
//   2. k_sample_scan:  exclusive prefix of the part sums and the total, sequential in one thread
//      (at most 4096 adds), so the offsets are exactly the running sums of the parts;
//   3. k_sample_draw:  one warp per shot: t = u * total, the last part whose offset is <= t, then
//      a walk through that part 32 amplitudes at a time with a warp prefix scan until the running
//      sum exceeds t. Every loop is bounded by the part length; nothing waits on another block.
// A batch of states of equal n (a DQAOA cycle's sub-QUBO states, 2^n amplitudes apart) runs as
// one launch of each kernel, the state index in blockIdx.y; each state has its own scratch
// (2P + 1 doubles), uniforms and shots.
#include <cuda_runtime.h>

#include "qaoa_common.cuh"
#include "qaoa_host.h"

namespace qaoa {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__global__ void __launch_bounds__(256) k_sample_parts(const float2* __restrict__ psi, int n, int pb,
                                                      double* __restrict__ scratch) {
    __shared__ double red[8];
    const uint64_t L = 1ull << pb, base = (uint64_t)blockIdx.x << pb;
    psi += (uint64_t)blockIdx.y << n;
    double* part = scratch + (size_t)blockIdx.y * (2 * ((size_t)1 << (n - pb)) + 1);
    double acc = 0.0;
    for (uint64_t u = threadIdx.x; u < L; u += blockDim.x) acc += exact_prob(psi[base + u]);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_sample_scan(double* __restrict__ scratch, int parts) {
    if (threadIdx.x != 0) return;
    const double* part = scratch + (size_t)blockIdx.x * (2 * (size_t)parts + 1);
    double* off = const_cast<double*>(part) + parts;
    double* total = off + parts;
    double acc = 0.0;
    for (int b = 0; b < parts; ++b) {
        off[b] = acc;
        acc += part[b];
    }
    *total = acc;
}

__global__ void __launch_bounds__(256) k_sample_draw(const float2* __restrict__ psi, int n, int pb, int parts,
                                                     const double* __restrict__ scratch, int64_t shots,
                                                     const double* __restrict__ u,
                                                     uint64_t* __restrict__ out) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // one warp per shot
    const int lane = threadIdx.x & 31;
    if (s >= shots) return;                                                    // warp-uniform
    psi += (uint64_t)blockIdx.y << n;
    const double* off = scratch + (size_t)blockIdx.y * (2 * (size_t)parts + 1) + parts;
    const double* total = off + parts;
    u += (size_t)blockIdx.y * shots;
    out += (size_t)blockIdx.y * shots;
    const double t = u[s] * *total;
    // the last part whose offset is <= t (offsets are non-decreasing; parts before a run of
    // empty parts are skipped that way)
    int lo = 0, hi = parts - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const uint64_t L = 1ull << pb, base = (uint64_t)lo << pb;
    double acc = off[lo];
    int64_t lastnz = -1;
    for (uint64_t c0 = 0; c0 < L; c0 += 32) {
        const bool in = c0 + (uint64_t)lane < L;
        const double p = in ? exact_prob(psi[base + c0 + lane]) : 0.0;
        double incl = p;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double o = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += o;
        }
        const unsigned hit = __ballot_sync(FULL, in && acc + incl > t);
        if (hit) {
            if (lane == 0) out[s] = base + c0 + (uint64_t)(__ffs(hit) - 1);
            return;
        }
        const unsigned nz = __ballot_sync(FULL, in && p > 0.0);
        if (nz) lastnz = (int64_t)(base + c0 + (uint64_t)(31 - __clz(nz)));
        acc += __shfl_sync(FULL, incl, 31);
    }
    // no running sum exceeded t (rounding at the part's end): the part's last nonzero amplitude
    if (lane == 0) out[s] = lastnz >= 0 ? (uint64_t)lastnz : base;
}

}  // namespace

int sample_part_bits(int n) { return n > 12 ? n - 12 : 0; }

size_t sample_scratch_bytes(int n) {
    const size_t parts = (size_t)1 << (n - sample_part_bits(n));
    return (2 * parts + 1) * sizeof(double);
}

cudaError_t launch_sample(int n, const void* psi, int count, int64_t shots, const double* u, uint64_t* out,
                          double* scratch, cudaStream_t st) {
    if (count < 1 || count > 65535) return cudaErrorInvalidValue;
    const int pb = sample_part_bits(n);
    const int parts = 1 << (n - pb);
    const float2* ps = static_cast<const float2*>(psi);
    k_sample_parts<<<dim3((unsigned)parts, (unsigned)count), 256, 0, st>>>(ps, n, pb, scratch);
    k_sample_scan<<<(unsigned)count, 32, 0, st>>>(scratch, parts);
    if (shots > 0) {
        const int64_t blocks = (shots * 32 + 255) / 256;
        k_sample_draw<<<dim3((unsigned)blocks, (unsigned)count), 256, 0, st>>>(ps, n, pb, parts, scratch, shots, u,
                                                                              out);
    }
    return cudaGetLastError();
}

}  // namespace qaoa
