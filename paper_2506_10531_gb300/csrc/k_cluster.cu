// k_cluster.cu -- cluster tier: one thread-block cluster of C = 2^cb CTAs per QAOA instance
// (complex64, 15 <= n <= 18), the state and its energies distributed over the CTAs' shared
// memory and resident for all p layers of Eq. 2 (Section IV).
//
// CTA rank r of the cluster holds the 2^L amplitudes z = (r << L) | u (L = n - cb local qubits)
// and their energies. Local qubits are mixed by the tile engine exactly as in the resident
// tier. The cb global qubits are mixed by a "global sub-pass": CTA r takes the slab of local
// positions u whose top cb bits equal r, gathers for each such u the C amplitudes
// (j << L) | u, j = 0..C-1, from the C CTAs through distributed shared memory, applies
// exp(-i beta X) on the cb global qubits in registers and writes them back to their owners.
// Slabs of different CTAs are disjoint, so one cluster barrier before and one after the pass
// suffice. In each layer the global sub-pass is placed before the last local window, so the
// snake fusion of consecutive layers (last window, cost, first window) is kept.
// <C> partials and top-k lists of the CTAs are merged by rank 0 through distributed shared
// memory, in rank order (deterministic).
#include <cooperative_groups.h>

#include "qaoa_engine.cuh"
#include "qaoa_kernels.h"

namespace cg = cooperative_groups;

namespace qaoa {

namespace {

struct ClusterSmem {
    float2* psi;
    float* E;
    float* Q;
    LayerConst<float>* lc;
    double* red;     // 32
    double* cex;     // this CTA's <C> partial
    TileTopk tk;     // top-k scratch; tk.out is this CTA's list (read by rank 0)
    float* escr;     // energy-build tables
};

__host__ __device__ inline size_t cl_align(size_t x) { return (x + 15) & ~(size_t)15; }

// One 32-amplitude group per thread per sub-pass.
inline int cluster_threads(int L) { return (1 << L) / 32; }

__host__ __device__ inline size_t cluster_layout(int n, int L, int p, int threads, size_t* off) {
    const size_t D = (size_t)1 << L;
    size_t o = 0;
    off[0] = o; o = cl_align(o + D * sizeof(float2));
    off[1] = o; o = cl_align(o + D * sizeof(float));
    off[2] = o; o = cl_align(o + (size_t)n * n * sizeof(float));
    off[3] = o; o = cl_align(o + (size_t)p * sizeof(LayerConst<float>));
    off[4] = o; o = cl_align(o + 32 * sizeof(double));
    // top-k scratch (used after the last sub-pass) and energy tables (used before the first)
    // share one region
    const size_t r0 = o;
    off[5] = o; o = cl_align(o + (size_t)((threads + 31) / 32) * 32 * sizeof(TopEnt));
    off[6] = o; o = cl_align(o + sizeof(double));
    off[7] = o; o = cl_align(o + 16 * sizeof(TopEnt));
    off[8] = o; o = cl_align(o + TOPK_CAP * sizeof(TopEnt));
    off[9] = o; o = cl_align(o + 16 * 32 * sizeof(float) + 4 * sizeof(int));
    off[10] = r0;
    const size_t eend = cl_align(r0 + tile_energy_scratch(L) * sizeof(float));
    if (eend > o) o = eend;
    return o;
}

// Global sub-pass of layer l: mix the CB global qubits of the slab of this CTA. Each thread
// takes NP = 16 / C slab positions at once so that 16 remote loads are in flight together.
template <int CB>
__device__ void global_subpass(cg::cluster_group& cl, const ClusterSmem& s, int L, uint32_t r,
                               const LayerConst<float>& lc) {
    constexpr int C = 1 << CB;
    constexpr int NP = (16 / C) > 0 ? (16 / C) : 1;
    float2* rp[C];
#pragma unroll
    for (int j = 0; j < C; ++j) rp[j] = cl.map_shared_rank(s.psi, j);
    const uint32_t slab = 1u << (L - CB);
    const uint32_t top = r << (L - CB);
    for (uint32_t w0 = threadIdx.x; w0 < slab; w0 += blockDim.x * NP) {
        float2 v[NP][C];
        uint32_t ix[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const uint32_t w = w0 + (uint32_t)q * blockDim.x;
            ix[q] = swz<float>(top | (w < slab ? w : 0u));
        }
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
            for (int j = 0; j < C; ++j) v[q][j] = rp[j][ix[q]];
#pragma unroll
        for (int q = 0; q < NP; ++q) mix_layer<CB>(v[q], C - 1, lc);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            if (w0 + (uint32_t)q * blockDim.x < slab) {
#pragma unroll
                for (int j = 0; j < C; ++j) rp[j][ix[q]] = v[q][j];
            }
        }
    }
}

template <int CB>
__device__ void run_cluster_instance(cg::cluster_group& cl, const InstDesc<float>& d, int L,
                                     unsigned char* sm) {
    constexpr int R = Num<float>::RB;
    const uint32_t r = cl.block_rank();
    const int n = d.n, p = d.p;
    size_t off[11];
    cluster_layout(n, L, p, blockDim.x, off);
    ClusterSmem s;
    s.psi = reinterpret_cast<float2*>(sm + off[0]);
    s.E = reinterpret_cast<float*>(sm + off[1]);
    s.Q = reinterpret_cast<float*>(sm + off[2]);
    s.lc = reinterpret_cast<LayerConst<float>*>(sm + off[3]);
    s.red = reinterpret_cast<double*>(sm + off[4]);
    s.tk.wlists = reinterpret_cast<TopEnt*>(sm + off[5]);
    s.cex = reinterpret_cast<double*>(sm + off[6]);
    s.tk.out = reinterpret_cast<TopEnt*>(sm + off[7]);
    s.tk.cand = reinterpret_cast<TopEnt*>(sm + off[8]);
    s.tk.wb = reinterpret_cast<float*>(sm + off[9]);
    s.tk.cnt = reinterpret_cast<int*>(sm + off[9] + 16 * 32 * sizeof(float));
    s.escr = reinterpret_cast<float*>(sm + off[10]);
    const uint32_t D = 1u << L;

    set_layer_consts<float>(s.lc, d.gamma, d.beta, p, n, true);
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) s.Q[i] = d.Q[i];
    __syncthreads();
    const FusedInit<float> fi{s.psi, (float)exp2(-0.5 * (double)n),
                              d.gamma[0] / 3.14159265358979323846f, __popc(r)};
    const bool started = build_tile_energy_any<float>(n, L, r << L, s.Q, s.E, s.escr, fi);
    __syncthreads();
    if (d.E_out)
        for (uint32_t u = threadIdx.x; u < D; u += blockDim.x) d.E_out[(r << L) | u] = s.E[swz<float>(u)];

    // ---- forward: local snake with the global sub-pass before each layer's last window ----
    const TileRef<float> tile{s.psi, nullptr, s.E, L};
    const int G = num_windows(0, L, R);
    const int S = snake_len(G, p);
    const float amp0 = (float)exp2(-0.5 * (double)n);
    auto nofin = [](uint32_t, int, bool) {};
    for (int si = 0; si < S; ++si) {
        SubPass sp;
        snake_step(si, G, p, 0, started ? 0 : 1, 0, L, L, R, sp);
        // sub-pass (l+1)(G-1) holds layer l's last local window (fused with the cost and the
        // first window of layer l+1); the global qubits of layer l are mixed just before it,
        // after the cost of layer l (G >= 2: L >= 10 is required by the host)
        const bool closes = (si >= G - 1) && (si % (G - 1) == 0);
        if (closes) {
            cl.sync();
            global_subpass<CB>(cl, s, L, r, s.lc[sp.la]);
            cl.sync();
        }
        sp.post = (si == S - 1);
        subpass_fwd<float, R>(tile, sp, s.lc, si == 0 && !started, amp0, __popc(r), nofin);
        __syncthreads();
    }
    // ---- per-CTA reductions, then rank 0 merges the CTAs (rank order for <C>) ----
    double ex = 0.0;
    tile_reduce<float>(tile, d.k, [&](uint32_t u) { return (r << L) | u; }, s.tk, ex);
    const double tot = block_sum(ex, s.red);
    if (threadIdx.x == 0) *s.cex = tot;
    if (d.psi_out) {              // back from the rotated frame: psi = (-i)^{|z|} psi~
        float2* pout = reinterpret_cast<float2*>(d.psi_out) + ((size_t)r << L);
        const int pr = __popc(r);
        for (uint32_t u = threadIdx.x; u < D; u += blockDim.x)
            pout[u] = times_i_pow(s.psi[swz<float>(u)], -(pr + __popc(u)));
    }
    cl.sync();
    if (r == 0) {
        constexpr int C = 1 << CB;
        if (threadIdx.x == 0 && d.expect) {
            double acc = 0.0;
            for (int j = 0; j < C; ++j) acc += *cl.map_shared_rank(s.cex, j);
            *d.expect = acc;
        }
        if (d.k > 0) {
            // gather the C lists (k entries each) into the candidate buffer, rank-select
            for (int e = threadIdx.x; e < C * d.k; e += blockDim.x)
                s.tk.cand[e] = cl.map_shared_rank(s.tk.out, e / d.k)[e % d.k];
        }
    }
    cl.sync();   // the lists of ranks != 0 have been read; rank 0 may overwrite its own
    if (r == 0 && d.k > 0) {
        constexpr int C = 1 << CB;
        rank_select(s.tk.cand, C * d.k, d.k, s.tk.out);
        __syncthreads();
        if (threadIdx.x < (unsigned)d.k) {
            const TopEnt e = s.tk.out[threadIdx.x];
            if (d.topk_idx) d.topk_idx[threadIdx.x] = (uint64_t)e.z;
            if (d.topk_prob) d.topk_prob[threadIdx.x] = e.p;
        }
    }
    cl.sync();   // the next instance reuses the shared memory
}

// Clusters walk the descriptors round-robin: cluster c takes c, c + #clusters, ...
template <int CB>
__global__ void __launch_bounds__(512) k_cluster(const InstDesc<float>* __restrict__ desc, int count,
                                                 int L) {
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = 1 << CB;
    const int ncl = gridDim.x / C;
    const int cid = blockIdx.x / C;
    for (int ii = cid; ii < count; ii += ncl) {
        const InstDesc<float> d = desc[ii];
        run_cluster_instance<CB>(cl, d, L, sm);
    }
}

template <int CB>
cudaError_t launch_cb(const void* desc, int count, int n, int L, int pmax, int clusters,
                      cudaStream_t st, int* max_clusters) {
    const int threads = cluster_threads(L);
    size_t off[11];
    const size_t sm = cluster_layout(n, L, pmax, threads, off);
    cudaError_t e = cudaFuncSetAttribute(k_cluster<CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if ((1 << CB) > 8) {
        e = cudaFuncSetAttribute(k_cluster<CB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1 << CB;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (max_clusters) {
        cfg.gridDim = dim3(1 << CB);
        int mc = 0;
        e = cudaOccupancyMaxActiveClusters(&mc, k_cluster<CB>, &cfg);
        *max_clusters = (e == cudaSuccess) ? mc : 0;
        return e;
    }
    cfg.gridDim = dim3((unsigned)(clusters << CB));
    e = cudaLaunchKernelEx(&cfg, k_cluster<CB>, static_cast<const InstDesc<float>*>(desc), count, L);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

size_t cluster_smem_bytes(int n, int L, int p) {
    size_t off[11];
    return cluster_layout(n, L, p, cluster_threads(L), off);
}

cudaError_t launch_cluster(const void* desc, int count, int n, int L, int pmax, int clusters,
                           cudaStream_t st, int* max_clusters) {
    switch (n - L) {
        case 1: return launch_cb<1>(desc, count, n, L, pmax, clusters, st, max_clusters);
        case 2: return launch_cb<2>(desc, count, n, L, pmax, clusters, st, max_clusters);
        case 3: return launch_cb<3>(desc, count, n, L, pmax, clusters, st, max_clusters);
        case 4: return launch_cb<4>(desc, count, n, L, pmax, clusters, st, max_clusters);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qaoa
