// k_resident.cu -- resident tier: one CTA per QAOA instance, the whole 2^n state (complex64
// up to n = 14, complex128 up to n = 13) and its energy vector held in shared memory for all
// p layers. One persistent launch walks a queue of instance descriptors; each CTA
//   1. builds E(z) = z^T Q z for all z by Gray-code increments (Section IV, the QUBO mapped to
//      the diagonal problem Hamiltonian),
//   2. applies the p layers of Eq. 2 (cost phase, then exp(-i beta X_q) on every qubit) from
//      |+> with the snake schedule of the tile engine,
//   3. reduces <C> = sum |psi|^2 E (FP32 per-thread partials over at most 2^R terms, FP64
//      above) and the k most probable bitstrings (the sub-solution of Section IV), fused into
//      the last sub-pass,
//   4. optionally runs the adjoint sweep for d<C>/d(gamma, beta) on the same shared tile.
#include <algorithm>

#include "qaoa_engine.cuh"
#include "qaoa_kernels.h"

namespace qaoa {

namespace {

template <typename T>
struct Smem {
    typename Num<T>::C* psi;
    typename Num<T>::C* lam;
    T* E;
    T* Q;
    LayerConst<T>* lc;
    double* red;       // 32 doubles
    double* acc;       // 2 p doubles: d gamma, d beta accumulators
    TileTopk tk;       // top-k scratch
    T* escr;           // energy-build tables
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename T>
__host__ __device__ inline size_t smem_layout(int n, int p, bool grad, int threads, size_t* off) {
    using C = typename Num<T>::C;
    const size_t D = (size_t)1 << n;
    size_t o = 0;
    off[0] = o; o = align_up(o + D * sizeof(C), 16);                       // psi
    off[1] = o; if (grad) o = align_up(o + D * sizeof(C), 16);             // lam
    off[2] = o; o = align_up(o + D * sizeof(T), 16);                       // E
    off[3] = o; o = align_up(o + (size_t)n * n * sizeof(T), 16);           // Q
    off[4] = o; o = align_up(o + (size_t)p * sizeof(LayerConst<T>), 16);   // layer consts
    off[5] = o; o = align_up(o + 32 * sizeof(double), 16);                 // reduction
    off[6] = o; o = align_up(o + 2 * (size_t)p * sizeof(double), 16);      // grad accum
    // the energy-build tables are used before the first sub-pass and the top-k scratch after
    // the last one: both live in one region
    const size_t nw = (size_t)(threads + 31) / 32;
    const size_t r0 = o;
    off[7] = o; o = align_up(o + nw * 32 * sizeof(TopEnt), 16);          // fallback lists
    off[8] = o; o = align_up(o + TOPK_CAP * sizeof(TopEnt), 16);         // candidates
    off[9] = o; o = align_up(o + 16 * sizeof(TopEnt), 16);               // tile top-k
    off[10] = o; o = align_up(o + 16 * 32 * sizeof(float) + 4 * sizeof(int), 16);  // bounds, counts
    off[11] = r0;                                                         // energy tables
    const size_t eend = align_up(r0 + tile_energy_scratch(n) * sizeof(T), 16);
    if (eend > o) o = eend;
    return o;
}

template <typename T, int R>
__device__ void forward_run(const InstDesc<T>& d, const Smem<T>& s, bool started) {
    const int n = d.n, p = d.p;
    const TileRef<T> tile{s.psi, s.lam, s.E, n};
    // started: the energy build already wrote |+> after the first cost layer
    const bool init = !(d.flags & F_INIT_PSI) && !started;
    const T amp0 = (T)exp2(-0.5 * (double)n);
    const int G = num_windows(0, n, R);
    const int S = snake_len(G, p);
    auto nofin = [](uint32_t, int, bool) {};
    for (int si = 0; si < S; ++si) {
        SubPass sp;
        snake_step(si, G, p, 0, started ? 0 : 1, 0, n, n, R, sp);
        sp.post = (si == S - 1);
        subpass_fwd<T, R>(tile, sp, s.lc, init && si == 0, amp0, 0, nofin);
        __syncthreads();
    }
    // <C> and the top-k list of the final state (the list is unique under (probability desc,
    // index asc), whatever the order of the reduction)
    double ex = 0.0;
    tile_reduce<T>(tile, d.k, [](uint32_t u) { return u; }, s.tk, ex);
    const double tot = block_sum(ex, s.red);
    if (threadIdx.x == 0 && d.expect) *d.expect = tot;
    if (threadIdx.x < (unsigned)d.k) {
        const TopEnt e = s.tk.out[threadIdx.x];
        if (d.topk_idx) d.topk_idx[threadIdx.x] = (uint64_t)e.z;
        if (d.topk_prob) d.topk_prob[threadIdx.x] = e.p;
    }
    __syncthreads();
}

template <typename T, int R>
__device__ void adjoint_run(const InstDesc<T>& d, const Smem<T>& s) {
    const int n = d.n, p = d.p;
    const TileRef<T> tile{s.psi, s.lam, s.E, n};
    const int G = num_windows(0, n, R);
    const int S = snake_len(G, p);
    for (int l = threadIdx.x; l < 2 * p; l += blockDim.x) s.acc[l] = 0.0;
    __syncthreads();
    for (int si = S - 1; si >= 0; --si) {
        SubPass sp;
        snake_step(si, G, p, 0, 1, 0, n, n, R, sp);
        T ab[2] = {T(0), T(0)}, ag[2] = {T(0), T(0)};
        subpass_adj<T, R>(tile, sp, s.lc, si == S - 1, ab, ag);
        __syncthreads();
        for (int j = 0; j <= sp.lb - sp.la; ++j) {
            const int l = sp.lb - j;
            const double sb = block_sum((double)ab[j], s.red);
            const double sg = block_sum((double)ag[j], s.red);
            if (threadIdx.x == 0) {
                s.acc[p + l] += sb;
                if (l > sp.la || sp.ph_first) s.acc[l] += sg;
            }
        }
        __syncthreads();
    }
    for (int l = threadIdx.x; l < p; l += blockDim.x) {
        if (d.dgamma) d.dgamma[l] = 2.0 * s.acc[l];
        if (d.dbeta) d.dbeta[l] = 2.0 * s.acc[p + l];
    }
    __syncthreads();
}

// Forward register window of an n-qubit instance: rb, narrowed to rmax when asked unless a
// window would then start above bit 9 (the engine's window starts are 0..9), at most n.
__host__ __device__ inline int resident_window(int n, int rb, int rmax) {
    const int r = (rmax < rb && n - rmax <= 9) ? rmax : rb;
    return n < r ? n : r;
}

template <typename T, int R, int RA>
__device__ void run_instance(const InstDesc<T>& d, unsigned char* sm) {
    using C = typename Num<T>::C;
    const int n = d.n, p = d.p;
    const bool grad = (d.flags & F_GRAD) != 0;
    size_t off[12];
    smem_layout<T>(n, p, grad, blockDim.x, off);
    Smem<T> s;
    s.psi = reinterpret_cast<C*>(sm + off[0]);
    s.lam = reinterpret_cast<C*>(sm + off[1]);
    s.E = reinterpret_cast<T*>(sm + off[2]);
    s.Q = reinterpret_cast<T*>(sm + off[3]);
    s.lc = reinterpret_cast<LayerConst<T>*>(sm + off[4]);
    s.red = reinterpret_cast<double*>(sm + off[5]);
    s.acc = reinterpret_cast<double*>(sm + off[6]);
    s.tk.wlists = reinterpret_cast<TopEnt*>(sm + off[7]);
    s.tk.cand = reinterpret_cast<TopEnt*>(sm + off[8]);
    s.tk.out = reinterpret_cast<TopEnt*>(sm + off[9]);
    s.tk.wb = reinterpret_cast<float*>(sm + off[10]);
    s.tk.cnt = reinterpret_cast<int*>(sm + off[10] + 16 * 32 * sizeof(float));
    s.escr = reinterpret_cast<T*>(sm + off[11]);
    const uint32_t D = 1u << n;

    set_layer_consts<T>(s.lc, d.gamma, d.beta, p, n, true);
    bool started = false;
    if (d.Q) {
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) s.Q[i] = d.Q[i];
        __syncthreads();
        FusedInit<T> fi{nullptr, T(0), T(0), 0};
        if (!(d.flags & F_INIT_PSI)) {
            fi.psi = s.psi;
            fi.amp0 = (T)exp2(-0.5 * (double)n);
            fi.gpi0 = d.gamma[0] / T(3.14159265358979323846);
        }
        started = build_tile_energy_any<T>(n, n, 0u, s.Q, s.E, s.escr, fi);
    } else {
        for (uint32_t z = threadIdx.x; z < D; z += blockDim.x) s.E[swz<T>(z)] = d.E_in[z];
    }
    if (d.flags & F_INIT_PSI) {   // into the rotated frame: psi~ = i^{|z|} psi
        const C* pin = reinterpret_cast<const C*>(d.psi_in);
        for (uint32_t z = threadIdx.x; z < D; z += blockDim.x)
            s.psi[swz<T>(z)] = times_i_pow(pin[z], __popc(z));
    }
    __syncthreads();
    if (d.E_out)
        for (uint32_t z = threadIdx.x; z < D; z += blockDim.x) d.E_out[z] = s.E[swz<T>(z)];

    forward_run<T, R>(d, s, started);

    if (d.psi_out) {              // back from the rotated frame: psi = (-i)^{|z|} psi~
        C* pout = reinterpret_cast<C*>(d.psi_out);
        for (uint32_t z = threadIdx.x; z < D; z += blockDim.x)
            pout[z] = times_i_pow(s.psi[swz<T>(z)], -__popc(z));
    }
    if (grad) adjoint_run<T, RA>(d, s);
}

template <typename T>
__device__ void dispatch_instance(const InstDesc<T>& d, unsigned char* sm, int rmax) {
    constexpr int RBF = Num<T>::RB, RBA = Num<T>::RB_ADJ;
    // register windows: RB (forward, or rmax when the launch asks for narrower windows that keep
    // every window start within the engine's 0..9) and RB_ADJ (adjoint) qubits, fewer when n is
    // smaller
    const int rf = resident_window(d.n, RBF, rmax), ra = min(d.n, RBA);
    if (rf == RBF && ra == RBA) run_instance<T, RBF, RBA>(d, sm);
    else if (rf == 4 && ra == 4) run_instance<T, 4, 4>(d, sm);
    else if (rf == 3) run_instance<T, 3, 3>(d, sm);
    else if (rf == 2) run_instance<T, 2, 2>(d, sm);
    else run_instance<T, 1, 1>(d, sm);
}

// Persistent walk over `count` descriptors (queue: device counter zeroed before the launch);
// with desc == nullptr the single instance `one` (passed by value) is run by block 0.
template <typename T>
__global__ void __launch_bounds__(512) k_resident(const InstDesc<T>* __restrict__ desc, int count,
                                                  int* queue, const InstDesc<T> one, int rmax) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_next;
    if (desc == nullptr) {
        if (blockIdx.x == 0) dispatch_instance<T>(one, sm, rmax);
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int ii = s_next;
        __syncthreads();
        if (ii >= count) break;
        const InstDesc<T> d = desc[ii];
        dispatch_instance<T>(d, sm, rmax);
        __syncthreads();
    }
}

}  // namespace

int resident_threads(bool dbl, int n, int rmax) {
    const int R = resident_window(n, dbl ? Num<double>::RB : Num<float>::RB, rmax);
    const int g = (n > R) ? (1 << (n - R)) : 1;
    return g < 32 ? 32 : (g > 512 ? 512 : g);
}

size_t resident_smem_bytes(bool dbl, int n, int p, bool grad, int rmax) {
    size_t off[12];
    const int th = resident_threads(dbl, n, rmax);
    return dbl ? smem_layout<double>(n, p, grad, th, off) : smem_layout<float>(n, p, grad, th, off);
}

int resident_max_blocks_per_sm(bool dbl, int n, int pmax, bool grad, int rmax) {
    int nb = 0;
    const int th = resident_threads(dbl, n, rmax);
    const size_t sm = resident_smem_bytes(dbl, n, pmax, grad, rmax);
    // the occupancy query counts a block that needs more than 48 KB of dynamic shared memory only
    // once the kernel may use that much, so the limit is raised first (the launch sets it again)
    if (dbl) {
        if (cudaFuncSetAttribute(k_resident<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_resident<double>, th, sm) != cudaSuccess)
            nb = 0;
    } else {
        if (cudaFuncSetAttribute(k_resident<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_resident<float>, th, sm) != cudaSuccess)
            nb = 0;
    }
    return nb;
}

cudaError_t launch_resident(bool dbl, const void* desc, int count, int n, int pmax, bool grad,
                            int* queue, int grid, cudaStream_t st, const void* one, int rmax) {
    const int th = resident_threads(dbl, n, rmax);
    const size_t sm = resident_smem_bytes(dbl, n, pmax, grad, rmax);
    cudaError_t e;
    if (dbl) {
        e = cudaFuncSetAttribute(k_resident<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        InstDesc<double> o{};
        if (one) o = *static_cast<const InstDesc<double>*>(one);
        k_resident<double><<<grid, th, sm, st>>>(static_cast<const InstDesc<double>*>(desc), count, queue, o, rmax);
    } else {
        e = cudaFuncSetAttribute(k_resident<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        InstDesc<float> o{};
        if (one) o = *static_cast<const InstDesc<float>*>(one);
        k_resident<float><<<grid, th, sm, st>>>(static_cast<const InstDesc<float>*>(desc), count, queue, o, rmax);
    }
    return cudaGetLastError();
}

}  // namespace qaoa
