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
#include "qaoa_engine.cuh"
#include "qaoa_kernels.h"

namespace qaoa {

namespace {

constexpr int MAXH = 8;   // high bits walked by the Gray code per thread

// E(z) = z^T Q z for all z of an n-bit tile. Thread t (blockDim a power of two, 2^m threads
// used) fixes the low m bits to t, evaluates E directly there, then walks the remaining
// n - m bits in Gray-code order: flipping bit b with direction d = +1 (0 -> 1) or -1 changes
// E by d (Q_bb + 2 F_b) with F_b = sum_{j != b} Q_bj z_j, and F of every other walked bit
// changes by d Q_{hb}. At most 2^MAXH steps per thread, so the FP32 drift stays small.
template <typename T>
__device__ void build_energy(int n, const T* Qs, T* E) {
    int m = 31 - __clz((int)blockDim.x);
    if (m > n) m = n;
    const int nh = n - m;
    const uint32_t t = threadIdx.x;
    if (t >= (1u << m)) return;
    T e = T(0);
    for (uint32_t bi = t; bi; bi &= bi - 1u) {          // set bits i of t
        const T* row = Qs + (__ffs((int)bi) - 1) * n;
        for (uint32_t bj = t; bj; bj &= bj - 1u) e += row[__ffs((int)bj) - 1];
    }
    T F[MAXH];
#pragma unroll
    for (int h = 0; h < MAXH; ++h) {
        T f = T(0);
        if (h < nh)
            for (uint32_t bj = t; bj; bj &= bj - 1u) f += Qs[(m + h) * n + (__ffs((int)bj) - 1)];
        F[h] = f;
    }
    uint32_t z = t;
    E[swz<T>(z)] = e;
    const uint32_t steps = 1u << nh;
    for (uint32_t k = 1; k < steps; ++k) {
        const int b = __ffs((int)k) - 1;
        const int hb = m + b;
        const T d = ((z >> hb) & 1u) ? T(-1) : T(1);
        T fb = T(0);
#pragma unroll
        for (int h = 0; h < MAXH; ++h)
            if (h == b) fb = F[h];
        e += d * (Qs[hb * n + hb] + T(2) * fb);
        z ^= 1u << hb;
#pragma unroll
        for (int h = 0; h < MAXH; ++h)
            if (h < nh && h != b) F[h] += d * Qs[(m + h) * n + hb];
        E[swz<T>(z)] = e;
    }
}

template <typename T>
struct Smem {
    typename Num<T>::C* psi;
    typename Num<T>::C* lam;
    T* E;
    T* Q;
    LayerConst<T>* lc;
    double* red;       // 32 doubles
    double* acc;       // 2 p doubles: d gamma, d beta accumulators
    TopEnt* top;       // (blockDim/32) * 32 entries
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
    off[7] = o; o = align_up(o + (size_t)(threads / 32) * 32 * sizeof(TopEnt), 16);  // top-k
    return o;
}

template <typename T, int R>
__device__ void forward_run(const InstDesc<T>& d, const Smem<T>& s) {
    const int n = d.n, p = d.p;
    const TileRef<T> tile{s.psi, s.lam, s.E, n};
    const bool init = !(d.flags & F_INIT_PSI);
    const T amp0 = (T)exp2(-0.5 * (double)n);
    const int G = num_windows(0, n, R);
    const int S = snake_len(G, p);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpTopK top;
    top.init(d.k > 0 ? d.k : 1);
    double ex = 0.0;
    for (int si = 0; si < S; ++si) {
        SubPass sp;
        snake_step(si, G, p, 0, 1, 0, n, n, R, sp);
        const bool last = (si == S - 1);
        auto fin = [&](uint32_t base, int a, bool valid) {
            if (last) reduce_group<T, R>(tile, base, a, valid, d.k, top, ex, [](uint32_t u) { return u; });
        };
        subpass_fwd<T, R>(tile, sp, s.lc, init && si == 0, amp0, 0, fin);
        __syncthreads();
    }
    // <C>
    const double tot = block_sum(ex, s.red);
    if (threadIdx.x == 0 && d.expect) *d.expect = tot;
    // top-k: per-warp lists -> shared -> warp 0 merges (order of equal keys is irrelevant:
    // the final list is unique under (probability desc, index asc))
    if (d.k > 0) {
        if (lane < d.k) s.top[warp * 32 + lane] = TopEnt{top.p, top.z};
        __syncthreads();
        if (warp == 0) {
            WarpTopK fin;
            fin.init(d.k);
            const int nw = blockDim.x >> 5;
            for (int w = 0; w < nw; ++w) {
                const bool ok = lane < d.k;
                const TopEnt e = ok ? s.top[w * 32 + lane] : TopEnt{-1.0, 0xffffffffu};
                fin.offer_exact(e.p, e.z, ok);
            }
            if (lane < d.k) {
                if (d.topk_idx) d.topk_idx[lane] = (uint64_t)fin.z;
                if (d.topk_prob) d.topk_prob[lane] = fin.p;
            }
        }
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

template <typename T, int R, int RA>
__device__ void run_instance(const InstDesc<T>& d, unsigned char* sm) {
    using C = typename Num<T>::C;
    const int n = d.n, p = d.p;
    const bool grad = (d.flags & F_GRAD) != 0;
    size_t off[8];
    smem_layout<T>(n, p, grad, blockDim.x, off);
    Smem<T> s;
    s.psi = reinterpret_cast<C*>(sm + off[0]);
    s.lam = reinterpret_cast<C*>(sm + off[1]);
    s.E = reinterpret_cast<T*>(sm + off[2]);
    s.Q = reinterpret_cast<T*>(sm + off[3]);
    s.lc = reinterpret_cast<LayerConst<T>*>(sm + off[4]);
    s.red = reinterpret_cast<double*>(sm + off[5]);
    s.acc = reinterpret_cast<double*>(sm + off[6]);
    s.top = reinterpret_cast<TopEnt*>(sm + off[7]);
    const uint32_t D = 1u << n;

    for (int l = threadIdx.x; l < p; l += blockDim.x) {
        const T g = d.gamma[l], b = d.beta[l];
        T sb, cb;
        sincos_full(b, sb, cb);
        s.lc[l] = LayerConst<T>{g / T(3.14159265358979323846), cb, sb};
    }
    if (d.Q) {
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) s.Q[i] = d.Q[i];
        __syncthreads();
        build_energy<T>(n, s.Q, s.E);
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

    forward_run<T, R>(d, s);

    if (d.psi_out) {              // back from the rotated frame: psi = (-i)^{|z|} psi~
        C* pout = reinterpret_cast<C*>(d.psi_out);
        for (uint32_t z = threadIdx.x; z < D; z += blockDim.x)
            pout[z] = times_i_pow(s.psi[swz<T>(z)], -__popc(z));
    }
    if (grad) adjoint_run<T, RA>(d, s);
}

template <typename T>
__device__ void dispatch_instance(const InstDesc<T>& d, unsigned char* sm) {
    constexpr int RBF = Num<T>::RB, RBA = Num<T>::RB_ADJ;
    // register windows: RB (forward) and RB_ADJ (adjoint) qubits, fewer when n is smaller
    const int rf = min(d.n, RBF), ra = min(d.n, RBA);
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
                                                  int* queue, const InstDesc<T> one) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_next;
    if (desc == nullptr) {
        if (blockIdx.x == 0) dispatch_instance<T>(one, sm);
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int ii = s_next;
        __syncthreads();
        if (ii >= count) break;
        const InstDesc<T> d = desc[ii];
        dispatch_instance<T>(d, sm);
        __syncthreads();
    }
}

}  // namespace

int resident_threads(bool dbl, int n) {
    const int R = dbl ? Num<double>::RB : Num<float>::RB;
    const int g = (n > R) ? (1 << (n - R)) : 1;
    return g < 32 ? 32 : (g > 512 ? 512 : g);
}

size_t resident_smem_bytes(bool dbl, int n, int p, bool grad) {
    size_t off[8];
    const int th = resident_threads(dbl, n);
    return dbl ? smem_layout<double>(n, p, grad, th, off) : smem_layout<float>(n, p, grad, th, off);
}

int resident_max_blocks_per_sm(bool dbl, int n, int pmax, bool grad) {
    int nb = 0;
    const int th = resident_threads(dbl, n);
    const size_t sm = resident_smem_bytes(dbl, n, pmax, grad);
    if (dbl) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_resident<double>, th, sm);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_resident<float>, th, sm);
    return nb;
}

cudaError_t launch_resident(bool dbl, const void* desc, int count, int n, int pmax, bool grad,
                            int* queue, int grid, cudaStream_t st, const void* one) {
    const int th = resident_threads(dbl, n);
    const size_t sm = resident_smem_bytes(dbl, n, pmax, grad);
    cudaError_t e;
    if (dbl) {
        e = cudaFuncSetAttribute(k_resident<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        InstDesc<double> o{};
        if (one) o = *static_cast<const InstDesc<double>*>(one);
        k_resident<double><<<grid, th, sm, st>>>(static_cast<const InstDesc<double>*>(desc), count, queue, o);
    } else {
        e = cudaFuncSetAttribute(k_resident<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        InstDesc<float> o{};
        if (one) o = *static_cast<const InstDesc<float>*>(one);
        k_resident<float><<<grid, th, sm, st>>>(static_cast<const InstDesc<float>*>(desc), count, queue, o);
    }
    return cudaGetLastError();
}

}  // namespace qaoa
