// k_cstream.cu -- cluster-streaming tier: complex64 forward runs of 15 <= n <= 17 qubits
// (Section IV, Eq. 2: energies, p layers of cost phase and mixer, <C> and the top-k bitstrings),
// one thread-block cluster per instance, the state streamed through L2 in tiles of 2^13
// amplitudes.
//
// A state of 2^n amplitudes (0.25-1 MiB) does not fit one SM, and the SM-to-SM network is slow
// on GB300 (about 30 GB/s per SM for remote shared-memory reads and writes, against about
// 120 GB/s per SM from L2), so the tier keeps the state in global memory and moves tiles
// between L2 and shared memory, like the streaming tier. What differs is the order: the C CTAs
// of one cluster run every pass of ONE instance, separated by cluster barriers, before taking
// the next instance. With about 40 clusters in flight the working set (state and energies of
// the instances in flight, 0.75-1.5 MiB each) stays far below the 126 MB L2, so the passes
// read and write L2, not HBM, and the whole batch is one launch.
//
// Passes (2^H tiles each, H = n - 13; CTA rank r takes tiles r, r + C, ...):
//   kind A: tile bits 0..12 are qubits 0..12 (2^13 contiguous amplitudes);
//   kind B: 2^c contiguous amplitudes (c = 13 - H) times the 2^H values of qubits 13..n-1.
// Pass 0 (A) builds the tile's energies from Q, starts |+>, applies the first cost phase and
// mixes qubits 0..12 of layer 0; pass j (0 < j < p) mixes the qubits of its kind for layer j-1,
// applies the cost phase of layer j and mixes them again for layer j; pass p finishes layer p-1
// and reduces <C> (FP64 across tiles) and the top-k list. Kinds alternate A, B, A, ...
//
// Tiles move by TMA (cp.async.bulk.tensor) with completion on an mbarrier: the state with the
// 128-byte swizzle (16-byte chunk index XOR 128-byte line index), the energies unswizzled. The
// register windows of a kind-A tile are bits [0,4) (16-byte pair accesses), [4,8) and [8,13);
// with the lanes of a warp on tile bits outside the window every shared access is free of bank
// conflicts under that swizzle, and the cost phase runs in the [8,13) window, where the lanes
// cover bits 0..4 and read the unswizzled energies conflict-free. A kind-B tile has one window
// (its H high bits). Between passes the writer waits for its bulk stores, fences the async
// proxy and arrives on the cluster barrier (release); the readers wait (acquire) and fence
// before their next TMA loads. Every mbarrier wait is bounded; a wait that runs out sets bit 0
// of the launch's status word and the kernel runs on to its end without further waits.
#include <cooperative_groups.h>
#include <cuda.h>

#include "qaoa_cstream.h"
#include "qaoa_engine.cuh"
#include "qaoa_kernels.h"

namespace cg = cooperative_groups;

namespace qaoa {

namespace {

constexpr int TB = CS_TILE_BITS;
constexpr uint32_t TD = 1u << TB;
constexpr int NT = 256;

// Shared-memory index of tile index u in a TMA tile with the 128-byte swizzle (buffer aligned to
// 1024 bytes): amplitude u sits at byte 8u, whose bits 4..6 are XORed with bits 7..9.
__device__ __forceinline__ uint32_t psw(uint32_t u) { return u ^ ((u >> 3) & 14u); }

struct TmaLayout {
    __device__ __forceinline__ static uint32_t p(uint32_t u) { return psw(u); }
    __device__ __forceinline__ static uint32_t e(uint32_t u) { return u; }
};

// ---- TMA, mbarrier and proxy-fence primitives ------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of the barrier for at most about 2^32 SM cycles (about two seconds).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 32)) return false;
    return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        ::"r"(saddr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n"
        ::"r"(saddr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n"
                 ::"l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(saddr(src))
                 : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                             int c3) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n"
                 ::"l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// the shared-memory sources of every committed bulk store have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// every committed bulk store has completed (its writes are visible to this thread)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the async proxy (before a TMA store)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// order global accesses of the generic and the async proxy (around the cluster hand-off)
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }

// ---- shared-memory layout ------------------------------------------------------------------
struct CsOff {
    size_t psi, E, Q, lc, red, wb, cnt, cand, out, wlists, lists, cex, mbar, total;
};
__host__ __device__ inline size_t cs_al(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline CsOff cs_offsets(int tpc) {
    CsOff o{};
    size_t x = 0;
    o.psi = x; x += (size_t)TD * 8;                        // 64 KiB, 1024-byte aligned at run time
    o.E = x; x += (size_t)TD * 4;                          // 32 KiB
    o.Q = x; x = cs_al(x + (size_t)CS_NMAX * CS_NMAX * 4);
    o.lc = x; x = cs_al(x + 64 * sizeof(LayerConst<float>));
    o.red = x; x = cs_al(x + 32 * sizeof(double));
    o.wb = x; x = cs_al(x + 16 * (NT / 32) * sizeof(float));
    o.cnt = x; x = cs_al(x + 4 * sizeof(int));
    o.cand = x; x = cs_al(x + TOPK_CAP * sizeof(TopEnt));
    o.out = x; x = cs_al(x + 16 * sizeof(TopEnt));
    o.wlists = x; x = cs_al(x + (NT / 32) * 32 * sizeof(TopEnt));
    o.lists = x; x = cs_al(x + (size_t)tpc * 16 * sizeof(TopEnt));
    o.cex = x; x = cs_al(x + sizeof(double));
    o.mbar = x; x = cs_al(x + sizeof(uint64_t));
    o.total = x + 1024;                                    // room to align psi to 1024 bytes
    return o;
}

// ---- register windows of a kind-A tile -------------------------------------------------------
// W2: bits [8, 13). Thread t owns u = t | (i << 8), i < 32: psw(u) = psw(t) + (i << 8) and the
// energy of u is at t + (i << 8).
__device__ __forceinline__ void w2_load(const float2* sp, float2 (&v)[32]) {
    const uint32_t b = psw(threadIdx.x);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = sp[b + (i << 8)];
}
__device__ __forceinline__ void w2_store(float2* sp, const float2 (&v)[32]) {
    const uint32_t b = psw(threadIdx.x);
#pragma unroll
    for (int i = 0; i < 32; ++i) sp[b + (i << 8)] = v[i];
}
template <int R>
__device__ __forceinline__ void phase_group(float2 (&v)[1 << R], const float* sE, uint32_t e0, int eshift,
                                            const LayerConst<float>& k) {
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) {
        float s, c;
        sincos_phase(k.gpi, sE[e0 + ((uint32_t)i << eshift)], s, c);
        rot_neg(v[i], s * k.pre, c * k.pre);
    }
}
// W1: bits [4, 8). Group g < 512 (thread t: g = t and t + 256): base = (g & 15) | (g >> 4) << 8,
// element i at (base ^ (i & 7) << 1) | (i << 4).
__device__ __forceinline__ uint32_t w1_base(uint32_t g) { return (g & 15u) | ((g >> 4) << 8); }
__device__ __forceinline__ void w1_load(const float2* sp, uint32_t b, float2 (&v)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = sp[(b ^ ((uint32_t)(i & 7) << 1)) | ((uint32_t)i << 4)];
}
__device__ __forceinline__ void w1_store(float2* sp, uint32_t b, const float2 (&v)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) sp[(b ^ ((uint32_t)(i & 7) << 1)) | ((uint32_t)i << 4)] = v[i];
}
// W0: bits [0, 4). Group g < 512: base = g << 4, x = (g & 7) << 1; the pair (2j, 2j+1) is the
// 16 bytes at base + (2j ^ x).
__device__ __forceinline__ void w0_load(const float2* sp, uint32_t g, float2 (&v)[16]) {
    const uint32_t b = g << 4, x = (g & 7u) << 1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 q = *reinterpret_cast<const float4*>(sp + (b + ((uint32_t)(2 * j) ^ x)));
        v[2 * j] = make_float2(q.x, q.y);
        v[2 * j + 1] = make_float2(q.z, q.w);
    }
}
__device__ __forceinline__ void w0_store(float2* sp, uint32_t g, const float2 (&v)[16]) {
    const uint32_t b = g << 4, x = (g & 7u) << 1;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        *reinterpret_cast<float4*>(sp + (b + ((uint32_t)(2 * j) ^ x))) =
            make_float4(v[2 * j].x, v[2 * j].y, v[2 * j + 1].x, v[2 * j + 1].y);
}

// Mix window W0 or W1 of every group with layer constants k (both groups of the thread).
template <int W>
__device__ __forceinline__ void mix_w01(float2* sp, const LayerConst<float>& k) {
#pragma unroll 1
    for (uint32_t g = threadIdx.x; g < 512u; g += NT) {
        float2 v[16];
        if (W == 0) w0_load(sp, g, v);
        else w1_load(sp, w1_base(g), v);
        mix_layer<4>(v, 15, k);
        if (W == 0) w0_store(sp, g, v);
        else w1_store(sp, w1_base(g), v);
    }
}

// ---- per-instance descriptor ---------------------------------------------------------------
struct CsInstDev {
    int n, p, k, out_psi;
    float amp0;
    const float* Q;
    const float* gamma;
    const float* beta;
    double* expect;
    uint64_t* topk_idx;
    double* topk_prob;
    const CUtensorMap* maps;   // psi kind A, psi kind B, E kind A, E kind B
};

// Energies of kind-A tile tau of pass 0 in the W2 layout (thread t owns u = t | j << 8), with
// the tile's fixed global bits S = tau << 13:
//   E(z) = [E_S + El(t)] + Eh[j] + X_t(j),  X_t(j) = sum_{b in j} W_b(t),
//   W_b(t) = sum_{i in t} (Q_{i, 8+b} + Q_{8+b, i}),
// (every pair of set bits of z counted once, Q_ij and Q_ji both). Eh is built by 32 threads in
// the scratch `eh`. ev[j] receives the energies; they are also written to sE (unswizzled).
__device__ __forceinline__ void w2_energies(int n, uint32_t zfix, const float* Qs, float* eh, float* sE,
                                            float (&ev)[32]) {
    const uint32_t t = threadIdx.x;
    if (t < 32u) {
        float acc = 0.0f;
        const uint32_t hb = t << 8;
        for (uint32_t bi = hb; bi; bi &= bi - 1u) {
            const int i = __ffs((int)bi) - 1;
            for (uint32_t bj = hb; bj; bj &= bj - 1u) acc += Qs[i * n + __ffs((int)bj) - 1];
            for (uint32_t bj = zfix; bj; bj &= bj - 1u) {
                const int j = __ffs((int)bj) - 1;
                acc += Qs[i * n + j] + Qs[j * n + i];
            }
        }
        eh[t] = acc;
    }
    float base = 0.0f;
    for (uint32_t bi = zfix; bi; bi &= bi - 1u) {
        const int i = __ffs((int)bi) - 1;
        for (uint32_t bj = zfix; bj; bj &= bj - 1u) base += Qs[i * n + __ffs((int)bj) - 1];
    }
    for (int i = 0; i < 8; ++i) {
        float si = Qs[i * n + i];
        for (uint32_t bj = zfix; bj; bj &= bj - 1u) {
            const int j = __ffs((int)bj) - 1;
            si += Qs[i * n + j] + Qs[j * n + i];
        }
        float cross = 0.0f;
        for (int j = 0; j < i; ++j)
            if ((t >> j) & 1u) cross += Qs[i * n + j] + Qs[j * n + i];
        if ((t >> i) & 1u) base += si + cross;
    }
    float X[32];
    X[0] = 0.0f;
#pragma unroll
    for (int b = 0; b < 5; ++b) {
        float w = 0.0f;
        const int q = 8 + b;
        for (int i = 0; i < 8; ++i)
            if ((t >> i) & 1u) w += Qs[i * n + q] + Qs[q * n + i];
#pragma unroll
        for (int m = 0; m < (1 << b); ++m) X[m | (1 << b)] = X[m] + w;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        ev[j] = base + (eh[j] + X[j]);
        sE[t + ((uint32_t)j << 8)] = ev[j];
    }
}

template <int H>
__global__ void __launch_bounds__(NT, 2) k_cstream(const CsInstDev* __restrict__ insts, int count,
                                                  unsigned* status) {
    constexpr int NTILE = 1 << H;                 // tiles per pass
    constexpr int C = NTILE < 8 ? NTILE : 8;      // CTAs per cluster
    constexpr int TPC = NTILE / C;                // tiles per CTA per pass
    constexpr int CB = TB - H;                    // contiguous bits of a kind-B tile
    constexpr int NB = 1 << (CB - 8);             // kind-B groups per thread
    extern __shared__ __align__(16) unsigned char sm_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t rank = cl.block_rank();
    const uint32_t raw = saddr(sm_raw);
    unsigned char* sm = sm_raw + (((raw + 1023u) & ~1023u) - raw);
    const CsOff o = cs_offsets(TPC);
    float2* sp = reinterpret_cast<float2*>(sm + o.psi);
    float* sE = reinterpret_cast<float*>(sm + o.E);
    float* sQ = reinterpret_cast<float*>(sm + o.Q);
    LayerConst<float>* lc = reinterpret_cast<LayerConst<float>*>(sm + o.lc);
    double* red = reinterpret_cast<double*>(sm + o.red);
    TileTopk ts;
    ts.wb = reinterpret_cast<float*>(sm + o.wb);
    ts.cnt = reinterpret_cast<int*>(sm + o.cnt);
    ts.cand = reinterpret_cast<TopEnt*>(sm + o.cand);
    ts.out = reinterpret_cast<TopEnt*>(sm + o.out);
    ts.wlists = reinterpret_cast<TopEnt*>(sm + o.wlists);
    TopEnt* lists = reinterpret_cast<TopEnt*>(sm + o.lists);
    double* cex = reinterpret_cast<double*>(sm + o.cex);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + o.mbar);
    if (threadIdx.x == 0) mbar_init(mbar, 1);
    __syncthreads();
    uint32_t parity = 0;
    bool ok = true;
    const int ncl = (int)(gridDim.x / C), cid = (int)(blockIdx.x / C);
    const TileRef<float> tile{sp, nullptr, sE, TB};
    for (int ii = cid; ii < count; ii += ncl) {
        const CsInstDev I = insts[ii];
        const int n = I.n, p = I.p;
        for (int i = threadIdx.x; i < n * n; i += NT) sQ[i] = I.Q[i];
        set_layer_consts<float>(lc, I.gamma, I.beta, p, n, true);   // ends with a barrier
        double my_ex = 0.0;
        for (int pass = 0; pass <= p; ++pass) {
            const bool kindA = (pass & 1) == 0;
            const bool fin = pass == p;
            for (int j = 0; j < TPC; ++j) {
                const uint32_t tau = rank + (uint32_t)(j * C);
                // the bulk stores of the previous tile must have read the buffers before they are
                // refilled (by TMA in passes > 0, by the threads in pass 0)
                if (threadIdx.x == 0) bulk_wait_read();
                if (pass == 0 && j > 0) __syncthreads();
                if (pass > 0) {
                    if (threadIdx.x == 0) {
                        if (ok) {
                            mbar_expect_tx(mbar, TD * 8 + TD * 4);
                            if (kindA) {
                                tma_load_4d(sp, &I.maps[0], 0, 0, 0, (int)tau, mbar);
                                tma_load_3d(sE, &I.maps[2], 0, 0, (int)tau, mbar);
                            } else {
                                tma_load_4d(sp, &I.maps[1], 0, 0, (int)tau, 0, mbar);
                                tma_load_4d(sE, &I.maps[3], 0, 0, (int)tau, 0, mbar);
                            }
                        }
                    }
                    if (ok) ok = mbar_wait_bounded(mbar, parity);
                    ok = __syncthreads_and(ok);
                    parity ^= 1u;
                }
                if (kindA) {
                    if (pass == 0) {
                        // energies, |+>, the first cost phase and layer 0 on window [8, 13)
                        float ev[32];
                        w2_energies(n, tau << TB, sQ, reinterpret_cast<float*>(ts.wlists), sE, ev);
                        const uint32_t t = threadIdx.x;
                        const int pc = __popc(tau) + __popc(t);
                        float2 v[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            float s, c;
                            sincos_phase(lc[0].gpi, ev[i], s, c);
                            float2 a = make_float2(I.amp0 * c, -I.amp0 * s);
                            v[i] = times_i_pow(a, pc + __popc(i));
                        }
                        mix_layer<5>(v, 31, lc[0]);
                        w2_store(sp, v);
                        __syncthreads();
                        mix_w01<1>(sp, lc[0]);
                        __syncthreads();
                        mix_w01<0>(sp, lc[0]);
                    } else {
                        mix_w01<0>(sp, lc[pass - 1]);
                        __syncthreads();
                        mix_w01<1>(sp, lc[pass - 1]);
                        __syncthreads();
                        float2 v[32];
                        w2_load(sp, v);
                        mix_layer<5>(v, 31, lc[pass - 1]);
                        if (!fin) {
                            phase_group<5>(v, sE, threadIdx.x, 8, lc[pass]);
                            mix_layer<5>(v, 31, lc[pass]);
                        } else if (lc[p - 1].shear) {
                            scale_group<5>(v, lc[p - 1].post);
                        }
                        w2_store(sp, v);
                        if (!fin) {
                            __syncthreads();
                            mix_w01<1>(sp, lc[pass]);
                            __syncthreads();
                            mix_w01<0>(sp, lc[pass]);
                        }
                    }
                } else {
#pragma unroll 1
                    for (int r = 0; r < NB; ++r) {
                        const uint32_t lo = threadIdx.x + (uint32_t)(r * NT);
                        const uint32_t b = psw(lo);
                        float2 v[1 << H];
#pragma unroll
                        for (int i = 0; i < (1 << H); ++i) v[i] = sp[b + ((uint32_t)i << CB)];
                        mix_layer<H>(v, (1 << H) - 1, lc[pass - 1]);
                        if (!fin) {
                            phase_group<H>(v, sE, lo, CB, lc[pass]);
                            mix_layer<H>(v, (1 << H) - 1, lc[pass]);
                        } else if (lc[p - 1].shear) {
                            scale_group<H>(v, lc[p - 1].post);
                        }
#pragma unroll
                        for (int i = 0; i < (1 << H); ++i) sp[b + ((uint32_t)i << CB)] = v[i];
                    }
                }
                __syncthreads();
                if (!fin) {
                    fence_async_smem();
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        if (kindA) tma_store_4d(&I.maps[0], sp, 0, 0, 0, (int)tau);
                        else tma_store_4d(&I.maps[1], sp, 0, 0, (int)tau, 0);
                        if (pass == 0) tma_store_3d(&I.maps[2], sE, 0, 0, (int)tau);
                        bulk_commit();
                    }
                } else {
                    // <C> partial and top-k list of the tile; the state leaves in the standard frame
                    const uint32_t cmask = (1u << CB) - 1u;
                    const auto zmap = [kindA, tau, cmask](uint32_t u) -> uint32_t {
                        return kindA ? (u | (tau << TB)) : ((u & cmask) | (tau << CB) | ((u >> CB) << TB));
                    };
                    double ex = 0.0;
                    tile_reduce<float, TmaLayout>(tile, I.k, zmap, ts, ex);
                    const double tot = block_sum(ex, red);
                    if (threadIdx.x == 0) my_ex += tot;
                    if (threadIdx.x < (unsigned)I.k) lists[j * I.k + threadIdx.x] = ts.out[threadIdx.x];
                    if (I.out_psi) {
                        __syncthreads();
                        for (uint32_t u = threadIdx.x; u < TD; u += NT)
                            sp[psw(u)] = times_i_pow(sp[psw(u)], -__popc(zmap(u)));
                        fence_async_smem();
                        __syncthreads();
                        if (threadIdx.x == 0) {
                            if (kindA) tma_store_4d(&I.maps[0], sp, 0, 0, 0, (int)tau);
                            else tma_store_4d(&I.maps[1], sp, 0, 0, (int)tau, 0);
                            bulk_commit();
                        }
                    }
                    __syncthreads();
                }
            }
            // pass boundary: this CTA's stores are complete and visible, then the cluster barrier
            if (threadIdx.x == 0) {
                bulk_wait_all();
                fence_async_global();
            }
            if (fin && threadIdx.x == 0) *cex = my_ex;
            cl.sync();
            if (threadIdx.x == 0) fence_async_global();
        }
        // rank 0 merges the CTAs' <C> partials (rank order) and top-k lists
        if (rank == 0) {
            if (threadIdx.x == 0 && I.expect) {
                double acc = 0.0;
                for (int r = 0; r < C; ++r) acc += *cl.map_shared_rank(cex, r);
                *I.expect = acc;
            }
            if (I.k > 0) {
                const int per = TPC * I.k;
                for (int e = threadIdx.x; e < C * per; e += NT)
                    ts.cand[e] = cl.map_shared_rank(lists, e / per)[e % per];
            }
        }
        cl.sync();   // the lists of every rank have been read
        if (rank == 0 && I.k > 0) {
            rank_select(ts.cand, C * TPC * I.k, I.k, ts.out);
            __syncthreads();
            if (threadIdx.x < (unsigned)I.k) {
                const TopEnt e = ts.out[threadIdx.x];
                if (I.topk_idx) I.topk_idx[threadIdx.x] = (uint64_t)e.z;
                if (I.topk_prob) I.topk_prob[threadIdx.x] = e.p;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bulk_wait_all();
        if (!ok) atomicOr(status, 1u);
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

template <int H>
cudaError_t cs_launch_h(const void* insts, int count, int clusters, cudaStream_t st, int* max_clusters,
                        unsigned* status) {
    constexpr int NTILE = 1 << H;
    constexpr int C = NTILE < 8 ? NTILE : 8;
    const size_t smem = cs_offsets(NTILE / C).total;
    cudaError_t e = cudaFuncSetAttribute(k_cstream<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (max_clusters) {
        cfg.gridDim = dim3(C);
        int mc = 0;
        e = cudaOccupancyMaxActiveClusters(&mc, k_cstream<H>, &cfg);
        *max_clusters = (e == cudaSuccess) ? mc : 0;
        return e;
    }
    cfg.gridDim = dim3((unsigned)(clusters * C));
    e = cudaLaunchKernelEx(&cfg, k_cstream<H>, static_cast<const CsInstDev*>(insts), count, status);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against the driver).
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encode_fn() {
    static EncodeFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeFn) nullptr;
        return reinterpret_cast<EncodeFn>(f);
    }();
    return fn;
}

bool encode(CUtensorMap* m, void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
            const cuuint32_t* box, bool swz128) {
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, base, dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE,
                       swz128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t cstream_inst_bytes() { return sizeof(CsInstDev); }

bool cstream_available() { return encode_fn() != nullptr; }

cudaError_t cstream_max_clusters(int n, int* out) {
    *out = 0;
    switch (n - TB) {
        case 2: return cs_launch_h<2>(nullptr, 0, 0, nullptr, out, nullptr);
        case 3: return cs_launch_h<3>(nullptr, 0, 0, nullptr, out, nullptr);
        case 4: return cs_launch_h<4>(nullptr, 0, 0, nullptr, out, nullptr);
        default: return cudaErrorInvalidValue;
    }
}

int cstream_cluster_size(int n) { return (1 << (n - TB)) < 8 ? (1 << (n - TB)) : 8; }

// The four tensor maps of one instance: state and energies (2^n values each, 16-byte aligned)
// as kind-A and kind-B tiles. Returns false if the driver refuses one of them.
bool cstream_encode_maps(int n, void* psi, void* E, void* maps_out) {
    if (!encode_fn() || n < CS_NMIN || n > CS_NMAX) return false;
    CUtensorMap* m = static_cast<CUtensorMap*>(maps_out);
    const int H = n - TB, c = TB - H;
    const cuuint64_t NH = 1ull << H;
    {   // psi, kind A: (32 floats = 16 amplitudes, 256 lines, 2 planes, tile)
        const cuuint64_t d[4] = {32, 256, 2, NH};
        const cuuint64_t s[3] = {128, 32768, 65536};
        const cuuint32_t b[4] = {32, 256, 2, 1};
        if (!encode(&m[0], psi, 4, d, s, b, true)) return false;
    }
    {   // psi, kind B: (32 floats, 2^(c-4) lines, tile = bits c..12, bits 13..n-1)
        const cuuint64_t d[4] = {32, 1ull << (c - 4), NH, NH};
        const cuuint64_t s[3] = {128, (1ull << c) * 8, (1ull << TB) * 8};
        const cuuint32_t b[4] = {32, 1u << (c - 4), 1, (cuuint32_t)NH};
        if (!encode(&m[1], psi, 4, d, s, b, true)) return false;
    }
    {   // E, kind A: (256 floats, 32 lines, tile)
        const cuuint64_t d[3] = {256, 32, NH};
        const cuuint64_t s[2] = {1024, 32768};
        const cuuint32_t b[3] = {256, 32, 1};
        if (!encode(&m[2], E, 3, d, s, b, false)) return false;
    }
    {   // E, kind B: (256 floats, 2^(c-8) lines, tile = bits c..12, bits 13..n-1)
        const cuuint64_t d[4] = {256, 1ull << (c - 8), NH, NH};
        const cuuint64_t s[3] = {1024, (1ull << c) * 4, (1ull << TB) * 4};
        const cuuint32_t b[4] = {256, 1u << (c - 8), 1, (cuuint32_t)NH};
        if (!encode(&m[3], E, 4, d, s, b, false)) return false;
    }
    return true;
}

void cstream_fill_inst(void* out, int n, int p, int k, bool out_psi, const float* Q, const float* gamma,
                       const float* beta, double* expect, uint64_t* topk_idx, double* topk_prob,
                       const void* maps_dev) {
    CsInstDev d{};
    d.n = n;
    d.p = p;
    d.k = k;
    d.out_psi = out_psi ? 1 : 0;
    d.amp0 = (float)exp2(-0.5 * n);
    d.Q = Q;
    d.gamma = gamma;
    d.beta = beta;
    d.expect = expect;
    d.topk_idx = topk_idx;
    d.topk_prob = topk_prob;
    d.maps = static_cast<const CUtensorMap*>(maps_dev);
    *static_cast<CsInstDev*>(out) = d;
}

cudaError_t launch_cstream(int n, const void* insts, int count, int clusters, unsigned* status, cudaStream_t st) {
    switch (n - TB) {
        case 2: return cs_launch_h<2>(insts, count, clusters, st, nullptr, status);
        case 3: return cs_launch_h<3>(insts, count, clusters, st, nullptr, status);
        case 4: return cs_launch_h<4>(insts, count, clusters, st, nullptr, status);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace qaoa
