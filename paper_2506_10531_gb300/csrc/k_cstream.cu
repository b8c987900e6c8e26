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
// the next instance. With about 70 clusters of 4 CTAs in flight, two instances each, the working
// set (state and energies of the instances in flight, 0.75-1.5 MiB each) stays below the 126 MB
// L2, so the passes read and write L2, not HBM, and the whole batch is one launch.
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
#include "qaoa_tma.cuh"

namespace cg = cooperative_groups;

namespace qaoa {

namespace {

using namespace tma;

constexpr int TB = CS_TILE_BITS;
// CTAs per cluster for a pass of `ntile` tiles (each CTA then takes ntile / C tiles per pass).
// Measured on GB300 (batches of 128-256 instances): 4 CTAs beat 8 by 4-7% at n = 16 and 17 (twice
// the clusters in flight, half the cluster barriers per tile), except where the instance count
// falls just past a multiple of the slots in flight.
constexpr int CS_CMAX = 4;
__host__ __device__ constexpr int cs_cluster(int ntile) { return ntile < CS_CMAX ? ntile : CS_CMAX; }
constexpr uint32_t TD = 1u << TB;
constexpr int NT = 256;

// ---- shared-memory layout ------------------------------------------------------------------
// One state tile and one energy tile, shared by the two instance slots of a CTA; the energy tile
// doubles as the top-k scratch of the final pass (after the <C> partial has read it) and of the
// merge on rank 0. Per slot: Q, layer constants, the CTA's top-k lists and <C> partial.
struct CsOff {
    size_t psi, E, red, escr, wbound, Q[2], lc[2], lists[2], cex[2], desc[2], mbar, total;
    size_t wb, cnt, cand, out, wlists;   // inside the energy tile
};
__host__ __device__ inline size_t cs_al(size_t x) { return (x + 15) & ~(size_t)15; }
constexpr size_t CS_DESC_BYTES = 128;   // a slot's copy of its instance descriptor
__host__ __device__ inline CsOff cs_offsets(int tpc) {
    CsOff o{};
    size_t x = 0;
    o.psi = x; x += (size_t)TD * 8;                        // 64 KiB, 1024-byte aligned at run time
    o.E = x; x += (size_t)TD * 4;                          // 32 KiB
    o.red = x; x = cs_al(x + 32 * sizeof(double));
    o.escr = x; x = cs_al(x + 256 * sizeof(float));       // energy tables of pass 0
    o.wbound = x; x = cs_al(x + (NT / 32) * sizeof(float));
    for (int s = 0; s < 2; ++s) {
        o.Q[s] = x; x = cs_al(x + (size_t)CS_NMAX * CS_NMAX * 4);
        o.lc[s] = x; x = cs_al(x + 64 * sizeof(LayerConst<float>));
        o.lists[s] = x; x = cs_al(x + (size_t)tpc * 16 * sizeof(TopEnt));
        o.cex[s] = x; x = cs_al(x + sizeof(double));
        o.desc[s] = x; x = cs_al(x + CS_DESC_BYTES);
    }
    o.mbar = x; x = cs_al(x + sizeof(uint64_t));
    o.total = x + 1024;                                    // room to align psi to 1024 bytes
    size_t y = o.E;
    o.wb = y; y = cs_al(y + 16 * (NT / 32) * sizeof(float));
    o.cnt = y; y = cs_al(y + 4 * sizeof(int));
    o.cand = y; y = cs_al(y + TOPK_CAP * sizeof(TopEnt));
    o.out = y; y = cs_al(y + 16 * sizeof(TopEnt));
    o.wlists = y;
    return o;
}

// Rank selection of the CTAs' merged lists (probability descending, index ascending; empty
// entries rank last): like rank_select, with the comparison loop unrolled so that its shared
// loads are in flight together.
__device__ __forceinline__ void cs_rank_select(const TopEnt* cand, int count, int k, TopEnt* out) {
    for (int c = threadIdx.x; c < count; c += blockDim.x) {
        const TopEnt me = cand[c];
        if (!is_entry(me.p)) continue;
        int rank = 0;
#pragma unroll 8
        for (int j = 0; j < count; ++j) {
            const TopEnt o = cand[j];
            rank += (is_entry(o.p) && better(o.p, o.z, me.p, me.z)) ? 1 : 0;
        }
        if (rank < k) out[rank] = me;
    }
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
static_assert(sizeof(CsInstDev) <= CS_DESC_BYTES && sizeof(CsInstDev) % 8 == 0, "descriptor copy");

// Energies of kind-A tile tau of pass 0 in the W2 layout (thread t owns u = t | j << 8), with
// the tile's fixed global bits S = tau << 13. With P_ik = Q_ik + Q_ki (i < k, tile qubits),
// d_i = Q_ii + sum_{s in S} (Q_is + Q_si) and E_S = sum_{s, s' in S} Q_ss',
//   E(z) = E_S + sum_{i<8} t_i d_i + sum_{i<k<8} t_i t_k P_ik + Eh[j] + sum_{b in j} W_b(t),
//   W_b(t) = sum_{i<8} t_i P_{i,8+b},   Eh[j] = sum_{b in j} d_{8+b} + sum_{b<c in j} P_{8+b,8+c},
// every pair of set bits of z counted once with both Q_ik and Q_ki. The tables (scr: 256 floats)
// are built once per tile; each thread's sums are unrolled with 0/1 weights (independent loads,
// no serial chains). ev[j] receives the energies (the caller writes them to the energy tile).
__device__ __forceinline__ void w2_energies(int n, uint32_t zfix, const float* Qs, float* scr, float (&ev)[32]) {
    float* P = scr;           // 13 x 13, upper triangle
    float* d = scr + 169;     // 13
    float* Eh = scr + 184;    // 32
    float* es = scr + 216;    // 1
    const uint32_t t = threadIdx.x;
    if (t < 169u) {
        const int i = (int)t / 13, k = (int)t % 13;
        P[t] = (i < k) ? Qs[i * n + k] + Qs[k * n + i] : 0.0f;
    } else if (t < 182u) {
        const int i = (int)t - 169;
        float a = Qs[i * n + i];
        for (uint32_t bs = zfix; bs; bs &= bs - 1u) {
            const int sb = __ffs((int)bs) - 1;
            a += Qs[i * n + sb] + Qs[sb * n + i];
        }
        d[i] = a;
    } else if (t == 182u) {
        float a = 0.0f;
        for (uint32_t bi = zfix; bi; bi &= bi - 1u) {
            const int i = __ffs((int)bi) - 1;
            for (uint32_t bj = zfix; bj; bj &= bj - 1u) a += Qs[i * n + __ffs((int)bj) - 1];
        }
        *es = a;
    }
    __syncthreads();
    if (t < 32u) {
        float a = 0.0f, c = 0.0f;
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const float wb = (float)((t >> b) & 1u);
            a = fmaf(wb, d[8 + b], a);
#pragma unroll
            for (int e = b + 1; e < 5; ++e) c = fmaf(wb * (float)((t >> e) & 1u), P[(8 + b) * 13 + 8 + e], c);
        }
        Eh[t] = a + c;
    }
    float tb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) tb[i] = (float)((t >> i) & 1u);
    float b0 = 0.0f, b1 = 0.0f, b2 = 0.0f, b3 = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        b0 = fmaf(tb[i], d[i], b0);
        float r = 0.0f;
#pragma unroll
        for (int k = i + 1; k < 8; ++k) r = fmaf(tb[k], P[i * 13 + k], r);
        if (i & 1) b1 = fmaf(tb[i], r, b1);
        else b2 = fmaf(tb[i], r, b2);
    }
    float W[5];
#pragma unroll
    for (int bb = 0; bb < 5; ++bb) {
        float w0 = 0.0f, w1 = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            w0 = fmaf(tb[i], P[i * 13 + 8 + bb], w0);
            w1 = fmaf(tb[i + 1], P[(i + 1) * 13 + 8 + bb], w1);
        }
        W[bb] = w0 + w1;
    }
    __syncthreads();   // Eh and es ready
    const float base = *es + ((b0 + b3) + (b1 + b2));
    float X[32];
    X[0] = 0.0f;
#pragma unroll
    for (int bb = 0; bb < 5; ++bb)
#pragma unroll
        for (int m = 0; m < (1 << bb); ++m) X[m | (1 << bb)] = X[m] + W[bb];
#pragma unroll
    for (int j = 0; j < 32; ++j) ev[j] = base + (Eh[j] + X[j]);
}

template <int H>
__global__ void __launch_bounds__(NT, 2) k_cstream(const CsInstDev* __restrict__ insts, int count,
                                                  unsigned* status) {
    constexpr int NTILE = 1 << H;                 // tiles per pass
    constexpr int C = cs_cluster(NTILE);          // CTAs per cluster
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
    double* red = reinterpret_cast<double*>(sm + o.red);
    TileTopk ts;
    ts.wb = reinterpret_cast<float*>(sm + o.wb);
    ts.cnt = reinterpret_cast<int*>(sm + o.cnt);
    ts.cand = reinterpret_cast<TopEnt*>(sm + o.cand);
    ts.out = reinterpret_cast<TopEnt*>(sm + o.out);
    ts.wlists = reinterpret_cast<TopEnt*>(sm + o.wlists);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + o.mbar);
    if (threadIdx.x == 0) mbar_init(mbar, 1);
    __syncthreads();
    uint32_t parity = 0;
    bool ok = true;
    const int ncl = (int)(gridDim.x / C), cid = (int)(blockIdx.x / C);
    const TileRef<float> tile{sp, nullptr, sE, TB};

    // Two instance slots per cluster, run in alternating steps: step j runs one pass of slot
    // j % 2. At the end of step j the stores of step j - 1 are complete and every CTA arrives at
    // and waits for the cluster barrier phase of step j - 1, so the data a pass reads (written by
    // the previous pass of the same slot, two steps earlier) is visible before its first tile is
    // loaded, while step j's stores drain during step j + 1. Instances come from a fixed
    // round-robin queue.
    int sidx[2], spass[2], sfin[2];
    int next = cid;
    auto refill = [&](int sl) {
        sidx[sl] = next < count ? next : -1;
        next += ncl;
        spass[sl] = 0;
        sfin[sl] = -1;
        if (sidx[sl] >= 0) {
            // the descriptor's fields in one round trip, then Q and the parameters in flight
            // together (staged in the pass-0 scratch, which is free here)
            const CsInstDev* Ip = insts + sidx[sl];
            // the slot's shared copy of the descriptor, read by every step and prefetch of the
            // instance (ordered before them by the barriers that end set_layer_consts)
            if (threadIdx.x < sizeof(CsInstDev) / 8)
                reinterpret_cast<unsigned long long*>(sm + o.desc[sl])[threadIdx.x] =
                    reinterpret_cast<const unsigned long long*>(Ip)[threadIdx.x];
            const int n = Ip->n, p = Ip->p;
            const float* Qg = Ip->Q;
            const float* gg = Ip->gamma;
            const float* bg = Ip->beta;
            float* sQ = reinterpret_cast<float*>(sm + o.Q[sl]);
            float* gst = reinterpret_cast<float*>(sm + o.escr);
            float* bst = gst + 64;
            const int nn = n * n;
            const float q0 = (int)threadIdx.x < nn ? Qg[threadIdx.x] : 0.0f;
            const float q1 = (int)threadIdx.x + NT < nn ? Qg[threadIdx.x + NT] : 0.0f;
            if ((int)threadIdx.x < p) {
                gst[threadIdx.x] = gg[threadIdx.x];
                bst[threadIdx.x] = bg[threadIdx.x];
            }
            if ((int)threadIdx.x < nn) sQ[threadIdx.x] = q0;
            if ((int)threadIdx.x + NT < nn) sQ[threadIdx.x + NT] = q1;
            // thread l reads back only its own staged gamma_l, beta_l; the Q stores are ordered
            // before their readers by the barriers that end set_layer_consts
            set_layer_consts<float>(reinterpret_cast<LayerConst<float>*>(sm + o.lc[sl]), gst, bst, p, n,
                                    true);
        }
    };
    refill(0);
    refill(1);
    // thread 0: TMA load of tile tau of a pass of instance I into the buffers: the energies at
    // once (no store of a pass > 0 reads their buffer), the state once the last tile's store has
    // read the state buffer (wait_store)
    const auto issue_load = [&](const CsInstDev& I, bool kindA, uint32_t tau, bool wait_store) {
        fence_async_global();
        mbar_expect_tx(mbar, TD * 8 + TD * 4);
        if (kindA) tma_load_3d(sE, &I.maps[2], 0, 0, (int)tau, mbar);
        else tma_load_4d(sE, &I.maps[3], 0, 0, (int)tau, 0, mbar);
        if (wait_store) bulk_wait_read();
        if (kindA) tma_load_4d(sp, &I.maps[0], 0, 0, 0, (int)tau, mbar);
        else tma_load_4d(sp, &I.maps[1], 0, 0, (int)tau, 0, mbar);
    };
    bool prefetched = false;   // the first tile of this step was loaded at the end of the last one

    int j = 0;
    for (;; ++j) {
        const int sl = j & 1;
        bool stored = false;   // thread 0: this step committed a bulk store group
        if (sfin[sl] >= 0) {
            // the instance of this slot finished two steps ago (its final pass is visible to the
            // cluster): rank 0 merges the CTAs' <C> partials (rank order) and top-k lists
            if (rank == 0) {
                const CsInstDev& I = *reinterpret_cast<const CsInstDev*>(sm + o.desc[sl]);
                double* cex = reinterpret_cast<double*>(sm + o.cex[sl]);
                TopEnt* lists = reinterpret_cast<TopEnt*>(sm + o.lists[sl]);
                if (threadIdx.x == 0 && I.expect) {
                    // the C remote loads in flight together, then the sum in rank order
                    double part[C];
#pragma unroll
                    for (int r = 0; r < C; ++r) part[r] = *cl.map_shared_rank(cex, r);
                    double acc = 0.0;
#pragma unroll
                    for (int r = 0; r < C; ++r) acc += part[r];
                    *I.expect = acc;
                }
                if (I.k > 0) {
                    const int per = TPC * I.k;
                    for (int e = threadIdx.x; e < C * per; e += NT)
                        ts.cand[e] = cl.map_shared_rank(lists, e / per)[e % per];
                    __syncthreads();
                    cs_rank_select(ts.cand, C * per, I.k, ts.out);
                    __syncthreads();
                    if (threadIdx.x < (unsigned)I.k) {
                        const TopEnt e = ts.out[threadIdx.x];
                        if (I.topk_idx) I.topk_idx[threadIdx.x] = (uint64_t)e.z;
                        if (I.topk_prob) I.topk_prob[threadIdx.x] = e.p;
                    }
                }
            }
            fence_async_smem();   // the merge's writes to the energy tile before a TMA load refills it
            __syncthreads();
            refill(sl);
        }
        if (sidx[0] < 0 && sidx[1] < 0) break;
        if (sidx[sl] >= 0) {
            const CsInstDev& I = *reinterpret_cast<const CsInstDev*>(sm + o.desc[sl]);
            const float* sQ = reinterpret_cast<const float*>(sm + o.Q[sl]);
            const LayerConst<float>* lc = reinterpret_cast<const LayerConst<float>*>(sm + o.lc[sl]);
            TopEnt* lists = reinterpret_cast<TopEnt*>(sm + o.lists[sl]);
            const int n = I.n, p = I.p, pass = spass[sl];
            const bool kindA = (pass & 1) == 0;
            const bool fin = pass == p;
            double my_ex = 0.0;
            for (int jt = 0; jt < TPC; ++jt) {
                const uint32_t tau = rank + (uint32_t)(jt * C);
                float accp = 0.0f, pmax = -1.0f;   // final pass: FP32 <C> terms (32 per thread) and max |psi|^2
                // the bulk stores of the previous tile have read the buffers before they are
                // refilled (by TMA in passes > 0, whose load waits for them itself; by the threads
                // in pass 0, once the tile's energies are in registers; the first tile of a step
                // follows the end-of-step wait)
                if (pass > 0) {
                    if (threadIdx.x == 0 && ok && !(jt == 0 && prefetched)) issue_load(I, kindA, tau, jt > 0);
                    if (ok) ok = mbar_wait_bounded(mbar, parity);
                    ok = __syncthreads_and(ok);
                    parity ^= 1u;
                }
                if (kindA) {
                    if (pass == 0) {
                        // energies, |+>, the first cost phase and layer 0 on window [8, 13)
                        float ev[32];
                        w2_energies(n, tau << TB, sQ, reinterpret_cast<float*>(sm + o.escr), ev);
                        if (jt > 0) {
                            if (threadIdx.x == 0) bulk_wait_read();
                            __syncthreads();
                        }
                        const uint32_t t = threadIdx.x;
#pragma unroll
                        for (int i = 0; i < 32; ++i) sE[t + ((uint32_t)i << 8)] = ev[i];
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
                        } else {
                            if (lc[p - 1].shear) scale_group<5>(v, lc[p - 1].post);
#pragma unroll
                            for (int i = 0; i < 32; ++i) {
                                const float pr = v[i].x * v[i].x + v[i].y * v[i].y;
                                accp = fmaf(pr, sE[threadIdx.x + (i << 8)], accp);
                                pmax = fmaxf(pmax, pr);
                            }
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
                        } else {
                            if (lc[p - 1].shear) scale_group<H>(v, lc[p - 1].post);
#pragma unroll
                            for (int i = 0; i < (1 << H); ++i) {
                                const float pr = v[i].x * v[i].x + v[i].y * v[i].y;
                                accp = fmaf(pr, sE[lo + ((uint32_t)i << CB)], accp);
                                pmax = fmaxf(pmax, pr);
                            }
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
                        stored = true;
                    }
                } else {
                    // <C> partial and top-k list of the tile (the top-k scratch overlays the
                    // energies once the partial has read them); the state leaves in the
                    // standard frame
                    const uint32_t cmask = (1u << CB) - 1u;
                    const auto zmap = [kindA, tau, cmask](uint32_t u) -> uint32_t {
                        return kindA ? (u | (tau << TB)) : ((u & cmask) | (tau << CB) | ((u >> CB) << TB));
                    };
                    // this thread's 32 elements in the final sub-pass: shared index and global index
                    const auto elem = [kindA, tau](int i, uint32_t& ix, uint32_t& z) {
                        if (kindA) {
                            ix = psw(threadIdx.x) + ((uint32_t)i << 8);
                            z = threadIdx.x | ((uint32_t)i << 8) | (tau << TB);
                        } else {
                            const uint32_t lo = threadIdx.x + (uint32_t)((i >> H) * NT), e = (uint32_t)(i & ((1 << H) - 1));
                            ix = psw(lo) + (e << CB);
                            z = lo | (tau << CB) | (e << TB);
                        }
                    };
                    const double tot = block_sum_df(accp, reinterpret_cast<float*>(red));   // its barriers end every energy read
                    if (threadIdx.x == 0) my_ex += tot;
                    if (I.k > 0) {
                        if (!topk_own(sp, I.k, pmax, elem, ts, reinterpret_cast<float*>(sm + o.wbound))) {
                            // flat distribution: the tile-wide selection, with each thread's maximum
                            // over the elements tile_topk assigns to it
                            float pm2 = -1.0f;
                            for (uint32_t u = threadIdx.x; u < TD; u += NT) {
                                const float2 v = sp[psw(u)];
                                pm2 = fmaxf(pm2, v.x * v.x + v.y * v.y);
                            }
                            tile_topk<float, TmaLayout>(tile, I.k, pm2, zmap, ts);
                        }
                        if (threadIdx.x < (unsigned)I.k) lists[jt * I.k + threadIdx.x] = ts.out[threadIdx.x];
                    }
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
                            stored = true;
                        }
                    }
                    fence_async_smem();   // the top-k scratch writes before the next tile's TMA writes
                    __syncthreads();
                }
            }
            if (fin) {
                if (threadIdx.x == 0) *reinterpret_cast<double*>(sm + o.cex[sl]) = my_ex;
                sfin[sl] = j;
            } else {
                spass[sl] = pass + 1;
            }
        }
        // end of step j. Step j's bulk stores drain while step j + 1 computes: here only step
        // j - 1's stores must be complete (every group but the newest when step j committed one,
        // a group per stored tile, so step j - 1's are older; else all) before the CTA arrives at
        // the cluster phase of step j - 1. While that phase completes (wait: every CTA's step
        // j - 1 data is complete), every store finishes reading the buffers, which the next
        // step's prefetch of its first tile (the slot step j - 1 advanced), the pass-0 threads
        // or rank 0's merge in the energy tile reuse once the barrier after the wait is passed.
        __syncthreads();
        if (threadIdx.x == 0 && j > 0) {
            if (stored) bulk_wait_all_but_one();
            else bulk_wait_all();   // step j stored nothing: the newest group may be step j - 1's
            fence_async_global();
        }
        if (j > 0) {
            __syncthreads();
            if (threadIdx.x < 32) cluster_arrive_release();
            else cluster_arrive();
        }
        if (threadIdx.x == 0) bulk_wait_read();
        if (j > 0) cluster_wait();
        __syncthreads();
        {
            const int ns = (j + 1) & 1;
            prefetched = sidx[ns] >= 0 && sfin[ns] < 0 && spass[ns] > 0;
            if (prefetched && threadIdx.x == 0 && ok) issue_load(*reinterpret_cast<const CsInstDev*>(sm + o.desc[ns]), (spass[ns] & 1) == 0, rank, false);
        }
    }
    // The loop ends at the start of a step j in which rank 0 may have just read every rank's
    // shared memory (the last merge). Every store completes, then the phase of step j - 1, which
    // each CTA arrives at after that merge in its program order: no CTA leaves before rank 0 is
    // done with its shared memory.
    if (threadIdx.x == 0) {
        bulk_wait_all();
        fence_async_global();
    }
    __syncthreads();
    if (j > 0) {
        if (threadIdx.x < 32) cluster_arrive_release();
        else cluster_arrive();
        cluster_wait();
    }
    if (threadIdx.x == 0 && !ok) atomicOr(status, 1u);
}

template <int H>
cudaError_t cs_launch_h(const void* insts, int count, int clusters, cudaStream_t st, int* max_clusters,
                        unsigned* status) {
    constexpr int NTILE = 1 << H;
    constexpr int C = cs_cluster(NTILE);
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

int cstream_cluster_size(int n) { return cs_cluster(1 << (n - TB)); }

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
