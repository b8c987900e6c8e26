// k_stream.cu -- HBM-streaming tier for states larger than one SM's shared memory, plus the
// standalone energy build and the standalone <C> / top-k reductions over a state in HBM.
//
// A layer of Eq. 2 (Section IV) on a 2^n state is split into HBM passes. Each pass moves
// tiles of 2^tb amplitudes between HBM and shared memory and runs the tile engine on them:
//   kind A: the tile is 2^tb contiguous amplitudes; its tile bits are qubits 0..tb-1;
//   kind B: the tile is 2^c contiguous amplitudes (qubits 0..c-1, c >= 4, so every run is at
//           least 128 bytes) times 2^h values of the high qubits [s, s+h), c + h = tb; only the
//           high qubits are mixed.
// The HBM passes follow the same snake order as the windows of a tile (A, B1, B2, ... then
// back), so consecutive layers share a pass; the cost phase of a layer is fused into the pass
// that opens it, |+> is generated in the first pass, and <C> plus the top-k candidates are
// reduced in the last one (per-tile partials, then one fixed-order finalize per instance).
#include "qaoa_engine.cuh"
#include "qaoa_kernels.h"
#include "qaoa_stream.h"

namespace qaoa {

namespace {

// Global index of tile-local index u for tile tau of pass P.
__device__ __forceinline__ uint64_t global_index(const StreamPass& P, uint64_t tau, uint32_t u) {
    if (P.kind == 0) return (tau << P.tb) | u;
    const uint64_t lo = u & ((1u << P.c) - 1u);
    const uint64_t hi = u >> P.c;
    const int midbits = P.s - P.c;
    const uint64_t mid = tau & ((1ull << midbits) - 1ull);
    const uint64_t top = tau >> midbits;
    return lo | (mid << P.c) | (hi << P.s) | (top << (P.s + P.h));
}

// Per-thread strided walk over a tile: element u = u0 + j * step (step a multiple of 2^c for kind
// B, any for kind A) has global index global_index(P, tau, u0) + j * gstep. Returns false when
// kind B's contiguous run is longer than the step (then the index is formed per element).
__device__ __forceinline__ bool linear_walk(const StreamPass& P, uint32_t step, uint64_t& gstep) {
    if (P.kind == 0) { gstep = step; return true; }
    if (step & ((1u << P.c) - 1u)) return false;
    gstep = (uint64_t)(step >> P.c) << P.s;
    return true;
}

// Stage the tile's amplitudes (16-byte copies) and optionally energies (8-byte copies) of
// tile tau into shared memory, asynchronously. The swizzle only permutes bits below the copy
// stride, so the shared-memory offset advances linearly as well.
template <typename T>
__device__ __forceinline__ void stage_tile(const StreamPass& P, uint64_t tau,
                                           const typename Num<T>::C* gsrc,
                                           typename Num<T>::C* sdst, const T* gE, T* sE) {
    using C = typename Num<T>::C;
    const uint32_t TD = 1u << P.tb;
    constexpr uint32_t PAIR = sizeof(C) == 8 ? 2u : 1u;   // amplitudes per 16-byte copy
    const uint32_t step = PAIR * blockDim.x, u0 = PAIR * threadIdx.x;
    uint64_t gstep;
    if (!gsrc) {
    } else if (linear_walk(P, step, gstep)) {
        const C* g = gsrc + global_index(P, tau, u0);
        C* sp = sdst + swz<T>(u0);
#pragma unroll 4
        for (uint32_t u = u0; u < TD; u += step, g += gstep, sp += step) cp_async16(sp, g);
    } else {
        for (uint32_t u = u0; u < TD; u += step) cp_async16(&sdst[swz<T>(u)], gsrc + global_index(P, tau, u));
    }
    if (gE) {
        constexpr uint32_t EP = 8u / sizeof(T);           // energies per 8-byte copy
        const uint32_t estep = EP * blockDim.x, e0 = EP * threadIdx.x;
        uint64_t egstep;
        if (linear_walk(P, estep, egstep)) {
            const T* g = gE + global_index(P, tau, e0);
            T* sp = sE + swz<T>(e0);
#pragma unroll 4
            for (uint32_t u = e0; u < TD; u += estep, g += egstep, sp += estep) cp_async8(sp, g);
        } else {
            for (uint32_t u = e0; u < TD; u += estep) cp_async8(&sE[swz<T>(u)], gE + global_index(P, tau, u));
        }
    }
}

// Write the tile back (16-byte accesses on both sides), same walk as stage_tile.
template <typename T>
__device__ __forceinline__ void store_tile(const StreamPass& P, uint64_t tau, const typename Num<T>::C* ssrc,
                                          typename Num<T>::C* gdst) {
    using C = typename Num<T>::C;
    const uint32_t TD = 1u << P.tb;
    constexpr uint32_t PAIR = sizeof(C) == 8 ? 2u : 1u;
    const uint32_t step = PAIR * blockDim.x, u0 = PAIR * threadIdx.x;
    uint64_t gstep;
    if (linear_walk(P, step, gstep)) {
        C* g = gdst + global_index(P, tau, u0);
        const C* sp = ssrc + swz<T>(u0);
        for (uint32_t u = u0; u < TD; u += step, g += gstep, sp += step)
            *reinterpret_cast<uint4*>(g) = *reinterpret_cast<const uint4*>(sp);
    } else {
        for (uint32_t u = u0; u < TD; u += step)
            *reinterpret_cast<uint4*>(gdst + global_index(P, tau, u)) =
                *reinterpret_cast<const uint4*>(&ssrc[swz<T>(u)]);
    }
}

template <typename T>
struct StreamSmem {
    typename Num<T>::C* psi;
    T* E;
    LayerConst<T>* lc;
    double* red;
    TileTopk tk;
    TopEnt* run;     // running top-k of the state's tiles this block reduced (last pass)
};

// have_run: this block reduced tile prev_tau of the same state just before (last pass, k >= 1);
// s.run then holds the top-k of all the state's tiles it reduced so far.
template <typename T, int R>
__device__ void stream_tile(const StreamPass& P, const StreamInst<T>& I, uint64_t tau,
                            const StreamSmem<T>& s, bool have_run, uint64_t prev_tau) {
    using C = typename Num<T>::C;
    const uint32_t TD = 1u << P.tb;
    const bool needE = P.need_e;
    C* gpsi = reinterpret_cast<C*>(I.psi);
    // ---- HBM -> shared: asynchronous 16-byte copies, all in flight before the wait ----
    // (tile bit 0 is global bit 0 and c >= 1, so aligned pairs stay adjacent in both layouts)
    if (!P.init) stage_tile<T>(P, tau, gpsi, s.psi, needE ? I.E : nullptr, s.E);
    else if (needE) stage_tile<T>(P, tau, nullptr, nullptr, I.E, s.E);
    cp_async_wait_all();
    __syncthreads();
    // ---- tile engine: snake over the local windows of the mixed bits, layers [la, lb] ----
    const TileRef<T> tile{s.psi, nullptr, s.E, P.tb};
    const int m0 = (P.kind == 0) ? 0 : P.c;
    const int G = num_windows(m0, P.tb, R);
    const int nl = P.lb - P.la + 1;
    const int S = snake_len(G, nl);
    const T amp0 = (T)I.amp0;
    auto nofin = [](uint32_t, int, bool) {};
    for (int si = 0; si < S; ++si) {
        SubPass sp;
        snake_step(si, G, nl, P.la, P.ph_first, m0, P.tb, P.tb, R, sp);
        sp.post = P.fin && (si == S - 1);
        subpass_fwd<T, R>(tile, sp, s.lc, P.init && si == 0, amp0, __popcll(tau), nofin);
        __syncthreads();
    }
    // ---- shared -> HBM (16-byte accesses on both sides). Between passes the state stays in
    // the rotated frame; the last pass converts back with (-i)^{|z|} (|z| = |tau| + |u|: the
    // tile map only permutes bits). ----
    if (!P.fin || P.keep_frame) {
        store_tile<T>(P, tau, s.psi, gpsi);
    } else if (!P.no_store) {
        const int pt = __popcll(tau);
        constexpr uint32_t PAIR = sizeof(C) == 8 ? 2u : 1u;
        const uint32_t step = PAIR * blockDim.x, u0 = PAIR * threadIdx.x;
        uint64_t gstep;
        if (linear_walk(P, step, gstep)) {
            C* g = gpsi + global_index(P, tau, u0);
            for (uint32_t u = u0; u < TD; u += step, g += gstep) {
                const uint32_t su = swz<T>(u);
                if constexpr (PAIR == 2) {
                    const C a = times_i_pow(s.psi[su], -(pt + __popc(u)));
                    const C b = times_i_pow(s.psi[su + 1], -(pt + __popc(u + 1)));
                    *reinterpret_cast<float4*>(g) = make_float4(a.x, a.y, b.x, b.y);
                } else {
                    *g = times_i_pow(s.psi[su], -(pt + __popc(u)));
                }
            }
        } else {
            for (uint32_t u = threadIdx.x; u < TD; u += blockDim.x)
                gpsi[global_index(P, tau, u)] = times_i_pow(s.psi[swz<T>(u)], -(pt + __popc(u)));
        }
    }
    if (P.fin) {
        double ex = 0.0;
        const StreamPass Pm = P;   // by value: the lambda then holds no address of a kernel parameter
        const auto zmap = [Pm, tau](uint32_t u) { return (uint32_t)global_index(Pm, tau, u); };
        const float pmax = tile_expect<T>(tile, ex);
        if (P.k > 0) {
            if (have_run) {
                running_topk<T>(tile, P.k, pmax, zmap, s.tk, s.run);
            } else {
                tile_topk<T>(tile, P.k, pmax, zmap, s.tk);
                if (threadIdx.x < (unsigned)P.k) s.run[threadIdx.x] = s.tk.out[threadIdx.x];
            }
        }
        const double tot = block_sum(ex, s.red);
        if (threadIdx.x == 0) I.part_expect[tau] = tot;
        // the running list goes to this tile's slot and the previous tile's slot is emptied (the
        // same thread wrote it), so each state's slots hold every candidate exactly once
        if (threadIdx.x < (unsigned)P.k) {
            const TopEnt e = s.run[threadIdx.x];
            I.part_topp[tau * P.k + threadIdx.x] = e.p;
            I.part_topz[tau * P.k + threadIdx.x] = e.z;
            if (have_run) {
                I.part_topp[prev_tau * P.k + threadIdx.x] = -1.0;
                I.part_topz[prev_tau * P.k + threadIdx.x] = 0xffffffffu;
            }
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_stream_pass(const StreamPass P,
                                                     const StreamInst<T>* __restrict__ insts,
                                                     int count, const StreamInst<T> one) {
    extern __shared__ __align__(16) unsigned char sm[];
    using C = typename Num<T>::C;
    const uint32_t TD = 1u << P.tb;
    StreamSmem<T> s;
    size_t o = 0;
    s.psi = reinterpret_cast<C*>(sm + o); o += (size_t)TD * sizeof(C);
    s.E = reinterpret_cast<T*>(sm + o); o += (size_t)TD * sizeof(T);
    s.lc = reinterpret_cast<LayerConst<T>*>(sm + o); o += 64 * sizeof(LayerConst<T>);
    o = (o + 15) & ~(size_t)15;
    s.red = reinterpret_cast<double*>(sm + o); o += 32 * sizeof(double);
    s.tk.wlists = reinterpret_cast<TopEnt*>(sm + o); o += 8 * 32 * sizeof(TopEnt);
    s.tk.cand = reinterpret_cast<TopEnt*>(sm + o); o += TOPK_CAP * sizeof(TopEnt);
    s.tk.out = reinterpret_cast<TopEnt*>(sm + o); o += 16 * sizeof(TopEnt);
    s.run = reinterpret_cast<TopEnt*>(sm + o); o += 16 * sizeof(TopEnt);
    s.tk.wb = reinterpret_cast<float*>(sm + o); o += 16 * 32 * sizeof(float);
    s.tk.cnt = reinterpret_cast<int*>(sm + o);
    const uint64_t ntiles = 1ull << (P.n - P.tb);
    const uint64_t total = ntiles * (uint64_t)count;
    // layer constants are rebuilt only when the parameters change (instances of a batch often
    // share one parameter vector)
    const T *cur_g = nullptr, *cur_b = nullptr;
    int cur_p = 0;
    // The last pass with a top-k gives each block a run of consecutive tiles instead of a
    // grid-strided share, so that the tiles of one state follow each other and the block carries
    // one top-k list across them. The run lengths are those of the strided share: total / grid,
    // one more for the first total % grid blocks.
    uint64_t b = blockIdx.x, bstep = gridDim.x, bend = total;
    if (P.fin && P.k > 0) {
        const uint64_t q = total / gridDim.x, rem = total % gridDim.x, c = blockIdx.x;
        b = c * q + (c < rem ? c : rem);
        bend = b + q + (c < rem ? 1 : 0);
        bstep = 1;
    }
    int run_ii = -1;
    uint64_t run_tau = 0;
    for (; b < bend; b += bstep) {
        const int ii = (int)(b / ntiles);
        const uint64_t tau = b % ntiles;
        const StreamInst<T>& I = insts ? insts[ii] : one;
        if (I.gamma != cur_g || I.beta != cur_b || I.p != cur_p) {
            __syncthreads();
            set_layer_consts<T>(s.lc, I.gamma, I.beta, I.p, P.n, true);
            __syncthreads();
            cur_g = I.gamma;
            cur_b = I.beta;
            cur_p = I.p;
        }
        constexpr int RB = Num<T>::RB;
        stream_tile<T, RB>(P, I, tau, s, run_ii == ii, run_tau);
        run_ii = ii;
        run_tau = tau;
    }
}

// Merge the top-k lists of `nl` lists (list j at tile slot j * stride) into one list of the k
// best (probability desc, index asc; unique, so any merge order gives the same list): each warp
// takes a strided share of the entries, then warp 0 merges the warps' lists. The result is in
// lanes 0..k-1 of warp 0 (f.p, f.z).
__device__ __forceinline__ void merge_lists(const double* topp, const uint32_t* topz, uint64_t nl,
                                            uint64_t stride, int k, TopEnt* tops, WarpTopK& f) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpTopK top;
    top.init(k);
    const uint64_t nent = nl * (uint64_t)k;
    for (uint64_t e0 = (uint64_t)warp * 32; e0 < nent; e0 += (uint64_t)(blockDim.x >> 5) * 32) {
        const uint64_t e = e0 + lane;
        const bool ok = e < nent;
        const uint64_t a = ok ? (e / k) * stride * k + e % k : 0;
        top.offer_exact(ok ? topp[a] : -1.0, ok ? topz[a] : 0u, ok);
    }
    if (lane < k) tops[warp * 32 + lane] = TopEnt{top.p, top.z};
    __syncthreads();
    if (warp == 0) {
        f.init(k);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const bool ok = lane < k;
            const TopEnt e = ok ? tops[w * 32 + lane] : TopEnt{-1.0, 0xffffffffu};
            f.offer_exact(e.p, e.z, ok);
        }
    }
}

// First merge level for instances with many tiles: block (c, i) merges the lists of tiles
// [c * FIN_CHUNK, (c + 1) * FIN_CHUNK) of instance i and writes the result over the list of the
// chunk's first tile (only this block reads the chunk, and it reads everything first).
constexpr uint64_t FIN_CHUNK = 256;

template <typename T>
__global__ void __launch_bounds__(256) k_stream_topk_chunks(const StreamInst<T>* __restrict__ insts,
                                                           int count, uint64_t ntiles, int k,
                                                           const StreamInst<T> one) {
    __shared__ TopEnt tops[8 * 32];
    const int ii = blockIdx.y;
    if (ii >= count) return;
    const StreamInst<T>& I = insts ? insts[ii] : one;
    const uint64_t t0 = (uint64_t)blockIdx.x * FIN_CHUNK;
    const uint64_t nl = (ntiles - t0) < FIN_CHUNK ? (ntiles - t0) : FIN_CHUNK;
    WarpTopK f;
    merge_lists(I.part_topp + t0 * k, I.part_topz + t0 * k, nl, 1, k, tops, f);
    __syncthreads();   // every read of the chunk is done before its first list is overwritten
    if (threadIdx.x < (unsigned)k) {
        I.part_topp[t0 * k + threadIdx.x] = f.p;
        I.part_topz[t0 * k + threadIdx.x] = f.z;
    }
}

// Per-instance finalize: <C> = fixed-order sum of the tile partials; top-k = merge of the lists
// at tile slots 0, stride, 2 stride, ... (stride 1: every tile's list; FIN_CHUNK after the first
// merge level).
template <typename T>
__global__ void __launch_bounds__(256) k_stream_finalize(const StreamInst<T>* __restrict__ insts,
                                                         int count, uint64_t ntiles, int k,
                                                         uint64_t stride, const StreamInst<T> one) {
    __shared__ double red[32];
    __shared__ TopEnt tops[8 * 32];
    const int ii = blockIdx.x;
    if (ii >= count) return;
    const StreamInst<T>& I = insts ? insts[ii] : one;
    // sum: each thread a contiguous slice (fixed), then the block tree
    double acc = 0.0;
    const uint64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const uint64_t b0 = threadIdx.x * per;
    for (uint64_t t = b0; t < b0 + per && t < ntiles; ++t) acc += I.part_expect[t];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0 && I.expect) *I.expect = tot;
    if (k > 0) {
        const uint64_t nl = (ntiles + stride - 1) / stride;
        WarpTopK f;
        merge_lists(I.part_topp, I.part_topz, nl, stride, k, tops, f);
        if (threadIdx.x < (unsigned)k) {
            if (I.topk_idx) I.topk_idx[threadIdx.x] = (uint64_t)f.z;
            if (I.topk_prob) I.topk_prob[threadIdx.x] = f.p;
        }
    }
}

// ---- adjoint passes -----------------------------------------------------------------------
// Two CTAs per SM: psi, lam and E tiles of 2^12 (float) or 2^11 (double) amplitudes each.
constexpr int ADJ_THREADS = 256;
// The forward pass P undone on a tile of psi and lam (both in the rotated frame), with the
// gradient accumulations of the tile engine's adjoint sub-passes: the local snake of P with
// RB_ADJ-bit windows, run in reverse. Per tile, four partial sums are written (as FP64):
//   [0] Im <lam|B|psi> of layer lb, [1] of layer la (lb > la), [2] Im <lam|E|psi> of layer lb,
//   [3] of layer la -- zero where the pass holds no such operation.
template <typename T, int RA>
__device__ void stream_adj_tile(const StreamPass& P, int si, bool lam_first, bool store,
                                const StreamInst<T>& I, uint64_t tau, const StreamSmem<T>& s,
                                typename Num<T>::C* slam) {
    using C = typename Num<T>::C;
    C* gpsi = reinterpret_cast<C*>(I.psi);
    C* glam = reinterpret_cast<C*>(I.lam);
    stage_tile<T>(P, tau, gpsi, s.psi, I.E, s.E);
    if (!lam_first) stage_tile<T>(P, tau, glam, slam, nullptr, nullptr);
    cp_async_wait_all();
    __syncthreads();
    const TileRef<T> tile{s.psi, slam, s.E, P.tb};
    const int m0 = (P.kind == 0) ? 0 : P.c;
    const int G = num_windows(m0, P.tb, RA);
    const int nl = P.lb - P.la + 1;
    const int S = snake_len(G, nl);
    // tile accumulators by the pass's layer slot (0: layer lb, 1: layer la); a local
    // sub-pass reports relative to its own last layer, mapped here
    T ab[2] = {T(0), T(0)}, ag[2] = {T(0), T(0)};
    for (int k = S - 1; k >= 0; --k) {
        SubPass sp;
        snake_step(k, G, nl, P.la, P.ph_first, m0, P.tb, P.tb, RA, sp);
        T lb_[2] = {T(0), T(0)}, lg_[2] = {T(0), T(0)};
        subpass_adj<T, RA>(tile, sp, s.lc, lam_first && k == S - 1, lb_, lg_);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int slot = P.lb - (sp.lb - j);
            if (j <= sp.lb - sp.la) {
                if (slot == 0) { ab[0] += lb_[j]; ag[0] += lg_[j]; }
                else { ab[1] += lb_[j]; ag[1] += lg_[j]; }
            }
        }
        __syncthreads();
    }
    double* out = I.part_grad + ((uint64_t)si << (P.n - P.tb)) * 4 + tau * 4;
    const double v0 = block_sum((double)ab[0], s.red);
    const double v1 = block_sum((double)ab[1], s.red);
    const double v2 = block_sum((double)ag[0], s.red);
    const double v3 = block_sum((double)ag[1], s.red);
    if (threadIdx.x == 0) { out[0] = v0; out[1] = v1; out[2] = v2; out[3] = v3; }
    if (store) {
        store_tile<T>(P, tau, s.psi, gpsi);
        store_tile<T>(P, tau, slam, glam);
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(ADJ_THREADS, 2) k_stream_adj_pass(const StreamPass P, int si, int lam_first,
                                                         int store,
                                                         const StreamInst<T>* __restrict__ insts,
                                                         int count, const StreamInst<T> one) {
    extern __shared__ __align__(16) unsigned char sm[];
    using C = typename Num<T>::C;
    const uint32_t TD = 1u << P.tb;
    StreamSmem<T> s;
    size_t o = 0;
    s.psi = reinterpret_cast<C*>(sm + o); o += (size_t)TD * sizeof(C);
    C* slam = reinterpret_cast<C*>(sm + o); o += (size_t)TD * sizeof(C);
    s.E = reinterpret_cast<T*>(sm + o); o += (size_t)TD * sizeof(T);
    s.lc = reinterpret_cast<LayerConst<T>*>(sm + o); o += 64 * sizeof(LayerConst<T>);
    o = (o + 15) & ~(size_t)15;
    s.red = reinterpret_cast<double*>(sm + o);
    const uint64_t ntiles = 1ull << (P.n - P.tb);
    const uint64_t total = ntiles * (uint64_t)count;
    const T *cur_g = nullptr, *cur_b = nullptr;
    int cur_p = 0;
    for (uint64_t b = blockIdx.x; b < total; b += gridDim.x) {
        const int ii = (int)(b / ntiles);
        const uint64_t tau = b % ntiles;
        const StreamInst<T>& I = insts ? insts[ii] : one;
        if (I.gamma != cur_g || I.beta != cur_b || I.p != cur_p) {
            __syncthreads();
            set_layer_consts<T>(s.lc, I.gamma, I.beta, I.p, P.n, false);
            cur_g = I.gamma;
            cur_b = I.beta;
            cur_p = I.p;
        }
        constexpr int RA = Num<T>::RB_ADJ;
        stream_adj_tile<T, RA>(P, si, lam_first != 0, store != 0, I, tau, s, slam);
    }
}

// Per instance: dgamma_l = 2 sum of the gamma slots of layer l, dbeta_l = 2 sum of the beta
// slots, over passes in order and tiles in fixed contiguous chunks per thread.
struct PassLayers {
    int la[256], lb[256];
};
template <typename T>
__global__ void __launch_bounds__(256) k_stream_grad_reduce(const PassLayers pl, int S,
                                                            const StreamInst<T>* __restrict__ insts,
                                                            int count, uint64_t ntiles,
                                                            const StreamInst<T> one) {
    __shared__ double red[32];
    const int ii = blockIdx.x;
    if (ii >= count) return;
    const StreamInst<T>& I = insts ? insts[ii] : one;
    const uint64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    for (int l = 0; l < I.p; ++l) {
        double gb = 0.0, gg = 0.0;
        for (int s = 0; s < S; ++s) {
            const bool hb = pl.lb[s] == l, ha = pl.la[s] == l && pl.lb[s] != pl.la[s];
            if (!hb && !ha) continue;
            const double* base = I.part_grad + ((uint64_t)s * ntiles) * 4;
            for (uint64_t t = threadIdx.x * per; t < (threadIdx.x + 1) * per && t < ntiles; ++t) {
                const double* q = base + t * 4;
                if (hb) { gb += q[0]; gg += q[2]; }
                if (ha) { gb += q[1]; gg += q[3]; }
            }
        }
        const double sb = block_sum(gb, red);
        const double sg = block_sum(gg, red);
        if (threadIdx.x == 0) {
            if (I.dbeta) I.dbeta[l] = 2.0 * sb;
            if (I.dgamma) I.dgamma[l] = 2.0 * sg;
        }
    }
}

// ---- energy build into HBM, row form (n >= 2) ------------------------------------------
// E(z) = sum_i Q_ii z_i + sum_{i<j} W_ij z_i z_j with W_ij = Q_ij + Q_ji (Q need not be
// symmetric). Split z = (hi, lo) with hi the top nh bits and m = n - nh. A thread fixes lo up to
// its two lowest bits and holds the four energies E(hi, lo | v), v = 0..3, and the cross fields
//   P_h(lo | v) = sum_{j in lo|v} W_{m+h, j}              (h < nh),
// then walks hi in Gray-code order: flipping bit b of hi changes every energy by
//   s * (P_b(lo|v) + Q_{b'b'} + sum_{j in hi, j != b} W_{b'j'})   (s = +1 setting, -1 clearing;
// primes: positions m + b, m + j). The hi-only part depends on the step alone, so a table D[k]
// of it (sign included) is built once per block; each step costs one select, eight adds and one
// 16-byte (float) or two (double) stores of four consecutive energies. The walk is at most 2^8
// steps, which bounds the FP32 rounding drift of the running sums.
constexpr int ROWS_NH_MAX = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_energy_rows(int n, int nh, const T* __restrict__ Q,
                                                     T* __restrict__ E, const StreamInst<T>* insts) {
    __shared__ T W[32 * 32];
    __shared__ T D[1 << ROWS_NH_MAX];
    if (insts) {
        Q = insts[blockIdx.y].Q;
        E = const_cast<T*>(insts[blockIdx.y].E);
    }
    for (int x = threadIdx.x; x < n * n; x += blockDim.x) {
        const int i = x / n, j = x - i * n;
        W[x] = (i == j) ? Q[x] : Q[x] + Q[j * n + i];
    }
    __syncthreads();
    const int m = n - nh;
    const int steps = 1 << nh;
    for (int k = 1 + threadIdx.x; k < steps; k += blockDim.x) {
        const int b = __ffs(k) - 1;
        const uint32_t g = (uint32_t)(k - 1) ^ ((uint32_t)(k - 1) >> 1);   // hi before the flip
        const T* row = W + (m + b) * n + m;
        T d = row[b];
        for (int j = 0; j < nh; ++j)
            if (j != b && ((g >> j) & 1u)) d += row[j];
        D[k] = ((g >> b) & 1u) ? -d : d;
    }
    __syncthreads();
    const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (1ull << (m - 2))) return;
    const uint32_t base = (uint32_t)gid << 2;
    // exact energies of lo = base | v at hi = 0
    T eb = T(0), f0 = W[0], f1 = W[n + 1];
    for (int i = 2; i < m; ++i) {
        if (!((base >> i) & 1u)) continue;
        const T* row = W + i * n;
        T r = row[i];
        for (int j = 2; j < i; ++j)
            if ((base >> j) & 1u) r += row[j];
        eb += r;
        f0 += row[0];
        f1 += row[1];
    }
    T e[4] = {eb, eb + f0, eb + f1, eb + f0 + f1 + W[1]};
    T P[ROWS_NH_MAX][4];
#pragma unroll
    for (int h = 0; h < ROWS_NH_MAX; ++h) {
        if (h < nh) {
            const T* row = W + (m + h) * n;
            T pb = T(0);
            for (int j = 2; j < m; ++j)
                if ((base >> j) & 1u) pb += row[j];
            P[h][0] = pb;
            P[h][1] = pb + row[0];
            P[h][2] = pb + row[1];
            P[h][3] = pb + row[0] + row[1];
        } else {
            P[h][0] = P[h][1] = P[h][2] = P[h][3] = T(0);
        }
    }
    // E is 8-byte aligned (checked when the plan is made); 16-byte stores where it is 16-aligned
    const bool v16 = (reinterpret_cast<uintptr_t>(E) & 15u) == 0;
    auto put = [&](uint32_t hi) {
        T* dst = E + (((uint64_t)hi << m) | base);
        if constexpr (sizeof(T) == 4) {
            if (v16) {
                *reinterpret_cast<float4*>(dst) = make_float4(e[0], e[1], e[2], e[3]);
            } else {
                reinterpret_cast<float2*>(dst)[0] = make_float2(e[0], e[1]);
                reinterpret_cast<float2*>(dst)[1] = make_float2(e[2], e[3]);
            }
        } else {
            if (v16) {
                reinterpret_cast<double2*>(dst)[0] = make_double2(e[0], e[1]);
                reinterpret_cast<double2*>(dst)[1] = make_double2(e[2], e[3]);
            } else {
                dst[0] = e[0]; dst[1] = e[1]; dst[2] = e[2]; dst[3] = e[3];
            }
        }
    };
    put(0u);
    uint32_t hi = 0;
    for (int k = 1; k < steps; ++k) {
        const int b = __ffs(k) - 1;
        hi ^= 1u << b;
        T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
#pragma unroll
        for (int h = 0; h < ROWS_NH_MAX; ++h)
            if (h == b) { p0 = P[h][0]; p1 = P[h][1]; p2 = P[h][2]; p3 = P[h][3]; }
        if (!((hi >> b) & 1u)) { p0 = -p0; p1 = -p1; p2 = -p2; p3 = -p3; }
        const T d = D[k];
        e[0] += p0 + d;
        e[1] += p1 + d;
        e[2] += p2 + d;
        e[3] += p3 + d;
        put(hi);
    }
}

// ---- energy build into HBM --------------------------------------------------------------
// Thread t of 2^m fixes the low m bits of z and walks the high n - m bits in Gray-code order
// (same increment rule as the resident tier); every step writes one coalesced row of E.
// blockIdx.y selects the instance when insts != nullptr (then Q and E come from it).
template <typename T>
__global__ void __launch_bounds__(256) k_energy(int n, int m, const T* __restrict__ Q,
                                                T* __restrict__ E, const StreamInst<T>* insts) {
    __shared__ T Qs[32 * 32];
    if (insts) {
        Q = insts[blockIdx.y].Q;
        E = const_cast<T*>(insts[blockIdx.y].E);
    }
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Qs[i] = Q[i];
    __syncthreads();
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (1ull << m)) return;
    const int nh = n - m;
    T e = T(0);
    for (int i = 0; i < m; ++i) {
        if (!((t >> i) & 1u)) continue;
        for (int j = 0; j < m; ++j)
            if ((t >> j) & 1u) e += Qs[i * n + j];
    }
    constexpr int MAXH = 12;
    T F[MAXH];
#pragma unroll
    for (int h = 0; h < MAXH; ++h) {
        T f = T(0);
        if (h < nh)
            for (int j = 0; j < m; ++j)
                if ((t >> j) & 1u) f += Qs[(m + h) * n + j];
        F[h] = f;
    }
    uint64_t z = t;
    E[z] = e;
    const uint32_t steps = 1u << nh;
    for (uint32_t k = 1; k < steps; ++k) {
        const int b = __ffs((int)k) - 1;
        const int hb = m + b;
        const T d = ((z >> hb) & 1ull) ? T(-1) : T(1);
        T fb = T(0);
#pragma unroll
        for (int h = 0; h < MAXH; ++h)
            if (h == b) fb = F[h];
        e += d * (Qs[hb * n + hb] + T(2) * fb);
        z ^= 1ull << hb;
#pragma unroll
        for (int h = 0; h < MAXH; ++h)
            if (h < nh && h != b) F[h] += d * Qs[(m + h) * n + hb];
        E[z] = e;
    }
}

// ---- standalone <C> and top-k over a state in HBM ----------------------------------------
// Grid-stride over elements; each thread accumulates FP32 products over at most 32 elements
// before adding them to its FP64 partial; per-CTA partials and top-k lists go to the
// caller-provided scratch and are merged by k_stream_finalize-style reduction.
template <typename T>
__global__ void __launch_bounds__(256) k_reduce_state(int n, const typename Num<T>::C* __restrict__ psi,
                                                      const T* __restrict__ E, int k,
                                                      double* part_expect, double* part_topp,
                                                      uint32_t* part_topz) {
    __shared__ double red[32];
    __shared__ TopEnt tops[8 * 32];
    const uint64_t D = 1ull << n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpTopK top;
    top.init(k > 0 ? k : 1);
    double ex = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // chunks of 32 consecutive strides so that the FP32 partial has at most 32 terms
    for (uint64_t c0 = (uint64_t)blockIdx.x * blockDim.x; c0 < D; c0 += stride * 32) {
        T acc = T(0);
        for (int r = 0; r < 32; ++r) {
            const uint64_t z = c0 + (uint64_t)r * stride + threadIdx.x;
            const bool ok = z < D;
            typename Num<T>::C v;
            v.x = T(0); v.y = T(0);
            if (ok) {
                v = psi[z];
                if (E) acc += (v.x * v.x + v.y * v.y) * E[z];
            }
            if (k > 0) top.offer(v, (uint32_t)z, ok);
        }
        ex += (double)acc;
    }
    const double tot = block_sum(ex, red);
    if (threadIdx.x == 0) part_expect[blockIdx.x] = tot;
    if (k > 0) {
        if (lane < k) tops[warp * 32 + lane] = TopEnt{top.p, top.z};
        __syncthreads();
        if (warp == 0) {
            WarpTopK f;
            f.init(k);
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                const bool ok = lane < k;
                const TopEnt e = ok ? tops[w * 32 + lane] : TopEnt{-1.0, 0xffffffffu};
                f.offer_exact(e.p, e.z, ok);
            }
            if (lane < k) {
                part_topp[(uint64_t)blockIdx.x * k + lane] = f.p;
                part_topz[(uint64_t)blockIdx.x * k + lane] = f.z;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_reduce_finalize(int nparts, const double* part_expect,
                                                         const double* part_topp,
                                                         const uint32_t* part_topz, int k,
                                                         double* expect, uint64_t* topk_idx,
                                                         double* topk_prob) {
    __shared__ double red[32];
    __shared__ TopEnt tops[8 * 32];
    double acc = 0.0;
    const int per = (nparts + blockDim.x - 1) / blockDim.x;
    for (int t = threadIdx.x * per; t < (int)(threadIdx.x + 1) * per && t < nparts; ++t)
        acc += part_expect[t];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0 && expect) *expect = tot;
    if (k > 0) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        WarpTopK top;
        top.init(k);
        const int nent = nparts * k;
        for (int e0 = warp * 32; e0 < nent; e0 += (int)(blockDim.x >> 5) * 32) {
            const int e = e0 + lane;
            const bool ok = e < nent;
            top.offer_exact(ok ? part_topp[e] : -1.0, ok ? part_topz[e] : 0u, ok);
        }
        if (lane < k) tops[warp * 32 + lane] = TopEnt{top.p, top.z};
        __syncthreads();
        if (warp == 0) {
            WarpTopK f;
            f.init(k);
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                const bool ok = lane < k;
                const TopEnt e = ok ? tops[w * 32 + lane] : TopEnt{-1.0, 0xffffffffu};
                f.offer_exact(e.p, e.z, ok);
            }
            if (lane < k) {
                if (topk_idx) topk_idx[lane] = (uint64_t)f.z;
                if (topk_prob) topk_prob[lane] = f.p;
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------

int stream_tile_bits(bool dbl) { return dbl ? 12 : 13; }
int stream_adj_tile_bits(bool dbl) { return dbl ? 11 : 12; }

// HBM windows of a layer: window 0 = kind A (qubits 0..tb-1); windows 1.. = kind B chunks of
// the qubits [tb, n), as equal as possible, each at most tb - 4 qubits.
int stream_plan(bool dbl, int n, int p, int k, StreamPass* out, int max_out, int tb) {
    if (tb < 0) tb = stream_tile_bits(dbl);
    if (n <= tb) return -1;
    const int hmax = tb - 4;
    const int rest = n - tb;
    const int nB = (rest + hmax - 1) / hmax;
    int chunk_s[16], chunk_h[16];
    int s0 = tb;
    for (int i = 0; i < nB; ++i) {
        const int h = rest / nB + (i < rest % nB ? 1 : 0);
        chunk_s[i] = s0;
        chunk_h[i] = h;
        s0 += h;
    }
    const int G = 1 + nB;
    const int S = (G <= 1) ? p : 1 + p * (G - 1);
    if (S > max_out) return -1;
    for (int si = 0; si < S; ++si) {
        int l, pos;
        if (si < G) { l = 0; pos = si; }
        else { l = 1 + (si - G) / (G - 1); pos = 1 + (si - G) % (G - 1); }
        const int w = (l % 2 == 0) ? pos : (G - 1 - pos);
        StreamPass P{};
        P.n = n;
        P.tb = tb;
        P.la = l;
        P.lb = (pos == G - 1 && l + 1 < p) ? l + 1 : l;
        P.ph_first = (l == 0 && pos == 0) ? 1 : 0;
        P.init = (si == 0) ? 1 : 0;
        P.fin = (si == S - 1) ? 1 : 0;
        P.k = P.fin ? k : 0;
        if (w == 0) {
            P.kind = 0;
            P.c = tb; P.s = tb; P.h = 0;
        } else {
            P.kind = 1;
            P.h = chunk_h[w - 1];
            P.s = chunk_s[w - 1];
            P.c = tb - P.h;
        }
        P.need_e = (P.ph_first || P.lb > P.la || P.fin) ? 1 : 0;
        out[si] = P;
    }
    return S;
}

size_t stream_smem_bytes(bool dbl) {
    const size_t TD = (size_t)1 << stream_tile_bits(dbl);
    const size_t c = dbl ? 16 : 8, r = dbl ? 8 : 4, lcs = dbl ? sizeof(LayerConst<double>) : sizeof(LayerConst<float>);
    size_t o = TD * c + TD * r + 64 * lcs;
    o = (o + 15) & ~(size_t)15;
    return o + 32 * sizeof(double) + (8 * 32 + TOPK_CAP + 16 + 16) * sizeof(TopEnt) +
           16 * 32 * sizeof(float) + 4 * sizeof(int);
}

template <typename T>
static StreamInst<T> one_of(const void* one) {
    StreamInst<T> o{};
    if (one) o = *static_cast<const StreamInst<T>*>(one);
    return o;
}

cudaError_t launch_stream_pass(bool dbl, const StreamPass& P, const void* insts, int count,
                               int grid, cudaStream_t st, const void* one) {
    const size_t sm = stream_smem_bytes(dbl);
    cudaError_t e;
    if (dbl) {
        e = cudaFuncSetAttribute(k_stream_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_stream_pass<double><<<grid, 256, sm, st>>>(P, static_cast<const StreamInst<double>*>(insts), count, one_of<double>(one));
    } else {
        e = cudaFuncSetAttribute(k_stream_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_stream_pass<float><<<grid, 256, sm, st>>>(P, static_cast<const StreamInst<float>*>(insts), count, one_of<float>(one));
    }
    return cudaGetLastError();
}

bool stream_finalize_two_level(uint64_t ntiles, int k) { return k > 0 && ntiles > FIN_CHUNK; }

cudaError_t launch_stream_finalize(bool dbl, const void* insts, int count, uint64_t ntiles, int k,
                                   cudaStream_t st, const void* one) {
    uint64_t stride = 1;
    if (stream_finalize_two_level(ntiles, k)) {
        const dim3 grid((unsigned)((ntiles + FIN_CHUNK - 1) / FIN_CHUNK), (unsigned)count);
        if (dbl) k_stream_topk_chunks<double><<<grid, 256, 0, st>>>(static_cast<const StreamInst<double>*>(insts), count, ntiles, k, one_of<double>(one));
        else k_stream_topk_chunks<float><<<grid, 256, 0, st>>>(static_cast<const StreamInst<float>*>(insts), count, ntiles, k, one_of<float>(one));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        stride = FIN_CHUNK;
    }
    if (dbl) k_stream_finalize<double><<<count, 256, 0, st>>>(static_cast<const StreamInst<double>*>(insts), count, ntiles, k, stride, one_of<double>(one));
    else k_stream_finalize<float><<<count, 256, 0, st>>>(static_cast<const StreamInst<float>*>(insts), count, ntiles, k, stride, one_of<float>(one));
    return cudaGetLastError();
}

static int energy_split(int n) {
    // low bits fixed per thread: enough threads to fill the GPU, at most 2^12 Gray steps each
    int m = n - 6;
    if (m < 0) m = 0;
    if (m > 20) m = 20;
    if (n - m > 12) m = n - 12;
    return m;
}

// Top bits walked per thread by the row form: enough threads in total (instances x 2^(n-2-nh))
// to fill the GPU, a walk of at most 2^8 steps.
static int rows_nh(int n, int count) {
    int lc = 0;
    while ((2ull << lc) <= (unsigned long long)count) ++lc;
    int nh = n - 20 + lc;
    if (nh > ROWS_NH_MAX) nh = ROWS_NH_MAX;
    if (nh > n - 4) nh = n - 4;
    return nh < 0 ? 0 : nh;
}

template <typename T>
static cudaError_t launch_rows(int n, int count, const void* Q, void* E, const void* insts, cudaStream_t st) {
    const int nh = rows_nh(n, count);
    const uint64_t threads = 1ull << (n - nh - 2);
    const int block = threads < 256 ? (int)threads : 256;
    const unsigned gx = (unsigned)((threads + block - 1) / block);
    const StreamInst<T>* in = static_cast<const StreamInst<T>*>(insts);
    for (int c0 = 0; c0 < count; c0 += 65535) {          // grid.y limit
        const int cy = count - c0 < 65535 ? count - c0 : 65535;
        k_energy_rows<T><<<dim3(gx, (unsigned)cy), block, 0, st>>>(n, nh, static_cast<const T*>(Q),
                                                                  static_cast<T*>(E), in ? in + c0 : nullptr);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_energy(bool dbl, int n, const void* Q, void* E, cudaStream_t st) {
    if (n >= 2 && (reinterpret_cast<uintptr_t>(E) & 7u) == 0)
        return dbl ? launch_rows<double>(n, 1, Q, E, nullptr, st) : launch_rows<float>(n, 1, Q, E, nullptr, st);
    const int m = energy_split(n);
    const uint64_t threads = 1ull << m;
    const int block = threads < 256 ? (int)threads : 256;
    const uint64_t grid = (threads + block - 1) / block;
    if (dbl) k_energy<double><<<(unsigned)grid, block, 0, st>>>(n, m, static_cast<const double*>(Q), static_cast<double*>(E), nullptr);
    else k_energy<float><<<(unsigned)grid, block, 0, st>>>(n, m, static_cast<const float*>(Q), static_cast<float*>(E), nullptr);
    return cudaGetLastError();
}

cudaError_t launch_energy_batch(bool dbl, int n, const void* insts, int count, cudaStream_t st) {
    // every instance's E is at least 8-byte aligned (plan validation)
    if (n >= 2)
        return dbl ? launch_rows<double>(n, count, nullptr, nullptr, insts, st)
                   : launch_rows<float>(n, count, nullptr, nullptr, insts, st);
    const int m = energy_split(n);
    const uint64_t threads = 1ull << m;
    const int block = threads < 256 ? (int)threads : 256;
    const dim3 grid((unsigned)((threads + block - 1) / block), (unsigned)count);
    if (dbl) k_energy<double><<<grid, block, 0, st>>>(n, m, nullptr, nullptr, static_cast<const StreamInst<double>*>(insts));
    else k_energy<float><<<grid, block, 0, st>>>(n, m, nullptr, nullptr, static_cast<const StreamInst<float>*>(insts));
    return cudaGetLastError();
}

size_t stream_adj_smem_bytes(bool dbl) {
    const size_t TD = (size_t)1 << stream_adj_tile_bits(dbl);
    const size_t c = dbl ? 16 : 8, r = dbl ? 8 : 4;
    const size_t lcs = dbl ? sizeof(LayerConst<double>) : sizeof(LayerConst<float>);
    size_t o = 2 * TD * c + TD * r + 64 * lcs;
    o = (o + 15) & ~(size_t)15;
    return o + 32 * sizeof(double);
}

cudaError_t launch_stream_adj_pass(bool dbl, const StreamPass& P, int si, bool lam_first, bool store,
                                   const void* insts, int count, int grid, cudaStream_t st,
                                   const void* one) {
    const size_t sm = stream_adj_smem_bytes(dbl);
    cudaError_t e;
    if (dbl) {
        e = cudaFuncSetAttribute(k_stream_adj_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_stream_adj_pass<double><<<grid, ADJ_THREADS, sm, st>>>(P, si, lam_first, store, static_cast<const StreamInst<double>*>(insts), count, one_of<double>(one));
    } else {
        e = cudaFuncSetAttribute(k_stream_adj_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_stream_adj_pass<float><<<grid, ADJ_THREADS, sm, st>>>(P, si, lam_first, store, static_cast<const StreamInst<float>*>(insts), count, one_of<float>(one));
    }
    return cudaGetLastError();
}

cudaError_t launch_stream_grad_reduce(bool dbl, const StreamPass* passes, int S, const void* insts,
                                      int count, uint64_t ntiles, cudaStream_t st, const void* one) {
    if (S > 256) return cudaErrorInvalidValue;
    PassLayers pl;
    for (int i = 0; i < S; ++i) { pl.la[i] = passes[i].la; pl.lb[i] = passes[i].lb; }
    if (dbl) k_stream_grad_reduce<double><<<count, 256, 0, st>>>(pl, S, static_cast<const StreamInst<double>*>(insts), count, ntiles, one_of<double>(one));
    else k_stream_grad_reduce<float><<<count, 256, 0, st>>>(pl, S, static_cast<const StreamInst<float>*>(insts), count, ntiles, one_of<float>(one));
    return cudaGetLastError();
}

cudaError_t launch_reduce_state(bool dbl, int n, const void* psi, const void* E, int k,
                                double* part_expect, double* part_topp, uint32_t* part_topz,
                                double* expect, uint64_t* topk_idx, double* topk_prob,
                                cudaStream_t st) {
    const int parts = reduce_parts(n);
    if (dbl) k_reduce_state<double><<<parts, 256, 0, st>>>(n, static_cast<const double2*>(psi), static_cast<const double*>(E), k, part_expect, part_topp, part_topz);
    else k_reduce_state<float><<<parts, 256, 0, st>>>(n, static_cast<const float2*>(psi), static_cast<const float*>(E), k, part_expect, part_topp, part_topz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_finalize<<<1, 256, 0, st>>>(parts, part_expect, part_topp, part_topz, k, expect, topk_idx, topk_prob);
    return cudaGetLastError();
}

}  // namespace qaoa
