// k_tstream.cu -- TMA streaming passes of the HBM tier (complex64 states of n >= 14 qubits whose
// passes walk the whole state in HBM; Section IV, Eq. 2: cost phase and mixer per layer, <C> and
// the top-k bitstrings at the end).
//
// Each pass is one persistent launch, two CTAs per SM, walking the tiles of every instance of its
// plan group. A tile is 2^13 amplitudes, moved between HBM and shared memory by TMA
// (cp.async.bulk.tensor; the state with the 128-byte swizzle, its energies unswizzled, the
// energies only in passes with a cost phase or the final reductions). A CTA loads its next tile
// as soon as the bulk store of the current one has read the buffer, and the other CTA of the SM
// works while it waits: measured on GB300 at n = 30 this beats one CTA per SM with a two-stage
// ring (8 warps per SM leave the sub-passes latency-bound) by 12% over the passes of a solve.
//
// Tiles follow the streaming tier's pass plan (stream_plan): kind A holds qubits 0..12 (2^13
// contiguous amplitudes), kind B the 2^c contiguous amplitudes of qubits 0..c-1 times the 2^h
// values of qubits s..s+h-1 (c = 13 - h, 1 <= h <= 9). Inside a tile the qubits are mixed in
// register windows of at most five bits: kind A in [0,4), [4,8), [8,13) (the cost phase in the
// last), kind B in [c, c+h) or, for h > 5, [c, c+5) and [c+5, c+h) (the phase in the last). With
// the lanes of a warp on tile bits outside the window, the swizzle makes every shared access free
// of bank conflicts. The final pass reduces each tile to an FP64 <C> partial and a top-k list;
// the streaming tier's finalize kernel merges them per instance.
#include <cuda.h>

#include "qaoa_engine.cuh"
#include "qaoa_kernels.h"
#include "qaoa_stream.h"
#include "qaoa_tma.cuh"
#include "qaoa_tstream.h"

namespace qaoa {

namespace {

using namespace tma;

constexpr int TB = 13;
constexpr uint32_t TD = 1u << TB;
constexpr int NT = TMA_NT;
constexpr int NSTAGE = 1;

struct TsOff {
    size_t stage[NSTAGE], estage[NSTAGE], lc, red, wbound, wb, cnt, cand, out, wlists, run, mbar, total;
};
__host__ __device__ inline size_t ts_al(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline TsOff ts_offsets() {
    TsOff o{};
    size_t x = 0;
    for (int s = 0; s < NSTAGE; ++s) { o.stage[s] = x; x += (size_t)TD * 8; }   // 1024-aligned at run time
    for (int s = 0; s < NSTAGE; ++s) { o.estage[s] = x; x += (size_t)TD * 4; }
    o.lc = x; x = ts_al(x + 64 * sizeof(LayerConst<float>));
    o.red = x; x = ts_al(x + 32 * sizeof(float));
    o.wbound = x; x = ts_al(x + sizeof(float));
    o.wb = x; x = ts_al(x + 16 * (NT / 32) * sizeof(float));
    o.cnt = x; x = ts_al(x + 4 * sizeof(int));
    o.cand = x; x = ts_al(x + TOPK_CAP * sizeof(TopEnt));
    o.out = x; x = ts_al(x + 16 * sizeof(TopEnt));
    o.wlists = x; x = ts_al(x + (NT / 32) * 32 * sizeof(TopEnt));
    o.run = x; x = ts_al(x + 16 * sizeof(TopEnt));
    o.mbar = x; x = ts_al(x + NSTAGE * sizeof(uint64_t));
    o.total = x + 1024;
    return o;
}

// Geometry of one tile of a pass: global index of tile-local index u is
//   kind A: u | zt,  kind B: (u & lomask) | zt | ((u >> c) << s),
// with zt the bits that the tile index fixes.
struct Geo {
    uint32_t lomask;
    int c, s;
    uint64_t zt;
    bool kindA;
    __device__ __forceinline__ uint64_t z(uint32_t u) const {
        return kindA ? ((uint64_t)u | zt) : ((uint64_t)(u & lomask) | zt | ((uint64_t)(u >> c) << s));
    }
};

// Group g of a window [A, A+R): tile index of its element 0 (the window bits clear).
template <int A, int R>
__device__ __forceinline__ uint32_t wbase(uint32_t g) {
    return (g & ((1u << A) - 1u)) | ((g >> A) << (A + R));
}
// Shared index of element i of a group whose base has shared index pb (the swizzle is linear
// over GF(2); for A >= 7 the window bits lie above the swizzled bits and the XOR is an add).
template <int A>
__device__ __forceinline__ uint32_t wix(uint32_t pb, int i) {
    if constexpr (A >= 7) return pb + ((uint32_t)i << A);
    else return pb ^ psw((uint32_t)i << A);
}

template <int A, int R>
__device__ __forceinline__ void wload(const float2* sp, uint32_t pb, float2 (&v)[1 << R]) {
    if constexpr (A == 0 && R >= 1) {
#pragma unroll
        for (int j = 0; j < (1 << R); j += 2) {
            const float4 q = *reinterpret_cast<const float4*>(sp + (pb ^ (uint32_t)j));
            v[j] = make_float2(q.x, q.y);
            v[j + 1] = make_float2(q.z, q.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) v[i] = sp[wix<A>(pb, i)];
    }
}
template <int A, int R>
__device__ __forceinline__ void wstore(float2* sp, uint32_t pb, const float2 (&v)[1 << R]) {
    if constexpr (A == 0 && R >= 1) {
#pragma unroll
        for (int j = 0; j < (1 << R); j += 2)
            *reinterpret_cast<float4*>(sp + (pb ^ (uint32_t)j)) = make_float4(v[j].x, v[j].y, v[j + 1].x, v[j + 1].y);
    } else {
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) sp[wix<A>(pb, i)] = v[i];
    }
}

// What one sub-pass does to a group, in order: the mixer of layer la; then, with `phase`, the
// cost phase of layer lb and its mixer; with `init`, the group starts as |+> (rotated frame)
// followed by the cost phase of layer 0 and its mixer (la, phase unused); with `fin`, the
// pending shear factor of the last layer and the thread's FP32 <C> terms and maximum |psi|^2.
struct SubOps {
    int la, lb;
    bool mix_la, phase, init, fin;
};

// One sub-pass over window [A, A+R) of the tile in sp: every group of the thread (2^(13-R) /
// 256 of them) is loaded, transformed and stored. zsh: shift of the window's bit 0 in the global
// index (kind A: A; kind B: A - c + s).
// The work of one group of window [A, A+R) (see wsub).
template <int A, int R>
__device__ __forceinline__ void wgroup(float2* sp, uint32_t g, const Geo& geo, const SubOps& op,
                                       const LayerConst<float>* lc, const float* sE, float amp0, float& accp,
                                       float& pmax) {
    const uint32_t base = wbase<A, R>(g);
    const uint32_t pb = psw(base);
    float2 v[1 << R];
    if (op.init) {
        const int pc = __popcll(geo.z(base));
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) {
            float s, c;
            sincos_phase(lc[0].gpi, sE[base + ((uint32_t)i << A)], s, c);
            v[i] = times_i_pow(make_float2(amp0 * c, -amp0 * s), pc + __popc(i));
        }
        mix_layer<R>(v, (1 << R) - 1, lc[0]);
    } else {
        wload<A, R>(sp, pb, v);
        if (op.mix_la) mix_layer<R>(v, (1 << R) - 1, lc[op.la]);
        if (op.phase) {
            const LayerConst<float>& k = lc[op.lb];
#pragma unroll
            for (int i = 0; i < (1 << R); ++i) {
                float s, c;
                sincos_phase(k.gpi, sE[base + ((uint32_t)i << A)], s, c);
                rot_neg(v[i], s * k.pre, c * k.pre);
            }
            mix_layer<R>(v, (1 << R) - 1, k);
        }
        if (op.fin) {
            if (lc[op.la].shear) scale_group<R>(v, lc[op.la].post);
#pragma unroll
            for (int i = 0; i < (1 << R); ++i) {
                const float pr = v[i].x * v[i].x + v[i].y * v[i].y;
                accp = fmaf(pr, sE[base + ((uint32_t)i << A)], accp);
                pmax = fmaxf(pmax, pr);
            }
        }
    }
    wstore<A, R>(sp, pb, v);
}

// One sub-pass over window [A, A+R) of the tile in sp: every group of the thread (2^(13-R) /
// 256 of them) is loaded, transformed and stored.
template <int A, int R>
__device__ __forceinline__ void wsub(float2* sp, const Geo& geo, int zsh, const SubOps& op,
                                     const LayerConst<float>* lc, const float* sE, float amp0,
                                     float& accp, float& pmax) {
    constexpr int NGT = (1 << (TB - R)) / NT;   // groups per thread
#pragma unroll 1
    for (int r = 0; r < NGT; ++r) wgroup<A, R>(sp, threadIdx.x + (uint32_t)(r * NT), geo, op, lc, sE, amp0, accp, pmax);
}

// Element i < 32 of the thread in the last sub-pass over window [A, A+R): shared and global index.
template <int A, int R>
__device__ __forceinline__ void welem(const Geo& geo, int zsh, int i, uint32_t& ix, uint64_t& z) {
    const uint32_t g = threadIdx.x + (uint32_t)((i >> R) * NT);
    const int e = i & ((1 << R) - 1);
    const uint32_t base = wbase<A, R>(g);
    ix = wix<A>(psw(base), e);
    z = geo.z(base) + ((uint64_t)e << zsh);
}

// Kind-A tile: the snake of the pass over the windows [0,4), [4,8), [8,13).
__device__ __forceinline__ void tile_kind_a(float2* sp, const Geo& geo, const StreamPass& P,
                                            const LayerConst<float>* lc, const float* sE, float amp0,
                                            float& accp, float& pmax) {
    if (P.init) {
        // |+>, the cost phase and the mixer of layer 0 (the pass opens the state), then the mixer
        // of layer 0 on the lower windows; a pass that also closes the layer is not planned
        wsub<8, 5>(sp, geo, 8, SubOps{0, 0, false, false, true, false}, lc, sE, amp0, accp, pmax);
        __syncthreads();
        wsub<4, 4>(sp, geo, 4, SubOps{0, 0, true, false, false, false}, lc, sE, amp0, accp, pmax);
        __syncthreads();
        wsub<0, 4>(sp, geo, 0, SubOps{0, 0, true, false, false, false}, lc, sE, amp0, accp, pmax);
        return;
    }
    const bool two = P.lb > P.la;
    wsub<0, 4>(sp, geo, 0, SubOps{P.la, P.la, true, false, false, false}, lc, sE, amp0, accp, pmax);
    __syncthreads();
    wsub<4, 4>(sp, geo, 4, SubOps{P.la, P.la, true, false, false, false}, lc, sE, amp0, accp, pmax);
    __syncthreads();
    wsub<8, 5>(sp, geo, 8, SubOps{P.la, P.lb, true, two, false, (bool)P.fin}, lc, sE, amp0, accp, pmax);
    if (two) {
        __syncthreads();
        wsub<4, 4>(sp, geo, 4, SubOps{P.lb, P.lb, true, false, false, false}, lc, sE, amp0, accp, pmax);
        __syncthreads();
        wsub<0, 4>(sp, geo, 0, SubOps{P.lb, P.lb, true, false, false, false}, lc, sE, amp0, accp, pmax);
    }
}

// Kind-B tile with H high qubits: one window [c, c+H) for H <= 5, else [c, c+5) and [c+5, c+H).
template <int H>
__device__ __forceinline__ void tile_kind_b(float2* sp, const Geo& geo, const StreamPass& P,
                                            const LayerConst<float>* lc, const float* sE, float amp0,
                                            float& accp, float& pmax) {
    constexpr int C = TB - H;
    const bool two = P.lb > P.la;
    if constexpr (H <= 5) {
        wsub<C, H>(sp, geo, P.s, SubOps{P.la, P.lb, true, two, false, (bool)P.fin}, lc, sE, amp0, accp, pmax);
    } else {
        constexpr int A2 = C + 5, R2 = H - 5;
        wsub<C, 5>(sp, geo, P.s, SubOps{P.la, P.la, true, false, false, false}, lc, sE, amp0, accp, pmax);
        __syncthreads();
        wsub<A2, R2>(sp, geo, P.s + 5, SubOps{P.la, P.lb, true, two, false, (bool)P.fin}, lc, sE, amp0, accp, pmax);
        if (two) {
            __syncthreads();
            wsub<C, 5>(sp, geo, P.s, SubOps{P.lb, P.lb, true, false, false, false}, lc, sE, amp0, accp, pmax);
        }
    }
}

// Element accessor of the thread's 32 elements in the pass's last sub-pass (reductions).
template <int H>
__device__ __forceinline__ void last_elem_b(const Geo& geo, const StreamPass& P, int i, uint32_t& ix, uint64_t& z) {
    constexpr int C = TB - H;
    if constexpr (H <= 5) welem<C, H>(geo, P.s, i, ix, z);
    else welem<C + 5, H - 5>(geo, P.s + 5, i, ix, z);
}

__device__ __forceinline__ void kind_b_dispatch(int h, float2* sp, const Geo& geo, const StreamPass& P,
                                                const LayerConst<float>* lc, const float* sE, float amp0,
                                                float& accp, float& pmax) {
    switch (h) {
        case 1: tile_kind_b<1>(sp, geo, P, lc, sE, amp0, accp, pmax); break;
        case 2: tile_kind_b<2>(sp, geo, P, lc, sE, amp0, accp, pmax); break;
        case 3: tile_kind_b<3>(sp, geo, P, lc, sE, amp0, accp, pmax); break;
        case 4: tile_kind_b<4>(sp, geo, P, lc, sE, amp0, accp, pmax); break;
        case 5: tile_kind_b<5>(sp, geo, P, lc, sE, amp0, accp, pmax); break;
        case 6: tile_kind_b<6>(sp, geo, P, lc, sE, amp0, accp, pmax); break;
        case 7: tile_kind_b<7>(sp, geo, P, lc, sE, amp0, accp, pmax); break;
        case 8: tile_kind_b<8>(sp, geo, P, lc, sE, amp0, accp, pmax); break;
        default: tile_kind_b<9>(sp, geo, P, lc, sE, amp0, accp, pmax); break;
    }
}

__device__ __forceinline__ void last_elem(const Geo& geo, const StreamPass& P, int i, uint32_t& ix, uint64_t& z) {
    if (P.kind == 0) {
        welem<8, 5>(geo, 8, i, ix, z);
        return;
    }
    switch (P.h) {
        case 1: last_elem_b<1>(geo, P, i, ix, z); break;
        case 2: last_elem_b<2>(geo, P, i, ix, z); break;
        case 3: last_elem_b<3>(geo, P, i, ix, z); break;
        case 4: last_elem_b<4>(geo, P, i, ix, z); break;
        case 5: last_elem_b<5>(geo, P, i, ix, z); break;
        case 6: last_elem_b<6>(geo, P, i, ix, z); break;
        case 7: last_elem_b<7>(geo, P, i, ix, z); break;
        case 8: last_elem_b<8>(geo, P, i, ix, z); break;
        default: last_elem_b<9>(geo, P, i, ix, z); break;
    }
}

// TMA coordinates of tile tau (TsPass::bmode, see qaoa_tstream.h); the energy maps have the same
// coordinates as the state maps.
__device__ __forceinline__ void tile_load(const TsPass& T, const CUtensorMap* map, void* dst, uint64_t tau,
                                          uint64_t* bar) {
    const int mid = (int)(tau & ((1ull << T.midbits) - 1ull)), top = (int)(tau >> T.midbits);
    switch (T.bmode) {
        case TS_A: tma_load_4d(dst, map, 0, 0, 0, (int)tau, bar); break;
        case TS_A3: tma_load_3d(dst, map, 0, 0, (int)tau, bar); break;
        case TS_B5: tma_load_5d(dst, map, 0, 0, mid, 0, top, bar); break;
        case TS_B4: tma_load_4d(dst, map, 0, 0, mid, 0, bar); break;
        case TS_B9_5: tma_load_5d(dst, map, 0, mid, 0, 0, top, bar); break;
        default: tma_load_4d(dst, map, 0, mid, 0, 0, bar); break;
    }
}
// L2 prefetch of the tile tile_load would copy (a cache hint only)
__device__ __forceinline__ void tile_prefetch(const TsPass& T, const CUtensorMap* map, uint64_t tau) {
    const int mid = (int)(tau & ((1ull << T.midbits) - 1ull)), top = (int)(tau >> T.midbits);
    switch (T.bmode) {
        case TS_A: tma_prefetch_4d(map, 0, 0, 0, (int)tau); break;
        case TS_A3: tma_prefetch_3d(map, 0, 0, (int)tau); break;
        case TS_B5: tma_prefetch_5d(map, 0, 0, mid, 0, top); break;
        case TS_B4: tma_prefetch_4d(map, 0, 0, mid, 0); break;
        case TS_B9_5: tma_prefetch_5d(map, 0, mid, 0, 0, top); break;
        default: tma_prefetch_4d(map, 0, mid, 0, 0); break;
    }
}
__device__ __forceinline__ void tile_store(const TsPass& T, const CUtensorMap* map, const void* src, uint64_t tau) {
    const int mid = (int)(tau & ((1ull << T.midbits) - 1ull)), top = (int)(tau >> T.midbits);
    switch (T.bmode) {
        case TS_A: tma_store_4d(map, src, 0, 0, 0, (int)tau); break;
        case TS_A3: tma_store_3d(map, src, 0, 0, (int)tau); break;
        case TS_B5: tma_store_5d(map, src, 0, 0, mid, 0, top); break;
        case TS_B4: tma_store_4d(map, src, 0, 0, mid, 0); break;
        case TS_B9_5: tma_store_5d(map, src, 0, mid, 0, 0, top); break;
        default: tma_store_4d(map, src, 0, mid, 0, 0); break;
    }
}

__global__ void __launch_bounds__(NT, 2) k_tstream_pass(const StreamPass P, const TsPass T,
                                                       const StreamInst<float>* __restrict__ insts, int count,
                                                       const CUtensorMap* __restrict__ maps, unsigned* status) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const uint32_t raw = saddr(sm_raw);
    unsigned char* sm = sm_raw + (((raw + 1023u) & ~1023u) - raw);
    const TsOff o = ts_offsets();
    // stage s at stage0 + s * TD (state) and estage0 + s * TD (energies): no arrays, so that no
    // dynamic index sends them to local memory
    float2* const stage0 = reinterpret_cast<float2*>(sm + o.stage[0]);
    float* const estage0 = reinterpret_cast<float*>(sm + o.estage[0]);
    LayerConst<float>* lc = reinterpret_cast<LayerConst<float>*>(sm + o.lc);
    float* red = reinterpret_cast<float*>(sm + o.red);
    TileTopk ts;
    ts.wb = reinterpret_cast<float*>(sm + o.wb);
    ts.cnt = reinterpret_cast<int*>(sm + o.cnt);
    ts.cand = reinterpret_cast<TopEnt*>(sm + o.cand);
    ts.out = reinterpret_cast<TopEnt*>(sm + o.out);
    ts.wlists = reinterpret_cast<TopEnt*>(sm + o.wlists);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + o.mbar);
    if (threadIdx.x == 0)
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&mbar[s], 1);
    __syncthreads();

    const uint64_t ntiles = 1ull << (P.n - TB);
    const uint64_t total = ntiles * (uint64_t)count;
    const uint64_t first = blockIdx.x, step = gridDim.x;
    const int nmine = first < total ? (int)((total - 1 - first) / step + 1) : 0;
    const bool loads = !P.init || P.need_e;   // the init pass loads only the energies
    const bool store = !P.fin || !P.no_store;
    const bool pf = P.init || !store;
    uint32_t parity = 0;   // bit s: parity of the next wait on stage s
    bool ok = true;
    // the energies first (their buffer is never stored from), then, once the last tile's store
    // has read the state buffer (wait_store), the state
    auto issue = [&](int k, bool wait_store) {
        const uint64_t q = first + (uint64_t)k * step;
        const int ii = (int)(q / ntiles);
        const uint64_t tau = q % ntiles;
        const int s = k % NSTAGE;
        const CUtensorMap* m = maps + (size_t)ii * T.maps_per_inst;
        mbar_expect_tx(&mbar[s], (P.init ? 0u : TD * 8) + (P.need_e ? TD * 4 : 0u));
        if (P.need_e) tile_load(T, m + T.emap, estage0 + (size_t)s * TD, tau, &mbar[s]);
        if (!P.init) {
            if (wait_store) bulk_wait_read();
            tile_load(T, m + T.map, stage0 + (size_t)s * TD, tau, &mbar[s]);
        }
        // the tile after it towards L2, a tile's compute ahead of its own load (in the passes
        // that store no state: with the state stores in flight it slowed the others down)
        if (pf && k + 1 < nmine) {
            const uint64_t q1 = q + step;
            const CUtensorMap* m1 = maps + (size_t)(q1 / ntiles) * T.maps_per_inst;
            if (P.need_e) tile_prefetch(T, m1 + T.emap, q1 % ntiles);
            if (!P.init) tile_prefetch(T, m1 + T.map, q1 % ntiles);
        }
    };
    if (loads && nmine > 0 && threadIdx.x == 0) issue(0, false);
    const float *cur_g = nullptr, *cur_b = nullptr;
    int cur_p = 0;
    TopEnt* run = reinterpret_cast<TopEnt*>(sm + o.run);
    bool run_valid = false;   // the run list holds this CTA's best k of the current instance so far
    for (int k = 0; k < nmine; ++k) {
        const uint64_t q = first + (uint64_t)k * step;
        const int ii = (int)(q / ntiles);
        const uint64_t tau = q % ntiles;
        const int s = k % NSTAGE;
        const StreamInst<float>& I = insts[ii];
        if (I.gamma != cur_g || I.beta != cur_b || I.p != cur_p) {
            __syncthreads();
            set_layer_consts<float>(lc, I.gamma, I.beta, I.p, P.n, true);
            cur_g = I.gamma;
            cur_b = I.beta;
            cur_p = I.p;
        }
        if (loads) {
            if (ok) ok = mbar_wait_bounded(&mbar[s], (parity >> s) & 1u);
            parity ^= 1u << s;
            // the init pass loads only the energies, issued before the last tile's store had read
            // the state buffer: that read must be over before this tile writes the buffer
            if (P.init && k >= 1 && threadIdx.x == 0) bulk_wait_read();
        } else if (k >= 1 && threadIdx.x == 0) {
            bulk_wait_read();   // the buffer's earlier store has read it
        }
        ok = __syncthreads_and(ok);
        Geo geo;
        geo.kindA = P.kind == 0;
        geo.c = P.c;
        geo.s = P.s;
        geo.lomask = (1u << P.c) - 1u;
        if (geo.kindA) {
            geo.zt = tau << TB;
        } else {
            const int midbits = P.s - P.c;
            const uint64_t mid = tau & ((1ull << midbits) - 1ull), top = tau >> midbits;
            geo.zt = (mid << P.c) | (top << (P.s + P.h));
        }
        float2* sp = stage0 + (size_t)s * TD;
        const float* sE = estage0 + (size_t)s * TD;
        float accp = 0.0f, pmax = -1.0f;
        if (geo.kindA) tile_kind_a(sp, geo, P, lc, sE, (float)I.amp0, accp, pmax);
        else kind_b_dispatch(P.h, sp, geo, P, lc, sE, (float)I.amp0, accp, pmax);
        __syncthreads();
        if (P.fin) {
            const double tot = block_sum_df(accp, red);
            if (threadIdx.x == 0) I.part_expect[tau] = tot;
            if (P.k > 0) {
                // Top-k: the CTA carries one list (run) across its tiles of an instance and writes
                // it into the slot of its last such tile (the other slots it owns stay empty); the
                // list of an instance is unique, so this does not depend on which tiles a CTA gets.
                const auto elem = [&geo, &P](int i, uint32_t& ix, uint32_t& z) {
                    uint64_t zz;
                    last_elem(geo, P, i, ix, zz);
                    z = (uint32_t)zz;
                };
                const int kk = P.k;
                const auto full_tile = [&]() {   // the tile's own list into ts.out
                    if (!topk_own(sp, kk, pmax, elem, ts, reinterpret_cast<float*>(sm + o.wbound))) {
                        float pm2 = -1.0f;
                        for (uint32_t u = threadIdx.x; u < TD; u += NT) {
                            const float2 v = sp[psw(u)];
                            pm2 = fmaxf(pm2, v.x * v.x + v.y * v.y);
                        }
                        const TileRef<float> tile{sp, nullptr, nullptr, TB};
                        const auto zmap = [&geo](uint32_t u) { return (uint32_t)geo.z(u); };
                        tile_topk<float, TmaLayout>(tile, kk, pm2, zmap, ts);
                    }
                };
                // the k best of `na` entries a[] and the run list, into run (rank selection)
                const auto merge_run = [&](const TopEnt* a, int na) {
                    TopEnt* merged = ts.wlists;
                    for (int c = threadIdx.x; c < na + kk; c += NT) {
                        const TopEnt me = c < na ? a[c] : run[c - na];
                        int rank = 0;
                        for (int j2 = 0; j2 < na; ++j2) rank += better(a[j2].p, a[j2].z, me.p, me.z) ? 1 : 0;
                        for (int j2 = 0; j2 < kk; ++j2) rank += better(run[j2].p, run[j2].z, me.p, me.z) ? 1 : 0;
                        if (rank < kk) merged[rank] = me;
                    }
                    __syncthreads();
                    if (threadIdx.x < (unsigned)kk) run[threadIdx.x] = merged[threadIdx.x];
                    __syncthreads();
                };
                if (!run_valid) {
                    full_tile();
                    if (threadIdx.x < (unsigned)kk) run[threadIdx.x] = ts.out[threadIdx.x];
                    __syncthreads();
                    run_valid = true;
                } else {
                    const float lo = __double2float_rd(run[kk - 1].p) * 0.99999904632568359375f;   // (1 - 2^-20)
                    if (threadIdx.x == 0) { ts.cnt[0] = 0; ts.cnt[1] = 0; }
                    if (__syncthreads_or(pmax * 1.000003814697265625f >= lo)) {
                        if (pmax * 1.000003814697265625f >= lo) {
                            for (int i = 0; i < 32; ++i) {
                                uint32_t ix, z;
                                elem(i, ix, z);
                                const float2 v = sp[ix];
                                if ((v.x * v.x + v.y * v.y) * 1.00000095367431640625f >= lo) {
                                    const int pos = atomicAdd(&ts.cnt[0], 1);
                                    if (pos < TOPK_CAP) {
                                        ts.cand[pos].p = __hiloint2double(__float_as_int(v.y), __float_as_int(v.x));
                                        ts.cand[pos].z = z;
                                    } else {
                                        ts.cnt[1] = 1;
                                    }
                                }
                            }
                        }
                        __syncthreads();
                        if (!ts.cnt[1]) {
                            const int cnt = ts.cnt[0];
                            for (int c = threadIdx.x; c < cnt; c += NT) {
                                const double raw = ts.cand[c].p;
                                ts.cand[c].p = exact_prob(make_float2(__int_as_float(__double2loint(raw)),
                                                                      __int_as_float(__double2hiint(raw))));
                            }
                            __syncthreads();
                            merge_run(ts.cand, cnt);
                        } else {
                            __syncthreads();   // every thread has read the overflow flag
                            full_tile();
                            merge_run(ts.out, kk);
                        }
                    }
                }
                // this tile's slot: the list when it is the CTA's last tile of the instance
                const uint64_t qn = q + step;
                const bool last_of_inst = k + 1 >= nmine || (int)(qn / ntiles) != ii;
                if (threadIdx.x < (unsigned)kk) {
                    const TopEnt e = last_of_inst ? run[threadIdx.x] : TopEnt{-1.0, 0xffffffffu};
                    I.part_topp[tau * kk + threadIdx.x] = e.p;
                    I.part_topz[tau * kk + threadIdx.x] = e.z;
                }
                if (last_of_inst) run_valid = false;
            }
            if (store && !P.keep_frame) {
                // the state leaves in the standard frame: psi = (-i)^{|z|} psi~
                __syncthreads();
                for (uint32_t u = threadIdx.x; u < TD; u += NT)
                    sp[psw(u)] = times_i_pow(sp[psw(u)], -__popcll(geo.z(u)));
            }
        }
        if (store) {
            fence_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) {
                tile_store(T, maps + (size_t)ii * T.maps_per_inst + T.map, sp, tau);
                bulk_commit();
            }
        } else {
            fence_async_smem();   // the sub-passes' shared writes before the next tile's TMA writes
            __syncthreads();
        }
        // the next tile's loads: the energies at once, the state once this tile's store has read
        // the buffer (the init pass loads only the energies)
        if (loads && k + 1 < nmine && threadIdx.x == 0 && ok) issue(k + 1, true);
    }
    if (threadIdx.x == 0) {
        bulk_wait_all();
        if (!ok) atomicOr(status, 1u);
    }
}

// ---- adjoint passes ---------------------------------------------------------------------------
// The forward pass P undone on 2^12-amplitude tiles of psi and lam (both in the rotated frame),
// with the adjoint sub-passes of the tile engine on the TMA layout (amplitudes in the 128-byte
// swizzle, energies unswizzled): the local snake of P run in reverse, a single layer that opens
// with its cost phase ordered so that the phase (an energy read) shares the top window, where
// the lanes of a warp cover the low tile bits. Per tile the four FP64 gradient partials of the
// cp.async adjoint ([0] Im <lam|B|psi> of layer lb, [1] of la, [2] Im <lam|E|psi> of lb, [3] of
// la) are written; psi and lam go back by TMA unless this is the last adjoint pass. Persistent,
// two CTAs per SM (psi, lam and energies of a tile: 80 KiB), a CTA's next tile loaded once the
// bulk stores of the current one have read the buffers.
constexpr uint32_t TDA = 1u << TSA_TB;

struct TaOff {
    size_t psi, lam, E, lc, red, mbar, total;
};
__host__ __device__ inline TaOff ta_offsets() {
    TaOff o{};
    size_t x = 0;
    o.psi = x; x += (size_t)TDA * 8;   // 1024-aligned at run time (swizzled)
    o.lam = x; x += (size_t)TDA * 8;   // 32 KiB further: still 1024-aligned
    o.E = x; x += (size_t)TDA * 4;
    o.lc = x; x = ts_al(x + 64 * sizeof(LayerConst<float>));
    o.red = x; x = ts_al(x + 32 * sizeof(double));
    o.mbar = x; x = ts_al(x + sizeof(uint64_t));
    o.total = x + 1024;
    return o;
}

__global__ void __launch_bounds__(NT, 2) k_tstream_adj_pass(const StreamPass P, const TsPass T, int si,
                                                           int lam_first, int store,
                                                           const StreamInst<float>* __restrict__ insts, int count,
                                                           const CUtensorMap* __restrict__ maps, unsigned* status) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const uint32_t raw = saddr(sm_raw);
    unsigned char* sm = sm_raw + (((raw + 1023u) & ~1023u) - raw);
    const TaOff o = ta_offsets();
    float2* spsi = reinterpret_cast<float2*>(sm + o.psi);
    float2* slam = reinterpret_cast<float2*>(sm + o.lam);
    float* sE = reinterpret_cast<float*>(sm + o.E);
    LayerConst<float>* lc = reinterpret_cast<LayerConst<float>*>(sm + o.lc);
    double* red = reinterpret_cast<double*>(sm + o.red);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + o.mbar);
    if (threadIdx.x == 0) mbar_init(mbar, 1);
    __syncthreads();

    constexpr int RA = Num<float>::RB_ADJ;
    const uint64_t ntiles = 1ull << (P.n - TSA_TB);
    const uint64_t total = ntiles * (uint64_t)count;
    const uint64_t first = blockIdx.x, step = gridDim.x;
    const int nmine = first < total ? (int)((total - 1 - first) / step + 1) : 0;
    const bool need_e = lam_first || P.ph_first || P.lb > P.la;
    uint32_t parity = 0;
    bool ok = true;
    // the energies first (never stored from), then, once the last tile's stores have read the
    // state buffers (wait_store), psi and lam
    auto issue = [&](int k, bool wait_store) {
        const uint64_t q = first + (uint64_t)k * step;
        const int ii = (int)(q / ntiles);
        const uint64_t tau = q % ntiles;
        const CUtensorMap* m = maps + (size_t)ii * T.maps_per_inst;
        mbar_expect_tx(mbar, TDA * 8 + (lam_first ? 0u : TDA * 8) + (need_e ? TDA * 4 : 0u));
        if (need_e) tile_load(T, m + T.emap, sE, tau, mbar);
        if (wait_store) bulk_wait_read();
        tile_load(T, m + T.map, spsi, tau, mbar);
        if (!lam_first) tile_load(T, m + T.map + 1, slam, tau, mbar);
        // the tile after it towards L2, a tile's compute ahead of its own loads
        if (k + 1 < nmine) {
            const uint64_t q1 = q + step;
            const CUtensorMap* m1 = maps + (size_t)(q1 / ntiles) * T.maps_per_inst;
            if (need_e) tile_prefetch(T, m1 + T.emap, q1 % ntiles);
            tile_prefetch(T, m1 + T.map, q1 % ntiles);
            if (!lam_first) tile_prefetch(T, m1 + T.map + 1, q1 % ntiles);
        }
    };
    if (nmine > 0 && threadIdx.x == 0) issue(0, false);
    const float *cur_g = nullptr, *cur_b = nullptr;
    int cur_p = 0;
    const TileRef<float> tile{spsi, slam, sE, TSA_TB};
    const int m0 = (P.kind == 0) ? 0 : P.c;
    const int G = num_windows(m0, TSA_TB, RA);
    const int nl = P.lb - P.la + 1;
    const int S = snake_len(G, nl);
    for (int k = 0; k < nmine; ++k) {
        const uint64_t q = first + (uint64_t)k * step;
        const int ii = (int)(q / ntiles);
        const uint64_t tau = q % ntiles;
        const StreamInst<float>& I = insts[ii];
        if (I.gamma != cur_g || I.beta != cur_b || I.p != cur_p) {
            __syncthreads();
            set_layer_consts<float>(lc, I.gamma, I.beta, I.p, P.n, false);
            cur_g = I.gamma;
            cur_b = I.beta;
            cur_p = I.p;
        }
        if (ok) ok = mbar_wait_bounded(mbar, parity);
        parity ^= 1u;
        float ab[2] = {0.0f, 0.0f}, ag[2] = {0.0f, 0.0f};
        for (int kk = S - 1; kk >= 0; --kk) {
            SubPass sp;
            snake_step(kk, G, nl, P.la, P.ph_first, m0, TSA_TB, TSA_TB, RA, sp, true);
            float lb_[2] = {0.0f, 0.0f}, lg_[2] = {0.0f, 0.0f};
            subpass_adj<float, RA, TmaLayout>(tile, sp, lc, lam_first && kk == S - 1, lb_, lg_);
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
        double* out = I.part_grad + ((uint64_t)si << (P.n - TSA_TB)) * 4 + tau * 4;
        const double v0 = block_sum((double)ab[0], red);
        const double v1 = block_sum((double)ab[1], red);
        const double v2 = block_sum((double)ag[0], red);
        const double v3 = block_sum((double)ag[1], red);
        if (threadIdx.x == 0) { out[0] = v0; out[1] = v1; out[2] = v2; out[3] = v3; }
        if (store) {
            fence_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) {
                const CUtensorMap* m = maps + (size_t)ii * T.maps_per_inst;
                tile_store(T, m + T.map, spsi, tau);
                tile_store(T, m + T.map + 1, slam, tau);
                bulk_commit();
            }
        } else {
            fence_async_smem();   // the sub-passes' shared writes before the next tile's TMA writes
            __syncthreads();
        }
        // the next tile's loads: the energies at once, psi and lam once this tile's stores have
        // read the buffers
        if (k + 1 < nmine && threadIdx.x == 0 && ok) issue(k + 1, true);
    }
    if (threadIdx.x == 0) {
        bulk_wait_all();
        if (!ok) atomicOr(status, 1u);
    }
}

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
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, base, dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE,
                       swz128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The map of one pass shape over an array of 2^n elements of `w` floats each (w = 2: the
// complex64 state, swizzled; w = 1: the energies, unswizzled). The innermost dimension is the 16
// elements of tile bits 0..3 (16 w floats); the others follow TsPass::bmode.
bool encode_shape(const StreamPass& P, void* base, int w, CUtensorMap* m) {
    const int n = P.n;
    const cuuint64_t f = (cuuint64_t)w * 4;            // bytes per element
    const cuuint32_t d0 = 16u * (cuuint32_t)w;
    const bool swz = w == 2;
    if (P.kind == 0 && P.tb == TSA_TB) {   // (16 elements, 256 lines, tile): the adjoint's tiles
        const cuuint64_t d[3] = {d0, 256, 1ull << (n - TSA_TB)};
        const cuuint64_t s[2] = {16 * f, 4096 * f};
        const cuuint32_t b[3] = {d0, 256, 1};
        return encode(m, base, 3, d, s, b, swz);
    }
    if (P.kind == 0) {   // (16 elements, 256 lines, 2 planes, tile)
        const cuuint64_t d[4] = {d0, 256, 2, 1ull << (n - TB)};
        const cuuint64_t s[3] = {16 * f, 4096 * f, 8192 * f};
        const cuuint32_t b[4] = {d0, 256, 2, 1};
        return encode(m, base, 4, d, s, b, swz);
    }
    const int c = P.c, sh = P.s, h = P.h;
    const bool top = sh + h < n;
    const cuuint64_t topd = 1ull << (n - sh - h);
    if (h <= 8) {   // (16 elements, lines of bits 4..c-1, tile bits c..s-1, hi bits s..s+h-1[, top])
        const cuuint64_t d[5] = {d0, 1ull << (c - 4), 1ull << (sh - c), 1ull << h, topd};
        const cuuint64_t s[4] = {16 * f, (1ull << c) * f, (1ull << sh) * f, (1ull << (sh + h)) * f};
        const cuuint32_t b[5] = {d0, 1u << (c - 4), 1, 1u << h, 1};
        return encode(m, base, top ? 5 : 4, d, s, b, swz);
    }
    // h = 9, c = 4: (16 elements, tile bits 4..s-1, hi bits s..s+7, hi bit s+8[, top])
    const cuuint64_t d[5] = {d0, 1ull << (sh - c), 256, 2, topd};
    const cuuint64_t s[4] = {16 * f, (1ull << sh) * f, (1ull << (sh + 8)) * f, (1ull << (sh + 9)) * f};
    const cuuint32_t b[5] = {d0, 1, 256, 2, 1};
    return encode(m, base, top ? 5 : 4, d, s, b, swz);
}

}  // namespace

bool tstream_available() { return encode_fn() != nullptr; }

size_t tstream_smem_bytes() { return ts_offsets().total; }

TsPass tstream_pass_geometry(const StreamPass& P, int map, int emap, int maps_per_inst) {
    TsPass T{};
    T.map = map;
    T.emap = emap;
    T.maps_per_inst = maps_per_inst;
    if (P.kind == 0) {
        T.bmode = TS_A;
        T.midbits = 0;
        return T;
    }
    T.midbits = P.s - P.c;
    const bool top = P.s + P.h < P.n;
    if (P.h <= 8) T.bmode = top ? TS_B5 : TS_B4;
    else T.bmode = top ? TS_B9_5 : TS_B9_4;
    return T;
}

bool tstream_encode_maps(const StreamPass& P, void* psi, void* E, void* psi_map, void* e_map) {
    if (!encode_fn() || P.tb != TB || P.n <= TB || P.n > 34) return false;
    return encode_shape(P, psi, 2, static_cast<CUtensorMap*>(psi_map)) &&
           encode_shape(P, E, 1, static_cast<CUtensorMap*>(e_map));
}

cudaError_t launch_tstream_pass(const StreamPass& P, const TsPass& T, const void* insts, int count,
                                const void* maps, int grid, unsigned* status, cudaStream_t st) {
    const size_t sm = tstream_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_tstream_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_tstream_pass<<<grid, NT, sm, st>>>(P, T, static_cast<const StreamInst<float>*>(insts), count,
                                         static_cast<const CUtensorMap*>(maps), status);
    return cudaGetLastError();
}

size_t tstream_adj_smem_bytes() { return ta_offsets().total; }

TsPass tstream_adj_geometry(const StreamPass& P, int map, int maps_per_inst) {
    TsPass T{};
    T.map = map;
    T.emap = map + 2;
    T.maps_per_inst = maps_per_inst;
    if (P.kind == 0) {
        T.bmode = TS_A3;
        T.midbits = 0;
        return T;
    }
    T.midbits = P.s - P.c;
    T.bmode = (P.s + P.h < P.n) ? TS_B5 : TS_B4;
    return T;
}

bool tstream_encode_adj_maps(const StreamPass& P, void* psi, void* lam, void* E, void* maps3) {
    if (!encode_fn() || P.tb != TSA_TB || P.n <= TSA_TB || P.n > 34 || (P.kind == 1 && (P.h > 8 || P.c < 4)))
        return false;
    char* b = static_cast<char*>(maps3);
    return encode_shape(P, psi, 2, reinterpret_cast<CUtensorMap*>(b)) &&
           encode_shape(P, lam, 2, reinterpret_cast<CUtensorMap*>(b + TS_MAP_BYTES)) &&
           encode_shape(P, E, 1, reinterpret_cast<CUtensorMap*>(b + 2 * TS_MAP_BYTES));
}

cudaError_t launch_tstream_adj_pass(const StreamPass& P, const TsPass& T, int si, bool lam_first, bool store,
                                    const void* insts, int count, const void* maps, int grid, unsigned* status,
                                    cudaStream_t st) {
    const size_t sm = tstream_adj_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_tstream_adj_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_tstream_adj_pass<<<grid, NT, sm, st>>>(P, T, si, lam_first ? 1 : 0, store ? 1 : 0,
                                             static_cast<const StreamInst<float>*>(insts), count,
                                             static_cast<const CUtensorMap*>(maps), status);
    return cudaGetLastError();
}

}  // namespace qaoa
