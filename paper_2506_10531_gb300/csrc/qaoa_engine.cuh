// qaoa_engine.cuh -- the shared-memory tile engine of libqaoa.
//
// A tile is 2^tb amplitudes of one QAOA state held in shared memory (swizzled, see swz()).
// The whole state is a tile in the resident tier; the streaming tier moves tiles between HBM
// and shared memory. Inside a tile the mixer (Section IV, Eq. 2: exp(-i beta X_q) on every
// qubit) is applied in *sub-passes*: a sub-pass loads groups of 2^R amplitudes that differ
// only in a window of R consecutive tile bits [a, a+R) into registers, applies the
// butterflies of the window's qubits (a bit mask chooses which), and writes them back. Each
// thread owns whole groups; the 32 lanes of a warp own groups that differ in the lowest tile
// bits outside the window, so with the swizzle every access of a warp hits distinct banks.
//
// Layers are scheduled in a "snake": within a layer the windows are visited in one order,
// in the next layer in the reverse order, so the last window of layer l and the first window
// of layer l+1 are the same and share one sub-pass: mixer_l(window), cost_{l+1} (elementwise),
// mixer_{l+1}(window). With G windows per layer this takes 1 + p (G - 1) sub-passes instead of
// p G. The adjoint runs the same sub-passes in reverse order with each operation inverted.
#pragma once
#include "qaoa_common.cuh"

namespace qaoa {

// Per-layer constants staged in shared memory: cost uses gamma/pi, the mixer (cos b, sin b).
// A layer with |cos b| >= |sin b| mixes with unscaled shears (t = tan b); the factor
// (cos b)^n it leaves is applied by the next layer's cost phase (`pre`) or, for the last layer,
// by the last sub-pass (`post`).
template <typename T>
struct LayerConst {
    T gpi;     // gamma_l / pi
    T c, s;    // cos(beta_l), sin(beta_l)
    T t;       // tan(beta_l) when shear != 0
    T pre;     // scale applied with this layer's cost phase (pending factor of layer l-1)
    T post;    // scale still pending after this layer (used for the last layer)
    int shear;
};

// x^n by repeated squaring in the working precision (no FP64 on the complex64 path).
template <typename T>
__device__ __forceinline__ T ipow(T x, int n) {
    T r = T(1);
    while (n) {
        if (n & 1) r *= x;
        x *= x;
        n >>= 1;
    }
    return r;
}

// Fill the constants of p layers of an n-qubit instance (one thread per layer; contains a
// __syncthreads, so every thread of the block calls it).
template <typename T>
__device__ __forceinline__ void set_layer_consts(LayerConst<T>* lc, const T* gamma, const T* beta,
                                                 int p, int n, bool allow_shear) {
    for (int l = threadIdx.x; l < p; l += blockDim.x) {
        T sb, cb;
        sincos_full(beta[l], sb, cb);
        LayerConst<T> k;
        k.gpi = gamma[l] * T(0.31830988618379067154);   // 1 / pi
        k.c = cb;
        k.s = sb;
        k.shear = (allow_shear && fabs(cb) >= fabs(sb)) ? 1 : 0;
        k.t = k.shear ? sb / cb : T(0);
        k.post = k.shear ? ipow(cb, n) : T(1);
        k.pre = T(1);
        lc[l] = k;
    }
    __syncthreads();
    for (int l = 1 + (int)threadIdx.x; l < p; l += blockDim.x) lc[l].pre = lc[l - 1].post;
    __syncthreads();
}

// One sub-pass: window start a, butterfly mask over the window bits, layers [la, lb]
// (lb <= la + 1), whether the cost of layer la opens the sub-pass; post != 0 applies the
// pending shear factor of layer lb after its mixer (set by the caller on the very last
// sub-pass of a state).
struct SubPass {
    int a, mask, la, lb, ph_first, post;
};

// Windows of a layer over the mixed tile bits [m0, m1): window w covers bits
// [m0 + w R, min(m0 + (w+1) R, m1)); its register window is shifted down when it would run
// past the tile top so that it always spans R valid bits.
__device__ __forceinline__ void window_of(int w, int m0, int m1, int tb, int R, int& a, int& mask) {
    const int lo = m0 + w * R;
    const int hi = min(lo + R, m1);
    a = min(lo, tb - R);
    if (a < 0) a = 0;
    mask = ((1 << (hi - lo)) - 1) << (lo - a);
}

__device__ __forceinline__ int num_windows(int m0, int m1, int R) { return (m1 - m0 + R - 1) / R; }

// Number of sub-passes of the snake schedule for layers [L0, L1] over G windows.
__device__ __forceinline__ int snake_len(int G, int nl) {
    return (G <= 1) ? nl : 1 + nl * (G - 1);
}

// The s-th sub-pass of the snake over layers L0..L0+nl-1 (ph_first of the very first one is
// given by `first_ph`). Returns window index w plus the SubPass fields. top_phase: a single
// layer that opens with its cost phase runs its windows top down, so the phase shares the top
// window (the mixer windows of one layer commute); the TMA adjoint keeps every energy read in a
// window whose lanes cover the low tile bits that way.
__device__ __forceinline__ void snake_step(int s, int G, int nl, int L0, int first_ph, int m0,
                                           int m1, int tb, int R, SubPass& sp, bool top_phase = false) {
    int w, la, lb, phf;
    if (G <= 1) {
        w = 0;
        la = lb = L0 + s;
        phf = (s == 0) ? first_ph : 1;
    } else {
        // sub-pass 0 is window order[0] of layer 0; afterwards layer l has G-1 sub-passes
        int l, pos;
        if (s < G) { l = 0; pos = s; }
        else { l = 1 + (s - G) / (G - 1); pos = 1 + (s - G) % (G - 1); }
        const bool fwd = (l % 2) == 0 && !(top_phase && nl == 1 && first_ph);
        w = fwd ? pos : (G - 1 - pos);
        la = L0 + l;
        lb = (pos == G - 1 && l + 1 < nl) ? la + 1 : la;
        phf = (l == 0 && pos == 0) ? first_ph : 0;
    }
    int a, mask;
    window_of(w, m0, m1, tb, R, a, mask);
    sp.a = a;
    sp.mask = mask;
    sp.la = la;
    sp.lb = lb;
    sp.ph_first = phf;
    sp.post = 0;
}

// Local index of element i of group g for window start a (R window bits).
template <int R>
__device__ __forceinline__ uint32_t group_base(uint32_t g, int a) {
    const uint32_t low = g & ((1u << a) - 1u);
    const uint32_t high = g >> a;
    return low | (high << (a + R));
}

// Mixer of one layer on the masked window bits of a register group (rotated frame).
template <int R, typename C, typename T>
__device__ __forceinline__ void mix_group(C (&v)[1 << R], int mask, T c, T s) {
    const RotCoef<T> k(c, s);
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (mask & (1 << j)) {
#pragma unroll
            for (int i = 0; i < (1 << R); ++i)
                if (!(i & (1 << j))) butterfly(v[i], v[i | (1 << j)], k);
        }
    }
}

// Shear-form mixer (see LayerConst): a' = a - t b, b' = b + t a on the masked window bits.
template <int R, typename C, typename T>
__device__ __forceinline__ void mix_group_shear(C (&v)[1 << R], int mask, T t) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (mask & (1 << j)) {
#pragma unroll
            for (int i = 0; i < (1 << R); ++i)
                if (!(i & (1 << j))) butterfly_shear(v[i], v[i | (1 << j)], t);
        }
    }
}

// Scale every amplitude of a group.
template <int R, typename C, typename T>
__device__ __forceinline__ void scale_group(C (&v)[1 << R], T f) {
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) {
        v[i].x *= f;
        v[i].y *= f;
    }
}

// Mixer of layer constants k on a register group (shear or full rotation).
template <int R, typename C, typename T>
__device__ __forceinline__ void mix_layer(C (&v)[1 << R], int mask, const LayerConst<T>& k) {
    if (k.shear) mix_group_shear<R>(v, mask, k.t);
    else mix_group<R>(v, mask, k.c, k.s);
}

// Mixer inverse on two states with the accumulation of Im <lam| X_q |psi> over the masked
// qubits. Any point of the layer's mixer gives the same value (X_q commutes with every
// exp(-i beta X_q')). In the rotated frame X_q becomes Y_q, so over the pairs (a, b)
//   Im <lam|X_q|psi> = sum Re(conj(lam~_b) psi~_a) - Re(conj(lam~_a) psi~_b).
// Four independent partial sums keep the accumulation off the FMA latency chain.
template <int R, typename C, typename T>
__device__ __forceinline__ T mix_group_adj(C (&v)[1 << R], C (&u)[1 << R], int mask, T c, T s) {
    const RotCoef<T> k(c, -s);
    T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int j = 0; j < R; ++j) {
        if (mask & (1 << j)) {
            int slot = 0;
#pragma unroll
            for (int i = 0; i < (1 << R); ++i)
                if (!(i & (1 << j))) {
                    const int b = i | (1 << j);
                    T& a = acc[slot++ & 3];
                    a = fma(u[b].x, v[i].x, a);
                    a = fma(u[b].y, v[i].y, a);
                    a = fma(-u[i].x, v[b].x, a);
                    a = fma(-u[i].y, v[b].y, a);
                    butterfly(v[i], v[b], k);
                    butterfly(u[i], u[b], k);
                }
        }
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// Shared-memory layout of a tile: position of amplitude u (p) and of energy u (e). The engine's
// own swizzle for both; the TMA tiers use the hardware's 128-byte swizzle for amplitudes and
// unswizzled energies. Both maps are linear over GF(2).
template <typename T>
struct SwzLayout {
    __device__ __forceinline__ static uint32_t p(uint32_t u) { return swz<T>(u); }
    __device__ __forceinline__ static uint32_t e(uint32_t u) { return swz<T>(u); }
};

// Element addresses of a group. The swizzle is linear over GF(2) and a group's base index and
// its window offsets (i << A) have disjoint bits, so
//   swz(base | (i << A)) = swz(base) ^ swz(i << A),
// one XOR of a per-thread value with a compile-time constant per element.
template <typename T, int A>
__device__ __forceinline__ uint32_t woff(int i) { return swz<T>((uint32_t)i << A); }

// Load / store the 2^R amplitudes of a group (window start A). complex64 windows starting at
// bit 0 move aligned pairs with one 16-byte shared access (the swizzle keeps pairs adjacent).
template <int R, int A, typename Lay = SwzLayout<float>>
__device__ __forceinline__ void load_group(const float2* psi, uint32_t sb, float2 (&v)[1 << R]) {
    if (A == 0 && R >= 1) {
#pragma unroll
        for (int i = 0; i < (1 << R); i += 2) {
            const float4 t = *reinterpret_cast<const float4*>(psi + (sb ^ Lay::p((uint32_t)i << A)));
            v[i] = make_float2(t.x, t.y);
            v[i + 1] = make_float2(t.z, t.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) v[i] = psi[sb ^ Lay::p((uint32_t)i << A)];
    }
}
template <int R, int A, typename Lay = SwzLayout<float>>
__device__ __forceinline__ void store_group(float2* psi, uint32_t sb, const float2 (&v)[1 << R]) {
    if (A == 0 && R >= 1) {
#pragma unroll
        for (int i = 0; i < (1 << R); i += 2)
            *reinterpret_cast<float4*>(psi + (sb ^ Lay::p((uint32_t)i << A))) =
                make_float4(v[i].x, v[i].y, v[i + 1].x, v[i + 1].y);
    } else {
#pragma unroll
        for (int i = 0; i < (1 << R); ++i) psi[sb ^ Lay::p((uint32_t)i << A)] = v[i];
    }
}
template <int R, int A, typename Lay = SwzLayout<double>>
__device__ __forceinline__ void load_group(const double2* psi, uint32_t sb, double2 (&v)[1 << R]) {
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) v[i] = psi[sb ^ Lay::p((uint32_t)i << A)];
}
template <int R, int A, typename Lay = SwzLayout<double>>
__device__ __forceinline__ void store_group(double2* psi, uint32_t sb, const double2 (&v)[1 << R]) {
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) psi[sb ^ Lay::p((uint32_t)i << A)] = v[i];
}

// Shared state of one tile.
template <typename T>
struct TileRef {
    typename Num<T>::C* psi;   // 2^tb amplitudes, swizzled
    typename Num<T>::C* lam;   // adjoint state (or nullptr)
    const T* E;                // 2^tb energies, swizzled
    int tb;                    // tile bits
};

// Forward sub-pass with a compile-time window start A (see subpass_fwd).
template <typename T, int R, int A, typename Fin>
__device__ __forceinline__ void subpass_fwd_a(const TileRef<T>& t, const SubPass& sp,
                                              const LayerConst<T>* lc, bool init, T amp0, int pc0,
                                              Fin&& fin) {
    using C = typename Num<T>::C;
    const uint32_t ngroups = 1u << (t.tb - R);
    for (uint32_t g0 = 0; g0 < ngroups; g0 += blockDim.x) {
        const uint32_t g = g0 + threadIdx.x;
        const bool valid = g < ngroups;
        const uint32_t base = group_base<R>(valid ? g : 0u, A);
        const uint32_t sb = swz<T>(base);
        C v[1 << R];
        if (valid) {
            if (init) {
                // |+> in the rotated frame: amp0 i^{|z|}, |z| = pc0 + |base| + |i|; the four
                // values i^m amp0 are formed once and picked by the compile-time |i|
                const int pb = pc0 + __popc(base);
                C a;
                a.x = amp0;
                a.y = T(0);
                const C q0 = times_i_pow(a, pb), q1 = times_i_pow(a, pb + 1);
                const C q2 = times_i_pow(a, pb + 2), q3 = times_i_pow(a, pb + 3);
#pragma unroll
                for (int i = 0; i < (1 << R); ++i) {
                    const int m = __popc(i) & 3;
                    v[i] = m == 0 ? q0 : (m == 1 ? q1 : (m == 2 ? q2 : q3));
                }
            } else {
                load_group<R, A>(t.psi, sb, v);
            }
            for (int l = sp.la; l <= sp.lb; ++l) {
                if (l > sp.la || sp.ph_first) {
                    const T gp = lc[l].gpi, pre = lc[l].pre;
#pragma unroll
                    for (int i = 0; i < (1 << R); ++i) {
                        T s, c;
                        sincos_phase(gp, t.E[sb ^ woff<T, A>(i)], s, c);
                        rot_neg(v[i], s * pre, c * pre);
                    }
                }
                mix_layer<R>(v, sp.mask, lc[l]);
            }
            if (sp.post && lc[sp.lb].shear) scale_group<R>(v, lc[sp.lb].post);
            store_group<R, A>(t.psi, sb, v);
        }
        fin(base, A, valid);
    }
}

// Forward sub-pass over all groups of the tile.
//   init:  amplitudes start as |+> (amp0 i^{|z|} in the rotated frame; pc0 = number of set
//          global bits that the tile index itself fixes) instead of being read
//   fin:   called once per group slot after the group has been written back, by every thread
//          of the block (warp-uniform trip count), as fin(base, a, valid); it re-reads the
//          group from shared memory, which keeps the final reductions out of the register
//          budget of the butterflies.
// The window start is dispatched to a compile-time constant (0 <= a <= tb - R <= 9).
template <typename T, int R, typename Fin>
__device__ __forceinline__ void subpass_fwd(const TileRef<T>& t, const SubPass& sp,
                                            const LayerConst<T>* lc, bool init, T amp0, int pc0,
                                            Fin&& fin) {
    switch (sp.a) {
        case 0: subpass_fwd_a<T, R, 0>(t, sp, lc, init, amp0, pc0, fin); break;
        case 1: subpass_fwd_a<T, R, 1>(t, sp, lc, init, amp0, pc0, fin); break;
        case 2: subpass_fwd_a<T, R, 2>(t, sp, lc, init, amp0, pc0, fin); break;
        case 3: subpass_fwd_a<T, R, 3>(t, sp, lc, init, amp0, pc0, fin); break;
        case 4: subpass_fwd_a<T, R, 4>(t, sp, lc, init, amp0, pc0, fin); break;
        case 5: subpass_fwd_a<T, R, 5>(t, sp, lc, init, amp0, pc0, fin); break;
        case 6: subpass_fwd_a<T, R, 6>(t, sp, lc, init, amp0, pc0, fin); break;
        case 7: subpass_fwd_a<T, R, 7>(t, sp, lc, init, amp0, pc0, fin); break;
        case 8: subpass_fwd_a<T, R, 8>(t, sp, lc, init, amp0, pc0, fin); break;
        default: subpass_fwd_a<T, R, 9>(t, sp, lc, init, amp0, pc0, fin); break;
    }
}

// Adjoint sub-pass with a compile-time window start A (see subpass_adj).
template <typename T, int R, int A, typename Lay = SwzLayout<T>>
__device__ __forceinline__ void subpass_adj_a(const TileRef<T>& t, const SubPass& sp,
                                              const LayerConst<T>* lc, bool lam_from_E,
                                              T (&acc_b)[2], T (&acc_g)[2]) {
    using C = typename Num<T>::C;
    const uint32_t ngroups = 1u << (t.tb - R);
    for (uint32_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const uint32_t base = group_base<R>(g, A);
        const uint32_t sb = Lay::p(base), eb = Lay::e(base);
        C v[1 << R], u[1 << R];
        load_group<R, A, Lay>(t.psi, sb, v);
        if (lam_from_E) {
#pragma unroll
            for (int i = 0; i < (1 << R); ++i) {
                const T e = t.E[eb ^ Lay::e((uint32_t)i << A)];
                u[i].x = e * v[i].x;
                u[i].y = e * v[i].y;
            }
        } else {
            load_group<R, A, Lay>(t.lam, sb, u);
        }
        for (int l = sp.lb; l >= sp.la; --l) {
            const int j = sp.lb - l;
            const T ab = mix_group_adj<R>(v, u, sp.mask, lc[l].c, lc[l].s);
            if (j == 0) acc_b[0] += ab; else acc_b[1] += ab;
            if (l > sp.la || sp.ph_first) {
                const T gp = -lc[l].gpi;
                T ag[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
                for (int i = 0; i < (1 << R); ++i) {
                    const T e = t.E[eb ^ Lay::e((uint32_t)i << A)];
                    ag[i & 3] = fma(e, im_conj_mul(u[i], v[i]), ag[i & 3]);
                    T s, c;
                    sincos_phase(gp, e, s, c);
                    rot_neg(v[i], s, c);
                    rot_neg(u[i], s, c);
                }
                const T agt = (ag[0] + ag[1]) + (ag[2] + ag[3]);
                if (j == 0) acc_g[0] += agt; else acc_g[1] += agt;
            }
        }
        store_group<R, A, Lay>(t.psi, sb, v);
        store_group<R, A, Lay>(t.lam, sb, u);
    }
}

// Adjoint sub-pass: the forward sub-pass `sp` undone on psi and lam, accumulating
//   acc_b[j] += Im <lam| sum_q X_q |psi> (window qubits) for layer lb - j,
//   acc_g[j] += Im <lam| E |psi>                          for layer lb - j (its cost op).
// lam_from_E: lam = E psi is formed on load (first adjoint sub-pass).
template <typename T, int R, typename Lay = SwzLayout<T>>
__device__ __forceinline__ void subpass_adj(const TileRef<T>& t, const SubPass& sp,
                                            const LayerConst<T>* lc, bool lam_from_E,
                                            T (&acc_b)[2], T (&acc_g)[2]) {
    switch (sp.a) {
        case 0: subpass_adj_a<T, R, 0, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
        case 1: subpass_adj_a<T, R, 1, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
        case 2: subpass_adj_a<T, R, 2, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
        case 3: subpass_adj_a<T, R, 3, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
        case 4: subpass_adj_a<T, R, 4, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
        case 5: subpass_adj_a<T, R, 5, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
        case 6: subpass_adj_a<T, R, 6, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
        case 7: subpass_adj_a<T, R, 7, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
        case 8: subpass_adj_a<T, R, 8, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
        default: subpass_adj_a<T, R, 9, Lay>(t, sp, lc, lam_from_E, acc_b, acc_g); break;
    }
}

// Final reductions of one group (2^R amplitudes of window start a, already written back):
// <C> partial (FP32 over the group, FP64 across groups) and the warp's top-k list. Before
// offering, the list threshold is raised to the k-th largest of the lanes' group maxima: the k
// lanes with the largest maxima hold k distinct elements at least that probable, so every
// element of the final top-k passes the FP32 filter (margins as in WarpTopK::offer), while
// most elements are rejected without an insertion. zmap(u) gives the global index of tile
// index u. Called by every thread of the warp.
template <typename T, int R, typename ZMap>
__device__ __forceinline__ void reduce_group(const TileRef<T>& t, uint32_t base, int a, bool valid,
                                             int k, WarpTopK& top, double& ex, ZMap&& zmap) {
    using C = typename Num<T>::C;
    T accp = T(0);
    float pmax = -1.0f;
#pragma unroll 1
    for (int i = 0; i < (1 << R); ++i) {
        if (valid) {
            const uint32_t ix = swz<T>(base | ((uint32_t)i << a));
            const C v = t.psi[ix];
            const T pr = v.x * v.x + v.y * v.y;
            accp += pr * t.E[ix];
            pmax = fmaxf(pmax, (float)pr);
        }
    }
    ex += (double)accp;
    if (k <= 0) return;
    const float kth = warp_kth_largest(pmax, k);
    if (kth > 0.0f) top.raise_threshold(kth * 0.99999904632568359375f);   // (1 - 2^-20)
#pragma unroll 1
    for (int i = 0; i < (1 << R); ++i) {
        const uint32_t u = base | ((uint32_t)i << a);
        C v;
        v.x = T(0);
        v.y = T(0);
        if (valid) v = t.psi[swz<T>(u)];
        top.offer(v, zmap(u), valid);
    }
}

// ---- energies of a tile -----------------------------------------------------------------
// E(z) = z^T Q z for the 2^L tile indices u of one n-qubit instance, z = zfix | u (zfix holds
// global bits >= L that the tile fixes, e.g. the CTA rank of a cluster). With u split into
// three bit fields lo = [0, B), ha = [B, B+A), hb = [B+A, L) and S = the set bits of zfix:
//   E(z) = E_S + El[lo] + Ea[ha] + Eb[hb] + Xa[lo][ha] + Xb[lo][hb] + Xab[ha][hb],
//   El[lo]  = sum_{i,j in lo} Q_ij + sum_{i in lo, j in S} (Q_ij + Q_ji)   (Ea, Eb likewise),
//   Xa[lo][ha] = sum_{i in lo, j in ha} (Q_ij + Q_ji)                        (Xb, Xab likewise).
// Every pair of set bits of z falls in exactly one term. The tables are small (a few KB)
// and built in parallel; then every element is six table reads and six adds, independent of
// all other elements (no serial walk). scratch: tile_energy_scratch(L) values of T.
__host__ __device__ inline void energy_fields(int L, int& B, int& A) {
    B = (L + 1) / 2;
    A = (L - B) / 2;
}
__host__ __device__ inline size_t tile_energy_scratch(int L) {
    int B, A;
    energy_fields(L, B, A);
    const int Hb = L - B - A;
    return 1 + ((size_t)1 << B) + ((size_t)1 << A) + ((size_t)1 << Hb) +
           ((size_t)1 << (B + A)) + ((size_t)1 << (B + Hb)) + ((size_t)1 << (A + Hb));
}

template <typename T>
__device__ __forceinline__ T pair_sum(const T* Qs, int n, uint32_t x, int xs, uint32_t y, int ys) {
    // sum over set bits i of x (shifted by xs) and j of y (shifted by ys) of Q_ij + Q_ji
    T acc = T(0);
    for (uint32_t bi = x; bi; bi &= bi - 1u) {
        const int i = xs + __ffs((int)bi) - 1;
        for (uint32_t bj = y; bj; bj &= bj - 1u) {
            const int j = ys + __ffs((int)bj) - 1;
            acc += Qs[i * n + j] + Qs[j * n + i];
        }
    }
    return acc;
}
template <typename T>
__device__ __forceinline__ T self_sum(const T* Qs, int n, uint32_t x, int xs, uint32_t zfix) {
    // sum_{i,j in x} Q_ij + sum_{i in x, j in zfix} (Q_ij + Q_ji)
    T acc = T(0);
    for (uint32_t bi = x; bi; bi &= bi - 1u) {
        const int i = xs + __ffs((int)bi) - 1;
        for (uint32_t bj = x; bj; bj &= bj - 1u) acc += Qs[i * n + xs + __ffs((int)bj) - 1];
        for (uint32_t bj = zfix; bj; bj &= bj - 1u) {
            const int j = __ffs((int)bj) - 1;
            acc += Qs[i * n + j] + Qs[j * n + i];
        }
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ void build_tile_energy(int n, int L, uint32_t zfix, const T* Qs, T* E,
                                                  T* scratch) {
    int B, A;
    energy_fields(L, B, A);
    const int Hb = L - B - A;
    const uint32_t NL = 1u << B, NA = 1u << A, NB = 1u << Hb;
    T* Es = scratch;
    T* El = Es + 1;
    T* Ea = El + NL;
    T* Eb = Ea + NA;
    T* Xa = Eb + NB;            // [ha][lo]: consecutive lanes read consecutive lo (no conflicts)
    T* Xb = Xa + NL * NA;       // [hb][lo]
    T* Xab = Xb + NL * NB;      // [ha][hb] (one address per warp: broadcast)
    const uint32_t total = 1u + NL + NA + NB + NL * NA + NL * NB + NA * NB;
    for (uint32_t x = threadIdx.x; x < total; x += blockDim.x) {
        uint32_t y = x;
        if (y == 0) {                                   // E_S
            T acc = T(0);
            for (uint32_t bi = zfix; bi; bi &= bi - 1u) {
                const int i = __ffs((int)bi) - 1;
                for (uint32_t bj = zfix; bj; bj &= bj - 1u) acc += Qs[i * n + __ffs((int)bj) - 1];
            }
            Es[0] = acc;
            continue;
        }
        y -= 1;
        if (y < NL) { El[y] = self_sum(Qs, n, y, 0, zfix); continue; }
        y -= NL;
        if (y < NA) { Ea[y] = self_sum(Qs, n, y, B, zfix); continue; }
        y -= NA;
        if (y < NB) { Eb[y] = self_sum(Qs, n, y, B + A, zfix); continue; }
        y -= NB;
        if (y < NL * NA) { Xa[y] = pair_sum(Qs, n, y & (NL - 1u), 0, y >> B, B); continue; }
        y -= NL * NA;
        if (y < NL * NB) { Xb[y] = pair_sum(Qs, n, y & (NL - 1u), 0, y >> B, B + A); continue; }
        y -= NL * NB;
        Xab[y] = pair_sum(Qs, n, y >> Hb, B, y & (NB - 1u), B + A);
    }
    __syncthreads();
    const T es = Es[0];
    for (uint32_t u = threadIdx.x; u < (1u << L); u += blockDim.x) {
        const uint32_t lo = u & (NL - 1u), ha = (u >> B) & (NA - 1u), hb = u >> (B + A);
        E[swz<T>(u)] = ((es + El[lo]) + (Ea[ha] + Eb[hb])) +
                       ((Xa[(ha << B) | lo] + Xb[(hb << B) | lo]) + Xab[(ha << Hb) | hb]);
    }
}

// Fast path of the tile energies when blockDim = 2^(L - HB): thread t owns the low field
// lo = t (B = L - HB bits) and the 2^HB elements u = t | (j << B). With S the set bits of zfix
//   E(z) = [E_S + El(t)] + Eh[j] + X_t(j),   X_t(j) = sum_{b in j} W_b(t),
//   W_b(t) = sum_{i in t} (Q_{i,B+b} + Q_{B+b,i}),
// El(t) and W_b(t) are evaluated by the thread (sums over the set bits of t), Eh (2^HB
// entries, shared) by 2^HB threads, and X_t(j) for all j by subset doubling in registers
// (2^HB - 1 additions). Each element is then one broadcast read, two adds and one store.
// Optional fused start of the state: with psi != nullptr every element is also set to the
// |+> amplitude after the first cost layer, amp0 i^{|z|} e^{-i gamma_0 E(z)} (rotated frame,
// |z| = pc0 + |u|), so the first sub-pass starts with the first mixer.
template <typename T>
struct FusedInit {
    typename Num<T>::C* psi;   // nullptr: energies only
    T amp0, gpi0;              // 2^{-n/2}, gamma_0 / pi
    int pc0;                   // set bits of zfix
};

template <typename T>
__device__ __forceinline__ void fused_init_store(const FusedInit<T>& fi, uint32_t u, uint32_t ix, T e) {
    typename Num<T>::C a;
    T s, c;
    sincos_phase(fi.gpi0, e, s, c);
    a.x = fi.amp0 * c;          // amp0 e^{-i theta}
    a.y = -fi.amp0 * s;
    fi.psi[ix] = times_i_pow(a, fi.pc0 + __popc(u));
}

template <typename T, int HB>
__device__ __forceinline__ void build_tile_energy_fast(int n, int L, uint32_t zfix, const T* Qs,
                                                       T* E, T* scratch, const FusedInit<T>& fi) {
    const int B = L - HB;
    const uint32_t t = threadIdx.x;
    T* Eh = scratch;                 // 2^HB entries: hi self terms + hi x S
    if (t < (1u << HB)) {
        T acc = T(0);
        const uint32_t hbits = t << B;
        for (uint32_t bi = hbits; bi; bi &= bi - 1u) {
            const int i = __ffs((int)bi) - 1;
            for (uint32_t bj = hbits; bj; bj &= bj - 1u) acc += Qs[i * n + __ffs((int)bj) - 1];
            for (uint32_t bj = zfix; bj; bj &= bj - 1u) {
                const int j = __ffs((int)bj) - 1;
                acc += Qs[i * n + j] + Qs[j * n + i];
            }
        }
        Eh[t] = acc;
    }
    // E_S + El(t), and W_b(t): loops over bit positions (the same for every lane, so each Q
    // read is a shared-memory broadcast) with predicated adds instead of loops over the set
    // bits of t (which diverge across the warp)
    T base = T(0);
    for (uint32_t bi = zfix; bi; bi &= bi - 1u) {
        const int i = __ffs((int)bi) - 1;
        for (uint32_t bj = zfix; bj; bj &= bj - 1u) base += Qs[i * n + __ffs((int)bj) - 1];
    }
    for (int i = 0; i < B; ++i) {
        const bool ti = (t >> i) & 1u;
        T si = Qs[i * n + i];
        for (uint32_t bj = zfix; bj; bj &= bj - 1u) {
            const int j = __ffs((int)bj) - 1;
            si += Qs[i * n + j] + Qs[j * n + i];
        }
        T cross = T(0);
        for (int j = 0; j < i; ++j)
            if ((t >> j) & 1u) cross += Qs[i * n + j] + Qs[j * n + i];
        if (ti) base += si + cross;
    }
    T X[1 << HB];
    X[0] = T(0);
#pragma unroll
    for (int b = 0; b < HB; ++b) {
        T w = T(0);
        const int q = B + b;
        for (int i = 0; i < B; ++i)
            if ((t >> i) & 1u) w += Qs[i * n + q] + Qs[q * n + i];
#pragma unroll
        for (int m = 0; m < (1 << b); ++m) X[m | (1 << b)] = X[m] + w;
    }
    __syncthreads();
    const uint32_t st = swz<T>(t);
#pragma unroll
    for (int j = 0; j < (1 << HB); ++j) {
        const uint32_t ix = st ^ swz<T>((uint32_t)j << B);
        const T ev = base + (Eh[j] + X[j]);
        E[ix] = ev;
        if (fi.psi) fused_init_store(fi, t | ((uint32_t)j << B), ix, ev);
    }
}

// Energies of the tile (fast path when blockDim = 2^(L - HB), HB <= 5), and optionally the
// fused start of the state (see FusedInit). Returns true if the state was started. Not
// inlined: its 2^HB register subset sums would otherwise add to the register pressure of the
// whole calling kernel (spills there cost more than the call).
template <typename T>
__device__ __noinline__ bool build_tile_energy_any(int n, int L, uint32_t zfix, const T* Qs,
                                                      T* E, T* scratch, const FusedInit<T>& fi) {
    const int lg = 31 - __clz((int)blockDim.x);
    switch (L - lg) {
        case 0: build_tile_energy_fast<T, 0>(n, L, zfix, Qs, E, scratch, fi); return fi.psi != nullptr;
        case 1: build_tile_energy_fast<T, 1>(n, L, zfix, Qs, E, scratch, fi); return fi.psi != nullptr;
        case 2: build_tile_energy_fast<T, 2>(n, L, zfix, Qs, E, scratch, fi); return fi.psi != nullptr;
        case 3: build_tile_energy_fast<T, 3>(n, L, zfix, Qs, E, scratch, fi); return fi.psi != nullptr;
        case 4: build_tile_energy_fast<T, 4>(n, L, zfix, Qs, E, scratch, fi); return fi.psi != nullptr;
        case 5: build_tile_energy_fast<T, 5>(n, L, zfix, Qs, E, scratch, fi); return fi.psi != nullptr;
        default: build_tile_energy<T>(n, L, zfix, Qs, E, scratch); return false;
    }
}

// ---- final reductions of a tile -----------------------------------------------------------
// Shared-memory placement of tile index u for the state (p) and the energies (e): the engine's
// swizzle for both (default), or another layout supplied by a tier (a TMA-staged tile).

// Shared scratch of tile_reduce (sizes: wb 16 * nwarps floats, cand TOPK_CAP entries, out 16,
// wlists 32 * nwarps entries, cnt 4 ints).
constexpr int TOPK_CAP = 256;
struct TileTopk {
    float* wb;        // per-warp sorted lane maxima (k per warp)
    TopEnt* cand;     // candidate buffer
    TopEnt* out;      // the tile's top-k (valid after tile_reduce)
    TopEnt* wlists;   // (blockDim/32) * 32 entries, used only by the fallback
    int* cnt;         // [0] candidate count, [1] overflow flag, [2..3] bound (float / double bits)
};

// Collect the elements whose probability can reach `bound_lo` (FP32 filter with the margins of
// WarpTopK::offer; with exact_bound != 0 the exact probability must also be >= *exact_bound)
// into ts.cand. Sets ts.cnt[1] on overflow. Each thread scans only its own elements
// u = tid + j * blockDim, and only if its FP32 maximum over them (pmax, from the pass that
// computed the tile's <C> partial) can reach the bound: a list of k entries has few owners, so
// most threads skip the scan. pmax and the per-element value are two FP32 roundings of the same
// probability, each within 2^-21 of it, hence the wider 2^-18 margin of the thread test.
template <typename T, typename Lay = SwzLayout<T>, typename ZMap>
__device__ __forceinline__ void collect_candidates(const TileRef<T>& t, float pmax, float bound_lo,
                                                   const double* exact_bound, ZMap&& zmap,
                                                   const TileTopk& ts) {
    using C = typename Num<T>::C;
    const uint32_t D = 1u << t.tb;
    if (!(pmax * 1.000003814697265625f >= bound_lo)) return;
    const long long eb = exact_bound ? pbits(*exact_bound) : -1ll;
    for (uint32_t c0 = 0; c0 < D; c0 += 32u * blockDim.x) {
        // FP32 test of up to 32 elements first (independent loads), then the hits one by one
        uint32_t hits = 0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const uint32_t u = c0 + (uint32_t)j * blockDim.x + threadIdx.x;
            if (u < D) {
                const C v = t.psi[Lay::p(u)];
                const float pf = (float)v.x * (float)v.x + (float)v.y * (float)v.y;
                if (pf * 1.00000095367431640625f >= bound_lo) hits |= 1u << j;
            }
        }
        while (hits) {
            const int j = __ffs(hits) - 1;
            hits &= hits - 1;
            const uint32_t u = c0 + (uint32_t)j * blockDim.x + threadIdx.x;
            const double pe = exact_prob(t.psi[Lay::p(u)]);
            if (pbits(pe) >= eb) {
                const int pos = atomicAdd(&ts.cnt[0], 1);
                if (pos < TOPK_CAP) ts.cand[pos] = TopEnt{pe, zmap(u)};
                else ts.cnt[1] = 1;
            }
        }
    }
}

// <C> partial of the tile (FP32 |psi|^2 E over at most 32 elements per thread, FP64 above, added
// to `ex`) and the thread's largest FP32 probability over its elements u = tid + j * blockDim
// (its lane maximum, returned). Called by all threads; no barrier.
template <typename T, typename Lay = SwzLayout<T>>
__device__ __forceinline__ float tile_expect(const TileRef<T>& t, double& ex) {
    using C = typename Num<T>::C;
    const uint32_t D = 1u << t.tb;
    float pmax = -1.0f;
    for (uint32_t c0 = 0; c0 < D; c0 += 32u * blockDim.x) {
        T accp = T(0);
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const uint32_t u = c0 + (uint32_t)j * blockDim.x + threadIdx.x;
            if (u < D) {
                const C v = t.psi[Lay::p(u)];
                const T pr = v.x * v.x + v.y * v.y;
                accp += pr * t.E[Lay::e(u)];
                pmax = fmaxf(pmax, (float)pr);
            }
        }
        ex += (double)accp;
    }
    return pmax;
}

// Top-k list of the whole tile into ts.out, given each thread's lane maximum pmax:
//  1. a lower bound on the tile's k-th largest probability: the k-th largest of all lane
//     maxima (k distinct elements are at least that probable). Each warp sorts its lane
//     maxima and offers its k largest; their k-th largest is found by rank;
//  2. every element whose probability can reach the bound goes to a shared candidate buffer
//     with its exact FP64 probability; on overflow (flat distributions) the bound is raised
//     to the k-th largest exact probability among the buffered elements and the collection
//     repeated with an exact test;
//  3. each candidate's rank = number of candidates better than it (probability descending,
//     index ascending: a strict total order, so ranks are distinct); ranks < k are the list.
// The result does not depend on the order of the buffer, so the reduction is deterministic.
// If the buffer still overflows (massive ties) the warps fall back to sorted insertion lists
// merged by warp 0. zmap(u): global index of tile index u. Called by all threads, k >= 1.
template <typename T, typename Lay = SwzLayout<T>, typename ZMap>
__device__ __forceinline__ void tile_topk(const TileRef<T>& t, int k, float pmax, ZMap&& zmap,
                                          const TileTopk& ts) {
    using C = typename Num<T>::C;
    const uint32_t D = 1u << t.tb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    // (1) the k-th largest lane maximum of the block
    const float srt = warp_sort_desc(pmax);
    if (lane < k) ts.wb[warp * k + lane] = srt;
    if (threadIdx.x == 0) { ts.cnt[0] = 0; ts.cnt[1] = 0; }
    __syncthreads();
    float* bound = reinterpret_cast<float*>(&ts.cnt[2]);
    const int nl = nw * k;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
        const float me = ts.wb[i];
        int rank = 0;
        for (int j = 0; j < nl; ++j) {
            const float o = ts.wb[j];
            rank += (o > me || (o == me && j < i)) ? 1 : 0;
        }
        if (rank == k - 1) *bound = me;
    }
    __syncthreads();
    const float thr = *bound;
    const float thr_lo = thr > 0.0f ? thr * 0.99999904632568359375f : -1.0f;   // (1 - 2^-20)
    // (2) candidates
    collect_candidates<T, Lay>(t, pmax, thr_lo, nullptr, zmap, ts);
    __syncthreads();
    if (ts.cnt[1]) {
        // raise the bound to the k-th best buffered exact probability and collect again
        double* b2 = reinterpret_cast<double*>(ts.wlists);
        for (int c = threadIdx.x; c < TOPK_CAP; c += blockDim.x) {
            const TopEnt me = ts.cand[c];
            int rank = 0;
            for (int j = 0; j < TOPK_CAP; ++j) {
                const TopEnt o = ts.cand[j];
                rank += better(o.p, o.z, me.p, me.z) ? 1 : 0;
            }
            if (rank == k - 1) *b2 = me.p;
        }
        __syncthreads();
        const float b2lo = __double2float_rd(*b2) * 0.99999904632568359375f;
        if (threadIdx.x == 0) { ts.cnt[0] = 0; ts.cnt[1] = 0; }
        __syncthreads();
        collect_candidates<T, Lay>(t, pmax, b2lo, b2, zmap, ts);
        __syncthreads();
    }
    const int cnt = min(ts.cnt[0], TOPK_CAP);
    if (!ts.cnt[1]) {
        // (3) rank selection
        for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
            const TopEnt me = ts.cand[c];
            int rank = 0;
            for (int j = 0; j < cnt; ++j) {
                const TopEnt o = ts.cand[j];
                rank += better(o.p, o.z, me.p, me.z) ? 1 : 0;
            }
            if (rank < k) ts.out[rank] = me;
        }
        if (threadIdx.x < (unsigned)k && threadIdx.x >= (unsigned)cnt) ts.out[threadIdx.x] = TopEnt{-1.0, 0xffffffffu};
    } else {
        __syncthreads();
        WarpTopK top;
        top.init(k);
        for (uint32_t u0 = 0; u0 < D; u0 += blockDim.x) {
            const uint32_t u = u0 + threadIdx.x;
            C v;
            v.x = T(0);
            v.y = T(0);
            if (u < D) v = t.psi[Lay::p(u)];
            top.offer(v, zmap(u < D ? u : 0u), u < D);
        }
        if (lane < k) ts.wlists[warp * 32 + lane] = TopEnt{top.p, top.z};
        __syncthreads();
        if (warp == 0) {
            WarpTopK f;
            f.init(k);
            for (int w = 0; w < nw; ++w) {
                const bool ok = lane < k;
                const TopEnt e = ok ? ts.wlists[w * 32 + lane] : TopEnt{-1.0, 0xffffffffu};
                f.offer_exact(e.p, e.z, ok);
            }
            if (lane < k) ts.out[lane] = TopEnt{f.p, f.z};
        }
    }
    __syncthreads();
}

// <C> partial (added to `ex`) and, for k >= 1, the top-k list (ts.out) of the whole tile after
// its last sub-pass. Called by all threads.
template <typename T, typename Lay = SwzLayout<T>, typename ZMap>
__device__ __forceinline__ void tile_reduce(const TileRef<T>& t, int k, ZMap&& zmap,
                                            const TileTopk& ts, double& ex) {
    const float pmax = tile_expect<T, Lay>(t, ex);
    if (k <= 0) return;
    tile_topk<T, Lay>(t, k, pmax, zmap, ts);
}

// Fold the tile into `run`, the top-k list (k entries, all present) of the tiles of the same
// state that this block reduced before: only elements that can beat run's k-th entry are
// collected (usually none once a few tiles are in), and the merged list is the k best of the
// candidates and run by rank. On candidate overflow the tile's own list (tile_topk) is merged
// instead. pmax as from tile_expect. Called by all threads.
template <typename T, typename ZMap>
__device__ __forceinline__ void running_topk(const TileRef<T>& t, int k, float pmax, ZMap&& zmap,
                                             const TileTopk& ts, TopEnt* run) {
    const double* pk = &run[k - 1].p;
    const float lo = __double2float_rd(*pk) * 0.99999904632568359375f;
    if (threadIdx.x == 0) { ts.cnt[0] = 0; ts.cnt[1] = 0; }
    if (!__syncthreads_or(pmax * 1.000003814697265625f >= lo)) return;
    collect_candidates<T>(t, pmax, lo, pk, zmap, ts);
    __syncthreads();
    const TopEnt* a = ts.cand;
    int na = ts.cnt[0];
    if (ts.cnt[1]) {
        __syncthreads();                        // every thread has read the counters that tile_topk resets
        tile_topk<T>(t, k, pmax, zmap, ts);
        a = ts.out;
        na = k;
    }
    if (na == 0) return;                        // uniform: every thread read the same count
    TopEnt* merged = ts.wlists;                 // free here (tile_topk ended with a barrier)
    for (int c = threadIdx.x; c < na + k; c += blockDim.x) {
        const TopEnt me = c < na ? a[c] : run[c - na];
        if (!is_entry(me.p)) continue;
        int rank = 0;
        for (int j = 0; j < na; ++j) rank += better(a[j].p, a[j].z, me.p, me.z) ? 1 : 0;
        for (int j = 0; j < k; ++j) rank += better(run[j].p, run[j].z, me.p, me.z) ? 1 : 0;
        if (rank < k) merged[rank] = me;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)k) run[threadIdx.x] = merged[threadIdx.x];
    __syncthreads();
}

// Top-k of a small set of candidate lists already in shared memory (count entries, entries
// with p < 0 are empty): rank selection as in tile_reduce; result in out[0..k).
__device__ __forceinline__ void rank_select(const TopEnt* cand, int count, int k, TopEnt* out) {
    for (int c = threadIdx.x; c < count; c += blockDim.x) {
        const TopEnt me = cand[c];
        if (!is_entry(me.p)) continue;
        int rank = 0;
        for (int j = 0; j < count; ++j) {
            const TopEnt o = cand[j];
            rank += (is_entry(o.p) && better(o.p, o.z, me.p, me.z)) ? 1 : 0;
        }
        if (rank < k) out[rank] = me;
    }
}

// Block-wide sum of one value per thread into slot[0] (thread 0 only); red has blockDim/32
// doubles. Fixed order: deterministic. Must be called by all threads.
__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) tot += red[i];
    return tot;
}

}  // namespace qaoa
