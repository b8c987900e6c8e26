// qaoa_common.cuh -- shared device helpers of libqaoa (types, shared-memory swizzle, the
// butterfly of the mixer, the cost phase, warp-level top-k lists and fixed-order reductions).
//
// Conventions used everywhere in the library (arXiv 2506.10531, Section IV, Eq. 2):
//   * bit q of a basis index z is qubit q (sub-QUBO variable S[q]);
//   * the cost layer multiplies psi(z) by exp(-i gamma E(z));
//   * the mixer layer applies exp(-i beta X_q) to every qubit q: on the amplitude pair
//     (a, b) = (psi[z], psi[z | 2^q]) with bit q of z clear,
//       a' = cos(beta) a - i sin(beta) b,   b' = -i sin(beta) a + cos(beta) b.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qaoa {

template <typename T> struct Num;
template <> struct Num<float> {
    using C = float2;
    static constexpr int RB = 5;        // register window (qubits) of one sub-pass, forward
    static constexpr int RB_ADJ = 4;    // register window of the adjoint (two states live)
};
template <> struct Num<double> {
    using C = double2;
    static constexpr int RB = 4;
    static constexpr int RB_ADJ = 3;
};

// Shared-memory swizzle of a tile index. complex64: bits 1..4 are XORed with bits 5..8, so the
// two amplitudes of an aligned pair (z, z^1) stay adjacent and in order (16-byte copies and
// 16-byte shared accesses keep working); complex128: bits 0..3 XOR bits 4..7. With the lanes of
// a warp on the lowest tile bits outside a register window [a, a+R), every sub-pass access is
// free of bank conflicts (windows that contain bit 0 use 16-byte accesses).
template <typename T>
__device__ __forceinline__ uint32_t swz(uint32_t z);
template <>
__device__ __forceinline__ uint32_t swz<float>(uint32_t z) { return z ^ ((z >> 4) & 30u); }
template <>
__device__ __forceinline__ uint32_t swz<double>(uint32_t z) { return z ^ ((z >> 4) & 15u); }

// ---- asynchronous global -> shared copies (16 / 8 bytes, L2 only for 16) -----------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- optimiser ------------------------------------------------------------------------------
// One Adam step (Kingma & Ba 2015) on one parameter; step >= 1 (bias correction). Shared by the
// flat-array and the per-job (serving) update kernels so both give the same bits.
__device__ __forceinline__ void adam_update(float& theta, float& m, float& v, double grad, int step,
                                            float lr, float b1, float b2, float eps, int minimise) {
    const float g = minimise ? (float)grad : -(float)grad;
    const float mi = b1 * m + (1.0f - b1) * g;
    const float vi = b2 * v + (1.0f - b2) * g * g;
    m = mi;
    v = vi;
    const float mh = mi / (1.0f - powf(b1, (float)step));
    const float vh = vi / (1.0f - powf(b2, (float)step));
    theta -= lr * mh / (sqrtf(vh) + eps);
}

// ---- complex helpers ---------------------------------------------------------------------

__device__ __forceinline__ void sincos_phase(float g_over_pi, float e, float& s, float& c) {
    // theta = gamma E = pi t with t = (gamma / pi) E. Periodicity: r = t - 2 rint(t / 2) lies in
    // [-1, 1] and is computed exactly (t and 2 rint(t/2) are within 1 of each other), so
    // theta' = pi r in [-pi, pi] has the same sine and cosine; the hardware sin/cos is then
    // evaluated on its accurate range (absolute error below 1e-6).
    const float t = g_over_pi * e;
    const float r = fmaf(-2.0f, rintf(0.5f * t), t);
    __sincosf(3.14159265358979323846f * r, &s, &c);
}
__device__ __forceinline__ void sincos_phase(double g_over_pi, double e, double& s, double& c) {
    sincospi(g_over_pi * e, &s, &c);
}

__device__ __forceinline__ void sincos_full(float x, float& s, float& c) { sincosf(x, &s, &c); }
__device__ __forceinline__ void sincos_full(double x, double& s, double& c) { sincos(x, &s, &c); }

// psi *= exp(-i theta) given (s, c) = (sin theta, cos theta)
template <typename C, typename T>
__device__ __forceinline__ void rot_neg(C& v, T s, T c) {
    const T r = v.x, i = v.y;
    v.x = r * c + i * s;
    v.y = i * c - r * s;
}

// ---- the rotated frame ----------------------------------------------------------------
// The kernels evolve psi~(z) = i^{|z|} psi(z) (|z| = number of set bits). This per-qubit
// diagonal change of basis D = diag(1, i) commutes with the cost phase (both diagonal), leaves
// every |amplitude|^2 unchanged bit for bit (it only swaps and negates components), and turns
// the mixer factor into a real rotation:
//   D exp(-i beta X) D^-1 = exp(-i beta Y) = [[cos b, -sin b], [sin b, cos b]],
// i.e. a' = c a - s b, b' = s a + c b applied identically to the real and imaginary parts.
// psi is converted back with (-i)^{|z|} only where a state leaves the library.

// Packed FP32 pair arithmetic (one instruction for both components).
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Mixer coefficients of one layer in the rotated frame.
template <typename T> struct RotCoef;
template <> struct RotCoef<float> {
    float2 cc, ss, ns;   // (c, c), (s, s), (-s, -s)
    __device__ __forceinline__ RotCoef(float c, float s)
        : cc(make_float2(c, c)), ss(make_float2(s, s)), ns(make_float2(-s, -s)) {}
};
template <> struct RotCoef<double> {
    double c, s;
    __device__ __forceinline__ RotCoef(double c_, double s_) : c(c_), s(s_) {}
};

// exp(-i beta X) on the pair (a, b) = (psi~[z], psi~[z | 2^q]) in the rotated frame.
__device__ __forceinline__ void butterfly(float2& a, float2& b, const RotCoef<float>& k) {
    const float2 t = mul2(b, k.ns);    // -s b
    const float2 u = mul2(a, k.ss);    //  s a
    a = fma2(a, k.cc, t);
    b = fma2(b, k.cc, u);
}
__device__ __forceinline__ void butterfly(double2& a, double2& b, const RotCoef<double>& k) {
    const double2 a0 = a, b0 = b;
    a.x = k.c * a0.x - k.s * b0.x;
    a.y = k.c * a0.y - k.s * b0.y;
    b.x = k.s * a0.x + k.c * b0.x;
    b.y = k.s * a0.y + k.c * b0.y;
}

// Unscaled shear form of the same rotation, used when |cos b| >= |sin b|:
//   [[c, -s], [s, c]] = c [[1, -t], [t, 1]],  t = tan b,
// so a' = a - t b, b' = b + t a (two packed FMAs per pair) and every qubit of the layer leaves
// a factor c that is applied once per amplitude (c^n) at the next cost phase or at the end.
__device__ __forceinline__ void butterfly_shear(float2& a, float2& b, float t) {
    const float2 a0 = a;
    a = fma2(b, make_float2(-t, -t), a);
    b = fma2(a0, make_float2(t, t), b);
}
__device__ __forceinline__ void butterfly_shear(double2& a, double2& b, double t) {
    const double2 a0 = a;
    a.x = fma(-t, b.x, a0.x);
    a.y = fma(-t, b.y, a0.y);
    b.x = fma(t, a0.x, b.x);
    b.y = fma(t, a0.y, b.y);
}

// Multiply by i^m (m mod 4): the frame change of an amplitude with m set bits. Branch-free
// (lanes of a warp usually have different m): i^m (x + iy) is (x, y), (-y, x), (-x, -y) or
// (y, -x).
template <typename C>
__device__ __forceinline__ C times_i_pow(C v, int m) {
    const int q = m & 3;
    const bool swap = q & 1;
    C r;
    r.x = swap ? v.y : v.x;
    r.y = swap ? v.x : v.y;
    if (q == 1 || q == 2) r.x = -r.x;
    if (q >= 2) r.y = -r.y;
    return r;
}

// Im(conj(x) * y) and Re(conj(x) * y)
template <typename C>
__device__ __forceinline__ auto im_conj_mul(const C& x, const C& y) -> decltype(x.x) {
    return x.x * y.y - x.y * y.x;
}
template <typename C>
__device__ __forceinline__ auto re_conj_mul(const C& x, const C& y) -> decltype(x.x) {
    return x.x * y.x + x.y * y.y;
}

// ---- warp reductions (fixed order: deterministic) ----------------------------------------

// Bitonic sort of one float per lane into descending order: lane l ends with the (l+1)-th
// largest value of the warp.
__device__ __forceinline__ float warp_sort_desc(float v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const float o = __shfl_xor_sync(0xffffffffu, v, stride);
            const bool asc = (lane & size) == 0;
            const bool lower = (lane & stride) == 0;
            v = (lower != asc) ? fminf(v, o) : fmaxf(v, o);
        }
    }
    return v;
}

// The k-th largest (k = 1..32) of one float per lane.
__device__ __forceinline__ float warp_kth_largest(float v, int k) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const float o = __shfl_xor_sync(0xffffffffu, v, stride);
            const bool asc = (lane & size) == 0;
            const bool lower = (lane & stride) == 0;
            v = (lower != asc) ? fminf(v, o) : fmaxf(v, o);
        }
    }
    return __shfl_sync(0xffffffffu, v, k - 1);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- top-k lists -------------------------------------------------------------------------
// A warp keeps one sorted list of k entries, entry l in lane l (lanes >= k hold no entry).
// Order: probability descending, then index ascending. Probabilities are exact FP64
// values of |psi|^2 computed from the stored amplitudes; candidates are pre-filtered in FP32
// against a threshold rounded down so that no entry that belongs in the list is skipped.

struct TopEnt {
    double p;
    uint32_t z;
};

// Probabilities are non-negative doubles (never -0: a sum of squares rounds to +0) and an empty
// entry holds -1. On those values the IEEE bit patterns, read as signed 64-bit integers, order
// exactly as the doubles do (every empty entry below every probability), so the list logic
// compares integers: GB300 issues FP64 at a small fraction of the integer rate.
__device__ __forceinline__ long long pbits(double p) { return __double_as_longlong(p); }
__device__ __forceinline__ bool is_entry(double p) { return pbits(p) >= 0; }

__device__ __forceinline__ bool better(double p1, uint32_t z1, double p2, uint32_t z2) {
    const long long a = pbits(p1), b = pbits(p2);
    return (a > b) || (a == b && z1 < z2);
}

// exact probability of a stored amplitude
__device__ __forceinline__ double exact_prob(float2 v) {
    // the products of two floats are exact in double; the one rounding is the final add
    return __dadd_rn(__dmul_rn((double)v.x, (double)v.x), __dmul_rn((double)v.y, (double)v.y));
}
__device__ __forceinline__ double exact_prob(double2 v) {
    return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y));
}

// The list length k (1..32) is a runtime value, warp-uniform.
struct WarpTopK {
    double p;          // this lane's entry (lane < k)
    uint32_t z;
    float thr_f;       // FP32 filter threshold (warp-uniform): max(list bound, boot)
    float boot;        // proven lower bound on the final k-th probability (raise_threshold)
    int k;

    __device__ __forceinline__ void init(int kk) {
        k = kk;
        p = -1.0;
        z = 0xffffffffu;
        thr_f = -1.0f;
        boot = -1.0f;
    }
    // Insert candidate (cp, cz) held by lane `src` if it beats the k-th entry (warp-uniform).
    __device__ __forceinline__ void insert_from(int src, double cp, uint32_t cz) {
        const int lane = threadIdx.x & 31;
        cp = __shfl_sync(0xffffffffu, cp, src);
        cz = __shfl_sync(0xffffffffu, cz, src);
        const bool b = (lane < k) && better(p, z, cp, cz);
        const uint32_t ball = __ballot_sync(0xffffffffu, b);
        const int pos = __popc(ball);      // entries better than the candidate form a prefix
        const double up_p = __shfl_up_sync(0xffffffffu, p, 1);
        const uint32_t up_z = __shfl_up_sync(0xffffffffu, z, 1);
        if (pos < k) {
            if (lane == pos) { p = cp; z = cz; }
            else if (lane > pos && lane < k) { p = up_p; z = up_z; }
        }
        const double kth = __shfl_sync(0xffffffffu, p, k - 1);
        thr_f = fmaxf(is_entry(kth) ? __double2float_rd(kth) : -1.0f, boot);
    }
    // Offer one amplitude per lane (all lanes call; lanes with valid == false offer nothing).
    template <typename C>
    __device__ __forceinline__ void offer(const C& v, uint32_t zi, bool valid) {
        const float pf = (float)v.x * (float)v.x + (float)v.y * (float)v.y;
        // |pf - P| <= 2^-21 P for the exact P, so P >= thr implies pf (1 + 2^-20) >= thr_f
        const bool cand = valid && (pf * 1.00000095367431640625f >= thr_f);
        uint32_t m = __ballot_sync(0xffffffffu, cand);
        if (!m) return;   // warp-uniform: the FP64 below runs only for warps with candidates
        double cp = -1.0;
        if (cand) cp = exact_prob(v);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            insert_from(src, cp, zi);
        }
    }
    // Raise the FP32 filter threshold to a value known to be <= the k-th largest probability
    // of the elements still to be offered (no list entry is changed).
    __device__ __forceinline__ void raise_threshold(float lower_bound) {
        boot = fmaxf(boot, lower_bound);
        thr_f = fmaxf(thr_f, boot);
    }
    // Offer an entry with a known exact probability (merging lists).
    __device__ __forceinline__ void offer_exact(double cp, uint32_t zi, bool valid) {
        uint32_t m = __ballot_sync(0xffffffffu, valid && is_entry(cp));
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            insert_from(src, cp, zi);
        }
    }
};

}  // namespace qaoa
