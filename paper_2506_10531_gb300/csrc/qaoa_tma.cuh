// qaoa_tma.cuh -- device helpers shared by the TMA-staged tiers of libqaoa (cluster streaming,
// k_cstream.cu; TMA streaming passes, k_tstream.cu): TMA tensor copies with mbarrier
// completion, bulk-store groups, proxy fences, the split cluster barrier, the 128-byte swizzle of
// a staged complex64 tile, and the reductions of a tile's final sub-pass (double-float block sum,
// top-k from each thread's 32 elements). Blocks of TMA_NT = 256 threads.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "qaoa_engine.cuh"

namespace qaoa {
namespace tma {

constexpr int TMA_NT = 256;

// Shared-memory index of tile index u in a TMA tile with the 128-byte swizzle (buffer aligned to
// 1024 bytes): amplitude u sits at byte 8u, whose bits 4..6 are XORed with bits 7..9.
__device__ __forceinline__ uint32_t psw(uint32_t u) { return u ^ ((u >> 3) & 14u); }

struct TmaLayout {
    __device__ __forceinline__ static uint32_t p(uint32_t u) { return psw(u); }   // amplitudes
    __device__ __forceinline__ static uint32_t e(uint32_t u) { return u; }        // energies
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
// L2 prefetch of a tile (no shared memory, no completion): a hint that can only change where the
// bytes are cached, never the values a later load reads
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(map), "r"(c0), "r"(c1),
                 "r"(c2)
                 : "memory");
}
__device__ __forceinline__ void tma_prefetch_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];\n" ::"l"(map), "r"(c0),
                 "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}
__device__ __forceinline__ void tma_prefetch_5d(const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4) {
    asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %2, %3, %4, %5}];\n" ::"l"(map), "r"(c0),
                 "r"(c1), "r"(c2), "r"(c3), "r"(c4)
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
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n"
        ::"r"(saddr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(saddr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                             int c3, int c4) {
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];\n"
                 ::"l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(saddr(src))
                 : "memory");
}
// the shared-memory sources of all but the most recent committed bulk store have been read
__device__ __forceinline__ void bulk_wait_read_all_but_one() {
    asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// the shared-memory sources of every committed bulk store have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// every committed bulk store has completed (its writes are visible to this thread)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// every committed bulk store but the most recent group has completed
__device__ __forceinline__ void bulk_wait_all_but_one() { asm volatile("cp.async.bulk.wait_group 1;\n" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the async proxy (before a TMA store)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// order global accesses of the generic and the async proxy (around the cluster hand-off)
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }
// split cluster barrier: arrive and wait (acquire), strictly alternating per thread. After a CTA
// barrier (which orders every write of the CTA before warp 0), warp 0 arrives with release
// semantics and the other warps arrive relaxed.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// Block sum of one FP32 value per thread in double-float arithmetic (each partial an unevaluated
// sum hi + lo of two floats, combined with Knuth's TwoSum), fixed order, returned to thread 0 as
// one FP64 value: about 44 bits of precision without the FP64 pipe, whose latency on this part
// would dominate a warp shuffle tree of FP64 adds. red: 2 * (TMA_NT / 32) floats.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ double block_sum_df(float v, float* red) {
    float hi = v, lo = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, oh, s, e);
        e += lo + ol;
        hi = s + e;
        lo = e - (hi - s);
    }
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { red[2 * w] = hi; red[2 * w + 1] = lo; }
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0) {
        float th = 0.0f, tl = 0.0f;
        for (int i = 0; i < TMA_NT / 32; ++i) {
            float s, e;
            two_sum(th, red[2 * i], s, e);
            e += tl + red[2 * i + 1];
            th = s + e;
            tl = e - (th - s);
        }
        tot = (double)th + (double)tl;
    }
    return tot;
}

// Top-k list of a tile whose amplitudes are in shared memory, given each thread's FP32
// probability maximum pmax over its own 32 elements elem(i) -> (shared index, global index):
// the bound is the k-th largest of the 256 thread maxima (k distinct elements are at least that
// probable, so the tile's k-th largest probability is not below it); every element that can
// reach it (FP32 test with the margins of WarpTopK::offer) goes to the candidate buffer with its
// exact FP64 probability, and the candidates are ranked (probability descending, index
// ascending). Returns false when the buffer overflowed (flat distributions); the caller then
// falls back to tile_topk. Called by all threads; result in ts.out.
template <typename Elem>
__device__ __forceinline__ bool topk_own(const float2* sp, int k, float pmax, Elem&& elem, const TileTopk& ts,
                                         float* wbound) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // (1) the k-th largest thread maximum of the tile: each warp offers its k largest (sorted),
    //     the k-th largest of those 8k values is found by rank
    const float srt = warp_sort_desc(pmax);
    if (lane < k) ts.wb[warp * k + lane] = srt;
    if (threadIdx.x == 0) { ts.cnt[0] = 0; ts.cnt[1] = 0; }
    __syncthreads();
    const int nl = (TMA_NT / 32) * k;   // a multiple of 8; ts.wb is 16-byte aligned
    if (threadIdx.x < (unsigned)nl) {
        const float me = ts.wb[threadIdx.x];
        const int t = (int)threadIdx.x;
        const float4* w4 = reinterpret_cast<const float4*>(ts.wb);
        int rank = 0;
#pragma unroll 4
        for (int q4 = 0; q4 < nl / 4; ++q4) {
            const float4 o = w4[q4];
            const int q = 4 * q4;
            rank += (o.x > me || (o.x == me && q < t)) ? 1 : 0;
            rank += (o.y > me || (o.y == me && q + 1 < t)) ? 1 : 0;
            rank += (o.z > me || (o.z == me && q + 2 < t)) ? 1 : 0;
            rank += (o.w > me || (o.w == me && q + 3 < t)) ? 1 : 0;
        }
        if (rank == k - 1) *wbound = me;
    }
    __syncthreads();
    const float bnd = *wbound;
    const float lo = bnd > 0.0f ? bnd * 0.99999904632568359375f : -1.0f;   // (1 - 2^-20)
    // (2) candidates: only threads whose maximum can reach the bound test their elements (all
    //     32 loads first, independent of one another, then the appends); a candidate is
    //     buffered with its amplitude (the slot's probability field holds the two floats) and
    //     its exact FP64 probability is formed afterwards, one thread per candidate, so that the
    //     slow FP64 pipe never runs in a serial per-thread chain
    if (pmax * 1.000003814697265625f >= lo) {
        uint32_t cm = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            uint32_t ix, z;
            elem(i, ix, z);
            const float2 v = sp[ix];
            const float pf = v.x * v.x + v.y * v.y;
            cm |= (pf * 1.00000095367431640625f >= lo) ? (1u << i) : 0u;
        }
        while (cm) {
            const int i = __ffs(cm) - 1;
            cm &= cm - 1u;
            uint32_t ix, z;
            elem(i, ix, z);
            const float2 v = sp[ix];
            const int pos = atomicAdd(&ts.cnt[0], 1);
            if (pos < TOPK_CAP) {
                ts.cand[pos].p = __hiloint2double(__float_as_int(v.y), __float_as_int(v.x));
                ts.cand[pos].z = z;
            } else {
                ts.cnt[1] = 1;
            }
        }
    }
    __syncthreads();
    if (ts.cnt[1]) return false;
    const int cnt = ts.cnt[0];
    for (int c = threadIdx.x; c < cnt; c += TMA_NT) {
        const double raw = ts.cand[c].p;
        ts.cand[c].p = exact_prob(make_float2(__int_as_float(__double2loint(raw)), __int_as_float(__double2hiint(raw))));
    }
    __syncthreads();
    // (3) rank selection (probability descending, index ascending: distinct ranks)
    for (int c = threadIdx.x; c < cnt; c += TMA_NT) {
        const TopEnt me = ts.cand[c];
        int rank = 0;
        for (int q = 0; q < cnt; ++q) {
            const TopEnt o = ts.cand[q];
            rank += better(o.p, o.z, me.p, me.z) ? 1 : 0;
        }
        if (rank < k) ts.out[rank] = me;
    }
    if (threadIdx.x < (unsigned)k && threadIdx.x >= (unsigned)cnt) ts.out[threadIdx.x] = TopEnt{-1.0, 0xffffffffu};
    __syncthreads();
    return true;
}


}  // namespace tma
}  // namespace qaoa
