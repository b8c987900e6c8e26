// qaoa_api.cu -- the C ABI of libqaoa (include/qaoa.h): argument validation, the context and
// its workspace, tier selection, batched launch plans, and the DQAOA host entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/qaoa.h"
#include "qaoa_common.cuh"
#include "qaoa_cstream.h"
#include "qaoa_host.h"
#include "qaoa_kernels.h"
#include "qaoa_stream.h"
#include "qaoa_tstream.h"

using namespace qaoa;

#include "qaoa_ctx.h"

namespace {

thread_local std::string g_err;

qaoa_status fail(qaoa_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

qaoa_status cuda_fail(cudaError_t e, const char* what) {
    return fail(QAOA_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

constexpr int NMAX = 30, PMAX = 64, KMAX = 16;

bool bad_nk(int n, int k) {
    return n < 1 || n > NMAX || k < 0 || k > KMAX || (uint64_t)k > (1ull << n);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Counter slot of a plan's header that holds its device status word (bit 0: a bounded wait ran out).
constexpr int PLAN_STATUS_SLOT = 62;

// Scratch of one streaming instance: per-tile <C> partials and top-k lists, laid out as
// [expect (nt doubles)] [probabilities (nt*k doubles)] [indices (nt*k uint32)], each 256-aligned.
size_t stream_scratch_bytes(bool dbl, int n, int k) {
    const int tb = stream_tile_bits(dbl);
    if (n <= tb) return 0;
    const size_t nt = (size_t)1 << (n - tb), kk = (size_t)std::max(k, 1);
    return align256(nt * sizeof(double)) + align256(nt * kk * sizeof(double)) +
           align256(nt * kk * sizeof(uint32_t));
}

// Scratch of the standalone reductions: the same three arrays for reduce_parts(n) blocks.
size_t reduce_scratch_bytes(int n) {
    const size_t parts = (size_t)reduce_parts(n);
    return align256(parts * sizeof(double)) + align256(parts * KMAX * sizeof(double)) +
           align256(parts * KMAX * sizeof(uint32_t));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Workspace of a streaming gradient: psi and lam (2^n complex each), the forward scratch and the
// per-pass, per-tile gradient partials of the adjoint plan (4 doubles).
size_t stream_grad_bytes(bool dbl, int n, int p) {
    const int tb = stream_tile_bits(dbl), tba = stream_adj_tile_bits(dbl);
    if (n <= tb) return 0;
    StreamPass tmp[256];
    const int S = stream_plan(dbl, n, p, 0, tmp, 256, tba);
    if (S < 0) return 0;
    const size_t D = (size_t)1 << n, nta = (size_t)1 << (n - tba), cs = dbl ? 16 : 8;
    return 2 * align256(D * cs) + stream_scratch_bytes(dbl, n, 0) + align256((size_t)S * nta * 4 * sizeof(double));
}

qaoa_status ensure_ws(qaoa_ctx* c, size_t bytes) {
    if (bytes <= c->ws_bytes) return QAOA_OK;
    return fail(QAOA_E_NOMEM, "workspace of %zu bytes needed, %zu reserved (call qaoa_reserve)",
                bytes, c->ws_bytes);
}

template <typename T>
bool is_dbl() { return sizeof(T) == 8; }

// ---- resident single instance ------------------------------------------------------------
template <typename T>
qaoa_status run_resident_one(qaoa_ctx* c, const InstDesc<T>& d, cudaStream_t st) {
    const bool dbl = is_dbl<T>();
    const bool grad = (d.flags & F_GRAD) != 0;
    // the descriptor travels by value as a kernel parameter
    CK(launch_resident(dbl, nullptr, 1, d.n, d.p, grad, nullptr, 1, st, &d));
    return QAOA_OK;
}

// ---- streaming single instance -----------------------------------------------------------
template <typename T>
qaoa_status run_stream_one(qaoa_ctx* c, int n, int p, const T* gamma, const T* beta, const T* E,
                           void* psi, bool init_plus, int k, double* expect, uint64_t* tidx,
                           double* tprob, size_t ws_off, cudaStream_t st) {
    const bool dbl = is_dbl<T>();
    if (!init_plus)
        return fail(QAOA_E_UNSUPPORTED, "streaming tier (n=%d) starts from |+> only", n);
    StreamPass passes[256];
    const int S = stream_plan(dbl, n, p, k, passes, 256);
    if (S < 0) return fail(QAOA_E_INVALID, "no streaming plan for n=%d p=%d", n, p);
    const int tb = stream_tile_bits(dbl);
    const uint64_t nt = 1ull << (n - tb);
    char* w = static_cast<char*>(c->ws) + ws_off;
    StreamInst<T> I{};
    I.p = p;
    I.amp0 = exp2(-0.5 * n);
    I.gamma = gamma;
    I.beta = beta;
    I.psi = psi;
    I.E = E;
    I.part_expect = reinterpret_cast<double*>(w);
    I.part_topp = reinterpret_cast<double*>(w + align256(nt * sizeof(double)));
    I.part_topz = reinterpret_cast<uint32_t*>(w + align256(nt * sizeof(double)) +
                                             align256(nt * std::max(k, 1) * sizeof(double)));
    I.expect = expect;
    I.topk_idx = tidx;
    I.topk_prob = tprob;
    const int grid = (int)std::min<uint64_t>(nt, (uint64_t)c->nsm * 2);
    for (int s = 0; s < S; ++s) CK(launch_stream_pass(dbl, passes[s], nullptr, 1, grid, st, &I));
    if (expect || (k > 0 && tidx)) CK(launch_stream_finalize(dbl, nullptr, 1, nt, k, st, &I));
    return QAOA_OK;
}

template <typename T>
qaoa_status grad_stream_one(qaoa_ctx* c, int n, int p, const T* gamma, const T* beta, const T* E,
                            double* expect, double* dgamma, double* dbeta, cudaStream_t st) {
    const bool dbl = is_dbl<T>();
    qaoa_status q = ensure_ws(c, stream_grad_bytes(dbl, n, p));
    if (q) return q;
    StreamPass passes[256];
    const int S = stream_plan(dbl, n, p, 0, passes, 256);
    if (S < 0) return fail(QAOA_E_INVALID, "no streaming plan for n=%d p=%d", n, p);
    passes[S - 1].keep_frame = 1;
    const int tb = stream_tile_bits(dbl);
    const uint64_t nt = 1ull << (n - tb), D = 1ull << n;
    const size_t cs = sizeof(typename qaoa::Num<T>::C);
    char* w = static_cast<char*>(c->ws);
    StreamInst<T> I{};
    I.p = p;
    I.amp0 = exp2(-0.5 * n);
    I.gamma = gamma;
    I.beta = beta;
    I.E = E;
    I.psi = w; w += align256(D * cs);
    I.lam = w; w += align256(D * cs);
    I.part_expect = reinterpret_cast<double*>(w);
    I.part_topp = reinterpret_cast<double*>(w + align256(nt * sizeof(double)));
    I.part_topz = reinterpret_cast<uint32_t*>(w + align256(nt * sizeof(double)) + align256(nt * sizeof(double)));
    w += stream_scratch_bytes(dbl, n, 0);
    I.part_grad = reinterpret_cast<double*>(w);
    I.expect = expect;
    I.dgamma = dgamma;
    I.dbeta = dbeta;
    StreamPass apasses[256];
    const int tba = stream_adj_tile_bits(dbl);
    const int SA = stream_plan(dbl, n, p, 0, apasses, 256, tba);
    if (SA < 0) return fail(QAOA_E_INVALID, "no adjoint plan for n=%d p=%d", n, p);
    const uint64_t nta = 1ull << (n - tba);
    const int grid = (int)std::min<uint64_t>(nt, (uint64_t)c->nsm * 2);
    const int agrid = (int)std::min<uint64_t>(nta, (uint64_t)c->nsm * 2);
    for (int s = 0; s < S; ++s) CK(launch_stream_pass(dbl, passes[s], nullptr, 1, grid, st, &I));
    if (expect) CK(launch_stream_finalize(dbl, nullptr, 1, nt, 0, st, &I));
    for (int s = SA - 1; s >= 0; --s)
        CK(launch_stream_adj_pass(dbl, apasses[s], s, s == SA - 1, s > 0, nullptr, 1, agrid, st, &I));
    CK(launch_stream_grad_reduce(dbl, apasses, SA, nullptr, 1, nta, st, &I));
    return QAOA_OK;
}

template <typename T>
qaoa_status build_energies_t(qaoa_ctx* c, int n, const T* Q, T* E, qaoa_stream_t stream) {
    if (!c) return fail(QAOA_E_INVALID, "ctx is NULL");
    if (n < 1 || n > NMAX || !Q || !E) return fail(QAOA_E_INVALID, "build_energies: bad n or NULL");
    CK(launch_energy(is_dbl<T>(), n, Q, E, (cudaStream_t)stream));
    return QAOA_OK;
}

template <typename T>
qaoa_status run_layers_t(qaoa_ctx* c, int n, int p, const T* gamma, const T* beta, const T* E,
                         void* psi, int init_plus, qaoa_stream_t stream) {
    if (!c) return fail(QAOA_E_INVALID, "ctx is NULL");
    if (n < 1 || n > NMAX || p < 1 || p > PMAX || !gamma || !beta || !E || !psi)
        return fail(QAOA_E_INVALID, "run_layers: n=%d p=%d or NULL pointer", n, p);
    if (!aligned16(psi)) return fail(QAOA_E_INVALID, "run_layers: psi must be 16-byte aligned");
    const bool dbl = is_dbl<T>();
    cudaStream_t st = (cudaStream_t)stream;
    if (n <= (dbl ? RES_NMAX_D : RES_NMAX_F)) {
        InstDesc<T> d{};
        d.n = n; d.p = p; d.k = 0; d.flags = init_plus ? 0 : F_INIT_PSI;
        d.E_in = E; d.gamma = gamma; d.beta = beta;
        d.psi_in = psi; d.psi_out = psi;
        return run_resident_one<T>(c, d, st);
    }
    qaoa_status s = ensure_ws(c, stream_scratch_bytes(dbl, n, 0));
    if (s) return s;
    return run_stream_one<T>(c, n, p, gamma, beta, E, psi, init_plus != 0, 0, nullptr, nullptr,
                             nullptr, 0, st);
}

template <typename T>
qaoa_status reduce_t(qaoa_ctx* c, int n, const void* psi, const T* E, int k, double* expect,
                     uint64_t* idx, double* prob, qaoa_stream_t stream) {
    if (!c) return fail(QAOA_E_INVALID, "ctx is NULL");
    if (bad_nk(n, k) || !psi) return fail(QAOA_E_INVALID, "reduce: bad n/k or NULL psi");
    qaoa_status s = ensure_ws(c, reduce_scratch_bytes(n));
    if (s) return s;
    const int parts = reduce_parts(n);
    char* w = static_cast<char*>(c->ws);
    double* pe = reinterpret_cast<double*>(w);
    double* pp = reinterpret_cast<double*>(w + align256(parts * sizeof(double)));
    uint32_t* pz = reinterpret_cast<uint32_t*>(w + align256(parts * sizeof(double)) +
                                               align256((size_t)parts * KMAX * sizeof(double)));
    CK(launch_reduce_state(is_dbl<T>(), n, psi, E, k, pe, pp, pz, expect, idx, prob,
                           (cudaStream_t)stream));
    return QAOA_OK;
}

template <typename T>
qaoa_status grad_t(qaoa_ctx* c, int n, int p, const T* gamma, const T* beta, const T* E,
                   double* expect, double* dgamma, double* dbeta, qaoa_stream_t stream) {
    if (!c) return fail(QAOA_E_INVALID, "ctx is NULL");
    if (n < 1 || n > NMAX || p < 1 || p > PMAX || !gamma || !beta || !E || !dgamma || !dbeta)
        return fail(QAOA_E_INVALID, "grad: n=%d p=%d or NULL pointer", n, p);
    const bool dbl = is_dbl<T>();
    if (n > (dbl ? RES_NMAX_D_ADJ : RES_NMAX_F_ADJ))
        return grad_stream_one<T>(c, n, p, gamma, beta, E, expect, dgamma, dbeta, (cudaStream_t)stream);
    InstDesc<T> d{};
    d.n = n; d.p = p; d.k = 0; d.flags = F_GRAD;
    d.E_in = E; d.gamma = gamma; d.beta = beta;
    d.expect = expect; d.dgamma = dgamma; d.dbeta = dbeta;
    return run_resident_one<T>(c, d, (cudaStream_t)stream);
}

}  // namespace

qaoa_status qaoa::report(qaoa_status s, const char* msg) { return fail(s, "%s", msg); }

// =============================================================================================
// Context
// =============================================================================================

extern "C" qaoa_status qaoa_create(qaoa_ctx** out, int device) {
    if (!out) return fail(QAOA_E_INVALID, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(QAOA_E_INVALID, "device %d of %d", device, ndev);
    CK(cudaSetDevice(device));
    qaoa_ctx* c = new qaoa_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaMalloc(&c->queue, 256);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaMalloc(queue)"); }
    c->ws_bytes = 1 << 20;
    e = cudaMalloc(&c->ws, c->ws_bytes);
    if (e != cudaSuccess) { cudaFree(c->queue); delete c; return cuda_fail(e, "cudaMalloc(ws)"); }
    *out = c;
    return QAOA_OK;
}

extern "C" void qaoa_destroy(qaoa_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    cudaFree(c->ws);
    cudaFree(c->queue);
    delete c;
}

extern "C" const char* qaoa_last_error(void) { return g_err.c_str(); }

extern "C" qaoa_status qaoa_reserve(qaoa_ctx* c, size_t bytes) {
    if (!c) return fail(QAOA_E_INVALID, "ctx is NULL");
    bytes = align256(bytes);
    if (bytes <= c->ws_bytes) return QAOA_OK;
    CK(cudaSetDevice(c->device));
    CK(cudaDeviceSynchronize());
    void* nw = nullptr;
    cudaError_t e = cudaMalloc(&nw, bytes);
    if (e != cudaSuccess) return fail(QAOA_E_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    cudaFree(c->ws);
    c->ws = nw;
    c->ws_bytes = bytes;
    return QAOA_OK;
}

extern "C" qaoa_status qaoa_set_tier(qaoa_ctx* c, int n, int tier, int param) {
    if (!c || n < 1 || n > NMAX) return fail(QAOA_E_INVALID, "set_tier: bad ctx or n");
    if (tier == QAOA_TIER_AUTO) { c->tier[n] = 0; c->cluster_L[n] = 0; return QAOA_OK; }
    if (tier == QAOA_TIER_RESIDENT) {
        if (n > RES_NMAX_F || !(param == 0 || (param == 4 && n <= 13) || param == 5))
            return fail(QAOA_E_INVALID, "set_tier: resident needs n <= %d and a window of 5 qubits, or 4 for n <= 13 "
                        "(0: default)", RES_NMAX_F);
        c->tier[n] = tier;
        c->cluster_L[n] = param;
        return QAOA_OK;
    }
    if (tier == QAOA_TIER_STREAM) {
        if (n <= RES_NMAX_F) return fail(QAOA_E_INVALID, "set_tier: n=%d is always resident", n);
        if (param < 0 || param > 2) return fail(QAOA_E_INVALID, "set_tier: streaming variant %d (0..2)", param);
        c->tier[n] = tier;
        c->cluster_L[n] = param;
        return QAOA_OK;
    }
    if (tier == QAOA_TIER_CSTREAM) {
        if (n < CS_NMIN || n > CS_NMAX) return fail(QAOA_E_INVALID, "set_tier: cluster streaming needs 15 <= n <= 17");
        if (!cstream_usable(c, n))
            return fail(QAOA_E_UNSUPPORTED, "set_tier: the cluster-streaming tier cannot run n=%d on this device", n);
        c->tier[n] = tier;
        return QAOA_OK;
    }
    if (tier == QAOA_TIER_CLUSTER) {
        if (n < CL_NMIN || n > CL_NMAX || param < 10 || param > 14 || n - param < 1 || n - param > 4)
            return fail(QAOA_E_INVALID, "set_tier: cluster needs 15 <= n <= 18 and 1 <= n - L <= 4");
        c->tier[n] = tier;
        c->cluster_L[n] = param;
        return QAOA_OK;
    }
    return fail(QAOA_E_INVALID, "set_tier: unknown tier %d", tier);
}

extern "C" size_t qaoa_workspace_bytes(int n, int dbl) {
    if (n < 1 || n > NMAX) return 0;
    return std::max({stream_scratch_bytes(dbl != 0, n, KMAX), reduce_scratch_bytes(n),
                     stream_grad_bytes(dbl != 0, n, PMAX)});
}

// =============================================================================================
// Single-instance calls
// =============================================================================================

extern "C" qaoa_status qaoa_build_energies(qaoa_ctx* c, int n, const float* Q, float* E, qaoa_stream_t s) {
    return build_energies_t<float>(c, n, Q, E, s);
}
extern "C" qaoa_status qaoa_build_energies_z(qaoa_ctx* c, int n, const double* Q, double* E, qaoa_stream_t s) {
    return build_energies_t<double>(c, n, Q, E, s);
}
extern "C" qaoa_status qaoa_run_layers(qaoa_ctx* c, int n, int p, const float* g, const float* b,
                                       const float* E, void* psi, int init_plus, qaoa_stream_t s) {
    return run_layers_t<float>(c, n, p, g, b, E, psi, init_plus, s);
}
extern "C" qaoa_status qaoa_run_layers_z(qaoa_ctx* c, int n, int p, const double* g, const double* b,
                                         const double* E, void* psi, int init_plus, qaoa_stream_t s) {
    return run_layers_t<double>(c, n, p, g, b, E, psi, init_plus, s);
}
extern "C" qaoa_status qaoa_expect(qaoa_ctx* c, int n, const void* psi, const float* E, double* out,
                                   qaoa_stream_t s) {
    if (!E || !out) return fail(QAOA_E_INVALID, "expect: NULL E or out");
    return reduce_t<float>(c, n, psi, E, 0, out, nullptr, nullptr, s);
}
extern "C" qaoa_status qaoa_expect_z(qaoa_ctx* c, int n, const void* psi, const double* E, double* out,
                                     qaoa_stream_t s) {
    if (!E || !out) return fail(QAOA_E_INVALID, "expect: NULL E or out");
    return reduce_t<double>(c, n, psi, E, 0, out, nullptr, nullptr, s);
}
extern "C" qaoa_status qaoa_topk(qaoa_ctx* c, int n, const void* psi, int k, uint64_t* idx, double* prob,
                                 qaoa_stream_t s) {
    if (k < 1 || !idx) return fail(QAOA_E_INVALID, "topk: k=%d or NULL idx", k);
    return reduce_t<float>(c, n, psi, (const float*)nullptr, k, nullptr, idx, prob, s);
}
extern "C" qaoa_status qaoa_topk_z(qaoa_ctx* c, int n, const void* psi, int k, uint64_t* idx, double* prob,
                                   qaoa_stream_t s) {
    if (k < 1 || !idx) return fail(QAOA_E_INVALID, "topk: k=%d or NULL idx", k);
    return reduce_t<double>(c, n, psi, (const double*)nullptr, k, nullptr, idx, prob, s);
}
extern "C" qaoa_status qaoa_sample(qaoa_ctx* c, int n, const void* psi, int64_t shots, const double* u,
                                   uint64_t* out, qaoa_stream_t s) {
    if (!c) return fail(QAOA_E_INVALID, "ctx is NULL");
    if (n < 1 || n > 30 || !psi || shots < 0 || shots > ((int64_t)1 << 26) || (shots > 0 && (!u || !out)))
        return fail(QAOA_E_INVALID, "sample: n=%d shots=%lld or NULL pointer", n, (long long)shots);
    qaoa_status st = ensure_ws(c, sample_scratch_bytes(n));
    if (st) return st;
    CK(launch_sample(n, psi, 1, shots, u, out, static_cast<double*>(c->ws), (cudaStream_t)s));
    return QAOA_OK;
}
extern "C" qaoa_status qaoa_grad(qaoa_ctx* c, int n, int p, const float* g, const float* b, const float* E,
                                 double* ex, double* dg, double* db, qaoa_stream_t s) {
    return grad_t<float>(c, n, p, g, b, E, ex, dg, db, s);
}
extern "C" qaoa_status qaoa_grad_z(qaoa_ctx* c, int n, int p, const double* g, const double* b,
                                   const double* E, double* ex, double* dg, double* db, qaoa_stream_t s) {
    return grad_t<double>(c, n, p, g, b, E, ex, dg, db, s);
}

// =============================================================================================
// Batched plans
// =============================================================================================

struct qaoa_plan {
    qaoa_ctx* ctx = nullptr;
    bool dbl = false;
    void* dev = nullptr;          // one device block: counters and descriptors, then scratch
    size_t dev_bytes = 0;
    bool owns = true;             // dev was allocated by the plan (else caller memory)
    cudaGraphExec_t graph = nullptr;  // captured launch sequence (qaoa_plan_capture)
    struct ResGroup { int n, pmax, count; bool grad; size_t desc_off; int grid; int q_slot; int rmax; };
    struct CluGroup { int n, L, pmax, count; size_t desc_off; int clusters; };
    struct CsGroup { int n, count; size_t desc_off; int clusters; };
    struct StrGroup { int n, p, k, count; bool grad; size_t inst_off; std::vector<StreamPass> passes;
                      std::vector<StreamPass> apasses;   // adjoint plan (adjoint tile bits)
                      int grid, agrid; std::vector<const void*> q; std::vector<void*> e;
                      // TMA streaming passes (complex64): per instance one state tensor map per
                      // pass shape, at maps_off in the header; tsp[i] is pass i's geometry
                      bool tma = false; size_t maps_off = 0; int maps_per_inst = 0; std::vector<TsPass> tsp;
                      int tgrid = 0;   // TMA passes' persistent grid
                      // TMA adjoint passes: per instance three maps (psi, lam, E) per adjoint pass
                      // shape at amaps_off; atsp[i] is adjoint pass i's geometry
                      bool tadj = false; size_t amaps_off = 0; int amaps_per_inst = 0; std::vector<TsPass> atsp; };
    std::vector<ResGroup> res;
    std::vector<CluGroup> clu;
    std::vector<CsGroup> cs;
    std::vector<StrGroup> str;
    int kernels = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev;       // 2 per kernel of one launch
    std::vector<const char*> names;    // kernel family per kernel of the last launch
    std::vector<double> bytes;         // algorithmic DRAM bytes per kernel, launch order
};

namespace {

// Caller-provided placement of a plan: the device block lives in [base, base + bytes) and the
// descriptor header is uploaded asynchronously on `st` from the pinned host buffer `staging`
// (staging_bytes), which must stay untouched until that copy has run.
struct PlanMem {
    void* base;
    size_t bytes;
    cudaStream_t st;
    void* staging;
    size_t staging_bytes;
};

template <typename T>
qaoa_status plan_create_t(qaoa_ctx* c, const qaoa_inst* desc, int count, const qaoa_batch_io* io,
                          const PlanMem* mem, qaoa_plan** out, size_t* need = nullptr) {
    using C2 = typename qaoa::Num<T>::C;
    const bool dbl = is_dbl<T>();
    const T* qpool = static_cast<const T*>(io->q);
    const T* ppool = static_cast<const T*>(io->params);
    C2* psipool = static_cast<C2*>(io->psi);
    T* epool = static_cast<T*>(io->e);
    // validate
    for (int i = 0; i < count; ++i) {
        const qaoa_inst& d = desc[i];
        if (bad_nk(d.n, d.k) || d.p < 1 || d.p > PMAX || d.q_off < 0 || d.par_off < 0)
            return fail(QAOA_E_INVALID, "instance %d: n=%d p=%d k=%d offsets %lld %lld", i, d.n, d.p,
                        d.k, (long long)d.q_off, (long long)d.par_off);
        if (d.k > 0 && (!io->topk_idx || io->k_stride < d.k))
            return fail(QAOA_E_INVALID, "instance %d: top-k output missing or k_stride < k", i);
        if (d.psi_off >= 0 && !io->psi) return fail(QAOA_E_INVALID, "instance %d: psi pool NULL", i);
        if (d.psi_off >= 0 && !aligned16(static_cast<const C2*>(io->psi) + d.psi_off))
            return fail(QAOA_E_INVALID, "instance %d: state at psi_off must be 16-byte aligned", i);
        if (d.e_off >= 0 && !io->e) return fail(QAOA_E_INVALID, "instance %d: energy pool NULL", i);
        if (d.e_off >= 0 && (reinterpret_cast<uintptr_t>(static_cast<const T*>(io->e) + d.e_off) & 7u) != 0)
            return fail(QAOA_E_INVALID, "instance %d: energies at e_off must be 8-byte aligned", i);
        if ((d.flags & QAOA_INST_GRAD) && !io->grad) return fail(QAOA_E_INVALID, "instance %d: grad pool NULL", i);
        if ((d.flags & QAOA_INST_GRAD) && d.n > (dbl ? RES_NMAX_D_ADJ : RES_NMAX_F_ADJ) && d.psi_off >= 0)
            return fail(QAOA_E_UNSUPPORTED, "instance %d: the final state is returned with a gradient only for n <= %d",
                        i, dbl ? RES_NMAX_D_ADJ : RES_NMAX_F_ADJ);
    }
    qaoa_plan* P = new qaoa_plan();
    P->ctx = c;
    P->dbl = dbl;
    // group: resident by (n, grad); streaming by (n, p, k)
    std::map<std::pair<int, int>, std::vector<int>> rg;
    std::map<std::pair<int, int>, std::vector<int>> cg;   // cluster groups by (n, local qubits)
    std::map<int, std::vector<int>> csg;                   // cluster-streaming groups by n
    std::map<std::tuple<int, int, int, int>, std::vector<int>> sg;
    const int nres = dbl ? RES_NMAX_D : RES_NMAX_F;
    const int nres_adj = dbl ? RES_NMAX_D_ADJ : RES_NMAX_F_ADJ;
    for (int i = 0; i < count; ++i) {
        const qaoa_inst& d = desc[i];
        const bool grad = (d.flags & QAOA_INST_GRAD) != 0;
        const int tier = (!dbl && !grad) ? qaoa::eff_tier(c, d.n, d.p) : QAOA_TIER_STREAM;
        // the cluster-streaming tier moves the energies by TMA: an energy output must be 16-byte aligned
        const bool e_ok = d.e_off < 0 || (reinterpret_cast<uintptr_t>(epool + d.e_off) & 15u) == 0;
        if (d.n <= nres && (!grad || d.n <= nres_adj)) rg[{d.n, grad ? 1 : 0}].push_back(i);
        else if (tier == QAOA_TIER_CSTREAM && d.n >= CS_NMIN && d.n <= CS_NMAX && e_ok && cstream_usable(c, d.n))
            csg[d.n].push_back(i);
        else if (!dbl && !grad && d.n >= CL_NMIN && d.n <= CL_NMAX && tier == QAOA_TIER_CLUSTER)
            cg[{d.n, qaoa::eff_cluster_L(c, d.n, d.p)}].push_back(i);
        else sg[{d.n, d.p, d.k, grad ? 1 : 0}].push_back(i);
    }
    auto make_desc = [&](int i) {
        const qaoa_inst& d = desc[i];
        InstDesc<T> x{};
        x.n = d.n; x.p = d.p; x.k = d.k;
        x.flags = (d.flags & QAOA_INST_GRAD) ? F_GRAD : 0;
        x.Q = qpool + d.q_off;
        x.gamma = ppool + d.par_off;
        x.beta = ppool + d.par_off + d.p;
        x.psi_out = d.psi_off >= 0 ? (void*)(psipool + d.psi_off) : nullptr;
        x.E_out = d.e_off >= 0 ? epool + d.e_off : nullptr;
        x.expect = io->expect ? io->expect + i : nullptr;
        x.topk_idx = d.k > 0 ? io->topk_idx + (int64_t)i * io->k_stride : nullptr;
        x.topk_prob = (d.k > 0 && io->topk_prob) ? io->topk_prob + (int64_t)i * io->k_stride : nullptr;
        x.dgamma = (x.flags & F_GRAD) ? io->grad + d.par_off : nullptr;
        x.dbeta = (x.flags & F_GRAD) ? io->grad + d.par_off + d.p : nullptr;
        return x;
    };
    // layout: header (256 bytes of counters, then every descriptor array) and scratch (the
    // per-instance buffers of the streaming tier); scratch offsets are relative to its start
    size_t hdr = 256, scr = 0;
    std::vector<InstDesc<T>> rdesc;
    int qslot = 0;
    for (auto& kv : rg) {
        qaoa_plan::ResGroup g{};
        g.n = kv.first.first;
        g.grad = kv.first.second != 0;
        g.count = (int)kv.second.size();
        g.pmax = 1;
        g.desc_off = hdr;
        g.q_slot = qslot++;
        for (int i : kv.second) {
            const qaoa_inst& d = desc[i];
            g.pmax = std::max(g.pmax, d.p);
            rdesc.push_back(make_desc(i));
        }
        hdr = align256(hdr + sizeof(InstDesc<T>) * g.count);
        g.rmax = dbl ? RES_RMAX : eff_resident_rmax(c, g.n, g.pmax);
        const int occ = std::max(1, resident_max_blocks_per_sm(dbl, g.n, g.pmax, g.grad, g.rmax));
        g.grid = std::min(g.count, occ * c->nsm);
        P->res.push_back(g);
    }
    std::vector<InstDesc<T>> cdesc;
    for (auto& kv : cg) {
        qaoa_plan::CluGroup g{};
        g.n = kv.first.first;
        g.L = kv.first.second;
        g.count = (int)kv.second.size();
        g.pmax = 1;
        g.desc_off = hdr;
        for (int i : kv.second) {
            g.pmax = std::max(g.pmax, desc[i].p);
            cdesc.push_back(make_desc(i));
        }
        hdr = align256(hdr + sizeof(InstDesc<T>) * g.count);
        int mc = 0;
        cudaError_t e = launch_cluster(nullptr, 0, g.n, g.L, g.pmax, 0, nullptr, &mc);
        if (e != cudaSuccess || mc < 1) {
            delete P;
            return fail(QAOA_E_UNSUPPORTED, "no cluster of %d CTAs with %zu B shared memory fits (n=%d): %s",
                        1 << (g.n - g.L), cluster_smem_bytes(g.n, g.L, g.pmax), g.n, cudaGetErrorString(e));
        }
        g.clusters = std::min(g.count, mc);
        P->clu.push_back(g);
    }
    // cluster-streaming: descriptors, then four tensor maps per instance (64-byte aligned);
    // per-instance state and energies in the scratch unless the caller receives them
    struct CsI { size_t psi_off, e_off; };
    std::vector<std::vector<CsI>> csinfo;
    std::vector<size_t> cs_maps_off;
    for (auto& kv : csg) {
        qaoa_plan::CsGroup g{};
        g.n = kv.first;
        g.count = (int)kv.second.size();
        g.desc_off = hdr;
        hdr = align256(hdr + cstream_inst_bytes() * g.count);
        cs_maps_off.push_back(hdr);
        hdr = align256(hdr + CS_MAPS_BYTES * g.count);
        int mc = 0;
        cstream_max_clusters(g.n, &mc);
        g.clusters = std::max(1, std::min(g.count, mc));
        std::vector<CsI> v;
        const size_t D = (size_t)1 << g.n;
        for (int i : kv.second) {
            CsI x{};
            x.psi_off = (desc[i].psi_off >= 0) ? (size_t)-1 : scr;
            if (desc[i].psi_off < 0) scr = align256(scr + D * sizeof(C2));
            x.e_off = (desc[i].e_off >= 0) ? (size_t)-1 : scr;
            if (desc[i].e_off < 0) scr = align256(scr + D * sizeof(T));
            v.push_back(x);
        }
        csinfo.push_back(v);
        P->cs.push_back(g);
    }
    if (qslot > 60) { delete P; return fail(QAOA_E_UNSUPPORTED, "too many resident groups"); }
    // streaming: per instance its own E / psi / partial buffers inside the plan block
    struct SI { size_t e_off, psi_off, part_off, lam_off, grad_off; };
    std::vector<std::vector<SI>> sinfo;
    const int tb = stream_tile_bits(dbl), tba = stream_adj_tile_bits(dbl);
    for (auto& kv : sg) {
        qaoa_plan::StrGroup g{};
        g.n = std::get<0>(kv.first);
        g.p = std::get<1>(kv.first);
        g.k = std::get<2>(kv.first);
        g.grad = std::get<3>(kv.first) != 0;
        g.count = (int)kv.second.size();
        StreamPass tmp[256];
        const int S = stream_plan(dbl, g.n, g.p, g.k, tmp, 256);
        if (S < 0) { delete P; return fail(QAOA_E_INVALID, "no streaming plan for n=%d p=%d", g.n, g.p); }
        if (g.grad) tmp[S - 1].keep_frame = 1;
        // the final state is written back only when an instance of the group returns it
        bool any_psi = false;
        for (int i : kv.second) any_psi = any_psi || desc[i].psi_off >= 0;
        if (!g.grad && !any_psi) tmp[S - 1].no_store = 1;
        g.passes.assign(tmp, tmp + S);
        int SA = 0;
        if (g.grad) {
            StreamPass atmp[256];
            SA = stream_plan(dbl, g.n, g.p, 0, atmp, 256, tba);
            if (SA < 0) { delete P; return fail(QAOA_E_INVALID, "no adjoint plan for n=%d p=%d", g.n, g.p); }
            g.apasses.assign(atmp, atmp + SA);
        }
        const uint64_t nta = 1ull << (g.n - tba);
        g.inst_off = hdr;
        hdr = align256(hdr + sizeof(StreamInst<T>) * g.count);
        const int variant = dbl ? 2 : eff_stream_variant(c, g.n, g.p);
        g.tgrid = (variant == 1 ? 1 : 2) * c->nsm;
        if (!dbl && variant != 2 && tstream_available()) {
            // map 0: the kind-A passes; map 1 + b: the kind-B passes of chunk b (by start qubit)
            std::vector<int> chunk_s;
            for (auto& ps : g.passes)
                if (ps.kind == 1 && std::find(chunk_s.begin(), chunk_s.end(), ps.s) == chunk_s.end())
                    chunk_s.push_back(ps.s);
            std::sort(chunk_s.begin(), chunk_s.end());
            g.tma = true;
            const int nshape = 1 + (int)chunk_s.size();   // state maps, then the energy maps
            g.maps_per_inst = 2 * nshape;
            for (auto& ps : g.passes) {
                const int mi = ps.kind == 0 ? 0
                                            : 1 + (int)(std::find(chunk_s.begin(), chunk_s.end(), ps.s) - chunk_s.begin());
                g.tsp.push_back(tstream_pass_geometry(ps, mi, nshape + mi, g.maps_per_inst));
            }
            g.maps_off = hdr;
            hdr = align256(hdr + TS_MAP_BYTES * (size_t)g.maps_per_inst * g.count);
            if (g.grad && tba == TSA_TB) {
                // adjoint shapes: kind A, then the kind-B chunks of the adjoint plan by start qubit
                std::vector<int> achunk;
                for (auto& ps : g.apasses)
                    if (ps.kind == 1 && std::find(achunk.begin(), achunk.end(), ps.s) == achunk.end())
                        achunk.push_back(ps.s);
                std::sort(achunk.begin(), achunk.end());
                g.amaps_per_inst = 3 * (1 + (int)achunk.size());
                for (auto& ps : g.apasses) {
                    const int ai = ps.kind == 0 ? 0
                                                : 1 + (int)(std::find(achunk.begin(), achunk.end(), ps.s) - achunk.begin());
                    g.atsp.push_back(tstream_adj_geometry(ps, 3 * ai, g.amaps_per_inst));
                }
                g.amaps_off = hdr;
                hdr = align256(hdr + TS_MAP_BYTES * (size_t)g.amaps_per_inst * g.count);
                g.tadj = true;
            }
        }
        std::vector<SI> v;
        const uint64_t D = 1ull << g.n, nt = 1ull << (g.n - tb);
        for (int i : kv.second) {
            SI s{};
            const qaoa_inst& d = desc[i];
            s.e_off = (d.e_off >= 0) ? (size_t)-1 : scr;
            if (d.e_off < 0) scr = align256(scr + D * sizeof(T));
            s.psi_off = (d.psi_off >= 0) ? (size_t)-1 : scr;
            if (d.psi_off < 0) scr = align256(scr + D * sizeof(C2));
            s.part_off = scr;
            scr = align256(scr + nt * sizeof(double));
            scr = align256(scr + nt * std::max(g.k, 1) * sizeof(double));
            scr = align256(scr + nt * std::max(g.k, 1) * sizeof(uint32_t));
            s.lam_off = s.grad_off = 0;
            if (g.grad) {
                s.lam_off = scr;
                scr = align256(scr + D * sizeof(C2));
                s.grad_off = scr;
                scr = align256(scr + (size_t)SA * nta * 4 * sizeof(double));
            }
            v.push_back(s);
        }
        const uint64_t tiles = nt * (uint64_t)g.count;
        g.grid = (int)std::min<uint64_t>(tiles, (uint64_t)c->nsm * 2);
        g.agrid = (int)std::min<uint64_t>(nta * (uint64_t)g.count, (uint64_t)c->nsm * 2);
        sinfo.push_back(v);
        P->str.push_back(std::move(g));
    }
    const size_t sbase = align256(hdr);
    const size_t bytes = sbase + scr;
    if (need) *need = bytes;
    cudaError_t e = cudaSuccess;
    if (mem) {
        if (bytes > mem->bytes || (mem->staging && sbase > mem->staging_bytes)) {
            delete P;
            return fail(QAOA_E_NOMEM, "plan needs %zu bytes (%zu of header), %zu / %zu provided", bytes, sbase,
                        mem->bytes, mem->staging_bytes);
        }
        P->dev = mem->base;
        P->owns = false;
    } else {
        e = cudaMalloc(&P->dev, bytes);
        if (e != cudaSuccess) { delete P; return fail(QAOA_E_NOMEM, "plan cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e)); }
    }
    P->dev_bytes = bytes;
    char* base = static_cast<char*>(P->dev);
    char* sb = base + sbase;
    // host image of the header: zero counters, then the descriptor arrays
    std::vector<char> img(sbase, 0);
    size_t ri = 0;
    for (auto& g : P->res) {
        std::memcpy(img.data() + g.desc_off, rdesc.data() + ri, sizeof(InstDesc<T>) * g.count);
        ri += g.count;
        P->kernels += 2;  // memset counter + kernel
    }
    size_t ci = 0;
    for (auto& g : P->clu) {
        std::memcpy(img.data() + g.desc_off, cdesc.data() + ci, sizeof(InstDesc<T>) * g.count);
        ci += g.count;
        P->kernels += 1;
    }
    {
        size_t gi = 0;
        for (auto& kv : csg) {
            auto& g = P->cs[gi];
            size_t j = 0;
            for (int i : kv.second) {
                const qaoa_inst& d = desc[i];
                const CsI& x = csinfo[gi][j];
                void* psi = (x.psi_off == (size_t)-1) ? (void*)(psipool + d.psi_off) : (void*)(sb + x.psi_off);
                void* E = (x.e_off == (size_t)-1) ? (void*)(epool + d.e_off) : (void*)(sb + x.e_off);
                const size_t moff = cs_maps_off[gi] + CS_MAPS_BYTES * j;
                if (!cstream_encode_maps(d.n, psi, E, img.data() + moff)) {
                    if (P->owns) cudaFree(P->dev);
                    delete P;
                    return fail(QAOA_E_CUDA, "instance %d: tensor maps of the cluster-streaming tier refused", i);
                }
                cstream_fill_inst(img.data() + g.desc_off + cstream_inst_bytes() * j, d.n, d.p, d.k,
                                  d.psi_off >= 0, reinterpret_cast<const float*>(qpool + d.q_off),
                                  reinterpret_cast<const float*>(ppool + d.par_off),
                                  reinterpret_cast<const float*>(ppool + d.par_off + d.p),
                                  io->expect ? io->expect + i : nullptr,
                                  d.k > 0 ? io->topk_idx + (int64_t)i * io->k_stride : nullptr,
                                  (d.k > 0 && io->topk_prob) ? io->topk_prob + (int64_t)i * io->k_stride : nullptr,
                                  base + moff);
                ++j;
            }
            P->kernels += 1;
            ++gi;
        }
    }
    // build streaming instances
    size_t gi = 0;
    for (auto& kv : sg) {
        auto& g = P->str[gi];
        std::vector<StreamInst<T>> si;
        const uint64_t nt = 1ull << (g.n - tb);
        size_t j = 0;
        for (int i : kv.second) {
            const qaoa_inst& d = desc[i];
            const SI& s = sinfo[gi][j++];
            StreamInst<T> I{};
            I.p = d.p;
            I.amp0 = exp2(-0.5 * d.n);
            I.gamma = ppool + d.par_off;
            I.beta = ppool + d.par_off + d.p;
            I.Q = qpool + d.q_off;
            I.psi = (s.psi_off == (size_t)-1) ? (void*)(psipool + d.psi_off) : (void*)(sb + s.psi_off);
            T* Ebuf = (s.e_off == (size_t)-1) ? epool + d.e_off : reinterpret_cast<T*>(sb + s.e_off);
            I.E = Ebuf;
            char* pw = sb + s.part_off;
            I.part_expect = reinterpret_cast<double*>(pw);
            pw += align256(nt * sizeof(double));
            I.part_topp = reinterpret_cast<double*>(pw);
            pw += align256(nt * std::max(g.k, 1) * sizeof(double));
            I.part_topz = reinterpret_cast<uint32_t*>(pw);
            I.expect = io->expect ? io->expect + i : nullptr;
            I.topk_idx = d.k > 0 ? io->topk_idx + (int64_t)i * io->k_stride : nullptr;
            I.topk_prob = (d.k > 0 && io->topk_prob) ? io->topk_prob + (int64_t)i * io->k_stride : nullptr;
            if (g.grad) {
                I.lam = sb + s.lam_off;
                I.part_grad = reinterpret_cast<double*>(sb + s.grad_off);
                I.dgamma = io->grad + d.par_off;
                I.dbeta = io->grad + d.par_off + d.p;
            }
            if (g.tma) {
                // one map per pass shape, for this instance's state
                std::vector<char> done(g.maps_per_inst, 0);
                for (size_t pi = 0; pi < g.passes.size(); ++pi) {
                    const int mi = g.tsp[pi].map, ei = g.tsp[pi].emap;
                    if (done[mi]) continue;
                    done[mi] = 1;
                    char* row = img.data() + g.maps_off + TS_MAP_BYTES * (size_t)(j - 1) * g.maps_per_inst;
                    if (!tstream_encode_maps(g.passes[pi], I.psi, const_cast<T*>(I.E), row + TS_MAP_BYTES * mi,
                                             row + TS_MAP_BYTES * ei)) {
                        g.tma = false;
                        break;
                    }
                }
            }
            if (g.tadj) {
                std::vector<char> done(g.amaps_per_inst, 0);
                for (size_t pi = 0; pi < g.apasses.size(); ++pi) {
                    const int mi = g.atsp[pi].map;
                    if (done[mi]) continue;
                    done[mi] = 1;
                    char* row = img.data() + g.amaps_off + TS_MAP_BYTES * (size_t)(j - 1) * g.amaps_per_inst;
                    if (!tstream_encode_adj_maps(g.apasses[pi], I.psi, I.lam, const_cast<T*>(I.E),
                                                 row + TS_MAP_BYTES * mi)) {
                        g.tadj = false;
                        break;
                    }
                }
            }
            si.push_back(I);
            g.q.push_back(qpool + d.q_off);
            g.e.push_back(Ebuf);
        }
        std::memcpy(img.data() + g.inst_off, si.data(), sizeof(StreamInst<T>) * g.count);
        P->kernels += 1 + (int)g.passes.size() + 1 + (g.grad ? (int)g.apasses.size() + 1 : 0) +
                      (stream_finalize_two_level(1ull << (g.n - tb), g.k) ? 1 : 0);
        ++gi;
    }
    // upload the header: synchronously into the plan's own memory, else asynchronously on the
    // caller's stream from its pinned staging buffer
    if (mem && mem->staging) {
        std::memcpy(mem->staging, img.data(), sbase);
        e = cudaMemcpyAsync(base, mem->staging, sbase, cudaMemcpyHostToDevice, mem->st);
    } else {
        e = cudaMemcpy(base, img.data(), sbase, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) { qaoa_plan_destroy(P); return cuda_fail(e, "upload plan descriptors"); }
    // algorithmic bytes, in the order qaoa_plan_launch issues the kernels
    for (auto& g : P->res) {
        double b = 0.0;
        for (int i = 0; i < count; ++i) {
            const qaoa_inst& d = desc[i];
            const bool in = d.n <= nres && d.n == g.n && (((d.flags & QAOA_INST_GRAD) != 0) == g.grad);
            if (!in) continue;
            const double D = (double)(1ull << d.n);
            b += (double)d.n * d.n * sizeof(T) + 2.0 * d.p * sizeof(T) + sizeof(double) +
                 d.k * 16.0 + (d.psi_off >= 0 ? D * sizeof(C2) : 0.0) + (d.e_off >= 0 ? D * sizeof(T) : 0.0) +
                 ((d.flags & QAOA_INST_GRAD) ? 16.0 * d.p : 0.0);
        }
        P->bytes.push_back(b);
    }
    for (auto& g : P->clu) {
        double b = 0.0;
        for (int i = 0; i < count; ++i) {
            const qaoa_inst& d = desc[i];
            if (d.n != g.n || d.n <= nres || (d.flags & QAOA_INST_GRAD)) continue;
            const double D = (double)(1ull << d.n);
            b += (double)d.n * d.n * sizeof(T) + 2.0 * d.p * sizeof(T) + sizeof(double) + d.k * 16.0 +
                 (d.psi_off >= 0 ? D * sizeof(C2) : 0.0) + (d.e_off >= 0 ? D * sizeof(T) : 0.0);
        }
        P->bytes.push_back(b);
    }
    {
        size_t gi = 0;
        for (auto& kv : csg) {
            double b = 0.0;
            for (int i : kv.second) {
                const qaoa_inst& d = desc[i];
                const double D = (double)(1ull << d.n);
                b += (double)d.n * d.n * sizeof(T) + 2.0 * d.p * sizeof(T) + sizeof(double) + d.k * 16.0 +
                     (d.psi_off >= 0 ? D * sizeof(C2) : 0.0) + (d.e_off >= 0 ? D * sizeof(T) : 0.0);
            }
            P->bytes.push_back(b);
            ++gi;
        }
    }
    for (auto& g : P->str) {
        const double D = (double)(1ull << g.n), cnt = (double)g.count;
        const double nt = (double)(1ull << (g.n - tb));
        P->bytes.push_back(cnt * (D * sizeof(T) + (double)g.n * g.n * sizeof(T)));
        for (auto& pass : g.passes)
            P->bytes.push_back(cnt * D * ((pass.init ? 0.0 : sizeof(C2)) + (pass.no_store ? 0.0 : sizeof(C2)) +
                                          (pass.need_e ? sizeof(T) : 0.0)));
        P->bytes.push_back(cnt * (nt * (sizeof(double) + std::max(g.k, 1) * 12.0) + 8.0 + g.k * 16.0));
        if (g.grad) {
            const int SA = (int)g.apasses.size();
            const double nta = (double)(1ull << (g.n - tba));
            for (int s = SA - 1; s >= 0; --s)   // psi and lam read (lam formed in the first), E read, both written back
                P->bytes.push_back(cnt * D * ((s == SA - 1 ? 1.0 : 2.0) * sizeof(C2) + sizeof(T) +
                                              (s > 0 ? 2.0 * sizeof(C2) : 0.0)));
            P->bytes.push_back(cnt * (double)SA * nta * 32.0);
        }
    }
    *out = P;
    return QAOA_OK;
}

}  // namespace

namespace qaoa {

bool cstream_usable(qaoa_ctx* c, int n) {
    if (n < CS_NMIN || n > CS_NMAX) return false;
    if (c->cs_ok[n] == 0) {
        int mc = 0, dev = -1;
        cudaGetDevice(&dev);
        if (dev != c->device) cudaSetDevice(c->device);
        const bool ok = cstream_available() && cstream_max_clusters(n, &mc) == cudaSuccess && mc >= 1;
        cudaGetLastError();
        if (dev >= 0 && dev != c->device) cudaSetDevice(dev);
        c->cs_ok[n] = ok ? 1 : -1;
    }
    return c->cs_ok[n] > 0;
}

// Record an error message for qaoa_last_error from another translation unit.
qaoa_status set_error(qaoa_status st, const char* msg) { return fail(st, "%s", msg); }

// Scratch bytes one complex64 instance adds to a plan (the streaming tier's per-instance
// buffers; the resident and cluster tiers need none), as plan_create_t lays them out.
size_t plan_inst_scratch_bytes(qaoa_ctx* c, int n, int p, int k, bool grad) {
    const bool res = n <= RES_NMAX_F && (!grad || n <= RES_NMAX_F_ADJ);
    const int tier = grad ? QAOA_TIER_STREAM : eff_tier(c, n, p);
    const bool clu = !grad && n >= CL_NMIN && n <= CL_NMAX && tier == QAOA_TIER_CLUSTER;
    if (res || clu) return 0;
    if (!grad && tier == QAOA_TIER_CSTREAM && n >= CS_NMIN && n <= CS_NMAX && cstream_usable(c, n))
        return align256(((size_t)1 << n) * sizeof(float2)) + align256(((size_t)1 << n) * sizeof(float));
    const int tb = stream_tile_bits(false), tba = stream_adj_tile_bits(false);
    const size_t D = (size_t)1 << n, nt = (size_t)1 << (n - tb), kk = (size_t)std::max(k, 1);
    size_t b = align256(D * sizeof(float)) + align256(D * sizeof(float2)) + align256(nt * sizeof(double)) +
               align256(nt * kk * sizeof(double)) + align256(nt * kk * sizeof(uint32_t));
    if (grad) {
        StreamPass tmp[256];
        const int SA = stream_plan(false, n, p, 0, tmp, 256, tba);
        b += align256(D * sizeof(float2)) + align256((size_t)std::max(SA, 0) * ((size_t)1 << (n - tba)) * 32);
    }
    return b;
}

// Upper bound of a complex64 plan's header (counters and descriptor arrays) for `count` instances.
size_t plan_header_bound(int count) {
    const size_t d = std::max(std::max(sizeof(InstDesc<float>), sizeof(StreamInst<float>)), cstream_inst_bytes());
    // tensor maps per instance: the cluster-streaming tier's, or at n <= 30 the TMA streaming
    // tier's forward maps (at most 3 shapes x 2) and adjoint maps (at most 4 shapes x 3)
    const size_t maps = std::max<size_t>(CS_MAPS_BYTES, 18 * TS_MAP_BYTES);
    return align256(256 + (size_t)count * (align256(d) + maps + 512));
}

// A complex64 plan placed in caller memory, its header uploaded on `st` from pinned `staging`.
qaoa_status plan_create_placed(qaoa_ctx* c, const qaoa_inst* desc, int count, const qaoa_batch_io* io,
                               void* base, size_t bytes, cudaStream_t st, void* staging,
                               size_t staging_bytes, qaoa_plan** out) {
    if (!c || !desc || !io || !out || count < 1) return fail(QAOA_E_INVALID, "plan_create_placed: bad arguments");
    *out = nullptr;
    const PlanMem m{base, bytes, st, staging, staging_bytes};
    return plan_create_t<float>(c, desc, count, io, &m, out);
}

}  // namespace qaoa

extern "C" qaoa_status qaoa_plan_create(qaoa_ctx* c, const qaoa_inst* desc, int count,
                                        const qaoa_batch_io* io, int dbl, qaoa_plan** out) {
    if (!c || !desc || !io || !out || count < 1 || !io->q || !io->params)
        return fail(QAOA_E_INVALID, "plan_create: NULL argument or count < 1");
    *out = nullptr;
    CK(cudaSetDevice(c->device));
    return dbl ? plan_create_t<double>(c, desc, count, io, nullptr, out)
               : plan_create_t<float>(c, desc, count, io, nullptr, out);
}

namespace {
qaoa_status plan_enqueue(qaoa_plan* P, cudaStream_t st);
}

extern "C" qaoa_status qaoa_plan_launch(qaoa_plan* P, qaoa_stream_t stream) {
    if (!P) return fail(QAOA_E_INVALID, "plan is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (P->graph) {
        CK(cudaGraphLaunch(P->graph, st));
        return QAOA_OK;
    }
    return plan_enqueue(P, st);
}

extern "C" qaoa_status qaoa_plan_capture(qaoa_plan* P, qaoa_stream_t stream) {
    if (!P || !stream) return fail(QAOA_E_INVALID, "plan_capture: NULL plan or the legacy stream");
    if (P->graph) return QAOA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const bool timing = P->timing;
    P->timing = false;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const qaoa_status q = plan_enqueue(P, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    P->timing = timing;
    if (q != QAOA_OK) {
        if (g) cudaGraphDestroy(g);
        return q;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    const cudaError_t e2 = cudaGraphInstantiate(&P->graph, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        P->graph = nullptr;
        return cuda_fail(e2, "cudaGraphInstantiate");
    }
    return QAOA_OK;
}

namespace {
qaoa_status plan_enqueue(qaoa_plan* P, cudaStream_t st) {
    char* base = static_cast<char*>(P->dev);
    int* counters = reinterpret_cast<int*>(base);
    P->names.clear();
    // wrap each kernel launch in a pair of timing events when timing is on
    auto timed = [&](const char* name, auto&& launch) -> cudaError_t {
        const size_t i = P->names.size();
        if (P->timing) {
            while (P->ev.size() < 2 * (i + 1)) {
                cudaEvent_t e;
                cudaError_t r = cudaEventCreate(&e);
                if (r != cudaSuccess) return r;
                P->ev.push_back(e);
            }
            cudaEventRecord(P->ev[2 * i], st);
        }
        cudaError_t r = launch();
        if (P->timing) cudaEventRecord(P->ev[2 * i + 1], st);
        P->names.push_back(name);
        return r;
    };
    for (auto& g : P->res) {
        CK(cudaMemsetAsync(counters + g.q_slot, 0, sizeof(int), st));
        CK(timed("resident", [&] {
            return launch_resident(P->dbl, base + g.desc_off, g.count, g.n, g.pmax, g.grad,
                                   counters + g.q_slot, g.grid, st, nullptr, g.rmax);
        }));
    }
    for (auto& g : P->clu)
        CK(timed("cluster", [&] {
            return launch_cluster(base + g.desc_off, g.count, g.n, g.L, g.pmax, g.clusters, st, nullptr);
        }));
    for (auto& g : P->cs)
        CK(timed("cstream", [&] {
            return launch_cstream(g.n, base + g.desc_off, g.count, g.clusters,
                                  reinterpret_cast<unsigned*>(counters + PLAN_STATUS_SLOT), st);
        }));
    const int tb = stream_tile_bits(P->dbl);
    for (auto& g : P->str) {
        CK(timed("energy", [&] { return launch_energy_batch(P->dbl, g.n, base + g.inst_off, g.count, st); }));
        for (size_t pi = 0; pi < g.passes.size(); ++pi) {
            const StreamPass& pass = g.passes[pi];
            if (g.tma)
                CK(timed("tstream_pass", [&] {
                    return launch_tstream_pass(pass, g.tsp[pi], base + g.inst_off, g.count, base + g.maps_off,
                                               g.tgrid, reinterpret_cast<unsigned*>(counters + PLAN_STATUS_SLOT), st);
                }));
            else
                CK(timed("stream_pass", [&] {
                    return launch_stream_pass(P->dbl, pass, base + g.inst_off, g.count, g.grid, st);
                }));
        }
        CK(timed("stream_finalize", [&] {
            return launch_stream_finalize(P->dbl, base + g.inst_off, g.count, 1ull << (g.n - tb), g.k, st);
        }));
        if (g.grad) {
            const int SA = (int)g.apasses.size();
            for (int s = SA - 1; s >= 0; --s)
                CK(timed("stream_adjoint", [&] {
                    if (g.tadj)
                        return launch_tstream_adj_pass(g.apasses[s], g.atsp[s], s, s == SA - 1, s > 0, base + g.inst_off,
                                                       g.count, base + g.amaps_off, 2 * P->ctx->nsm,
                                                       reinterpret_cast<unsigned*>(counters + PLAN_STATUS_SLOT), st);
                    return launch_stream_adj_pass(P->dbl, g.apasses[s], s, s == SA - 1, s > 0, base + g.inst_off,
                                                  g.count, g.agrid, st);
                }));
            CK(timed("stream_grad_reduce", [&] {
                return launch_stream_grad_reduce(P->dbl, g.apasses.data(), SA, base + g.inst_off, g.count,
                                                 1ull << (g.n - stream_adj_tile_bits(P->dbl)), st);
            }));
        }
    }
    return QAOA_OK;
}

}  // namespace

extern "C" qaoa_status qaoa_plan_set_timing(qaoa_plan* P, int on) {
    if (!P) return fail(QAOA_E_INVALID, "plan is NULL");
    P->timing = on != 0;
    return QAOA_OK;
}

extern "C" int qaoa_plan_kernel_times(qaoa_plan* P, float* ms, const char** names, int max) {
    if (!P || !P->timing || P->ev.size() < 2 * P->names.size()) return 0;
    const int n = std::min<int>(max, (int)P->names.size());
    if (n > 0) cudaEventSynchronize(P->ev[2 * (P->names.size() - 1) + 1]);
    for (int i = 0; i < n; ++i) {
        float t = 0.f;
        cudaEventElapsedTime(&t, P->ev[2 * i], P->ev[2 * i + 1]);
        if (ms) ms[i] = t;
        if (names) names[i] = P->names[i];
    }
    return n;
}

extern "C" int qaoa_plan_kernel_count(const qaoa_plan* P) { return P ? P->kernels : 0; }

extern "C" qaoa_status qaoa_plan_check(qaoa_plan* P) {
    if (!P) return fail(QAOA_E_INVALID, "plan is NULL");
    unsigned st = 0;
    CK(cudaSetDevice(P->ctx->device));
    CK(cudaMemcpy(&st, static_cast<char*>(P->dev) + PLAN_STATUS_SLOT * sizeof(int), sizeof(st),
                  cudaMemcpyDeviceToHost));
    if (st) return fail(QAOA_E_TIMEOUT, "a device-side wait of the plan ran out of time (status %u)", st);
    return QAOA_OK;
}

extern "C" int qaoa_plan_kernel_bytes(const qaoa_plan* P, double* bytes, int max) {
    if (!P) return 0;
    const int n = std::min<int>(max, (int)P->bytes.size());
    for (int i = 0; i < n; ++i) bytes[i] = P->bytes[i];
    return n;
}

extern "C" void qaoa_plan_destroy(qaoa_plan* P) {
    if (!P) return;
    cudaSetDevice(P->ctx->device);
    if (P->graph) cudaGraphExecDestroy(P->graph);
    if (P->owns) {
        cudaDeviceSynchronize();
        cudaFree(P->dev);
    }
    for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
    delete P;
}

static qaoa_status batch_run(qaoa_ctx* c, const qaoa_inst* desc, int count, const qaoa_batch_io* io,
                             qaoa_stream_t stream, int dbl) {
    if (!c || !desc || !io || count < 1 || !io->q || !io->params)
        return fail(QAOA_E_INVALID, "batch_run: NULL argument or count < 1");
    CK(cudaSetDevice(c->device));
    qaoa_plan* P = nullptr;
    // the plan's bytes: placed in the context workspace when it is large enough (no allocation),
    // else allocated for this call
    size_t need = 0;
    const PlanMem probe{nullptr, 0, (cudaStream_t)stream, nullptr, 0};
    qaoa_status s = dbl ? plan_create_t<double>(c, desc, count, io, &probe, &P, &need)
                        : plan_create_t<float>(c, desc, count, io, &probe, &P, &need);
    if (s != QAOA_OK && s != QAOA_E_NOMEM) return s;
    P = nullptr;
    if (need > 0 && need <= c->ws_bytes) {
        CK(cudaStreamSynchronize((cudaStream_t)stream));   // earlier work on the stream may use the workspace
        const PlanMem inws{c->ws, c->ws_bytes, (cudaStream_t)stream, nullptr, 0};
        s = dbl ? plan_create_t<double>(c, desc, count, io, &inws, &P)
                : plan_create_t<float>(c, desc, count, io, &inws, &P);
    } else {
        s = qaoa_plan_create(c, desc, count, io, dbl, &P);
    }
    if (s) return s;
    s = qaoa_plan_launch(P, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    const qaoa_status st = (s == QAOA_OK && e == cudaSuccess) ? qaoa_plan_check(P) : QAOA_OK;
    qaoa_plan_destroy(P);
    if (s) return s;
    if (e != cudaSuccess) return cuda_fail(e, "batch_run synchronize");
    return st;
}

extern "C" qaoa_status qaoa_batch_run(qaoa_ctx* c, const qaoa_inst* d, int n, const qaoa_batch_io* io,
                                      qaoa_stream_t s) {
    return batch_run(c, d, n, io, s, 0);
}
extern "C" qaoa_status qaoa_batch_run_z(qaoa_ctx* c, const qaoa_inst* d, int n, const qaoa_batch_io* io,
                                        qaoa_stream_t s) {
    return batch_run(c, d, n, io, s, 1);
}

extern "C" qaoa_status qaoa_adam_step(int count, float* theta, const double* grad, float* m, float* v,
                                      int step, float lr, float b1, float b2, float eps, int minimise,
                                      qaoa_stream_t stream) {
    if (count < 0 || (count > 0 && (!theta || !grad || !m || !v)) || step < 1 || !(lr > 0.0f) ||
        !(b1 >= 0.0f && b1 < 1.0f) || !(b2 >= 0.0f && b2 < 1.0f) || !(eps > 0.0f))
        return fail(QAOA_E_INVALID, "adam_step: bad arguments");
    if (count == 0) return QAOA_OK;
    CK(launch_adam(count, theta, grad, m, v, step, lr, b1, b2, eps, minimise, (cudaStream_t)stream));
    return QAOA_OK;
}

// =============================================================================================
// Plain path
// =============================================================================================

extern "C" qaoa_status qaoa_plain_solve(qaoa_ctx* c, int n, int p, const float* Q, const float* gamma,
                                        const float* beta, float* E, void* psi, int k, double* expect,
                                        uint64_t* topk_idx, double* topk_prob, qaoa_stream_t stream) {
    if (!c) return fail(QAOA_E_INVALID, "ctx is NULL");
    if (bad_nk(n, k) || p < 1 || p > PMAX || !Q || !gamma || !beta || !E || !psi)
        return fail(QAOA_E_INVALID, "plain_solve: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    CK(launch_energy(false, n, Q, E, st));
    CK(launch_plain_layers(n, p, gamma, beta, E, static_cast<float2*>(psi), 1, st, nullptr));
    return reduce_t<float>(c, n, psi, E, k, expect, topk_idx, topk_prob, stream);
}

// =============================================================================================
// DQAOA host steps
// =============================================================================================

extern "C" qaoa_status dqaoa_draw_indices(const double* Q, int N, const uint8_t* x, int method, int m,
                                          int k, uint64_t seed, uint64_t cycle, int32_t* idx) {
    if (N < 1 || m < 1 || k < 1 || k > N || !idx) return fail(QAOA_E_INVALID, "draw: N=%d m=%d k=%d", N, m, k);
    const int base = method & 15;
    const bool sgn = (method & DQAOA_SIGNED_IMPACT) != 0;
    if ((method & ~31) || base > DQAOA_PFS || (sgn && base == DQAOA_RANDOM))
        return fail(QAOA_E_INVALID, "unknown decomposition method %d", method);
    if (method == DQAOA_RANDOM) {
        draw_random(N, m, k, seed, cycle, idx);
        return QAOA_OK;
    }
    if (base == DQAOA_IFD) {
        if (!Q || !x) return fail(QAOA_E_INVALID, "IFD needs Q and x");
        if (m + k - 1 > N) return fail(QAOA_E_INVALID, "IFD needs m + k - 1 <= N");
        draw_ifd(Q, N, x, m, k, idx, sgn);
        return QAOA_OK;
    }
    if (base == DQAOA_BFS || base == DQAOA_PFS) {
        if (!Q || !x) return fail(QAOA_E_INVALID, "BFS / PFS need Q and x");
        if (m > N) return fail(QAOA_E_INVALID, "BFS / PFS need m <= N");
        draw_graph(Q, N, x, base, m, k, idx, nullptr, sgn);
        return QAOA_OK;
    }
    return fail(QAOA_E_INVALID, "unknown decomposition method %d", method);
}

extern "C" qaoa_status dqaoa_decompose(const double* Q, int N, const uint8_t* x, int method, int conditioned,
                                       int m, int k, uint64_t seed, uint64_t cycle, int32_t* idx,
                                       double* Qsub) {
    if (!Q || !Qsub) return fail(QAOA_E_INVALID, "decompose: NULL Q or Qsub");
    if (conditioned && !x) return fail(QAOA_E_INVALID, "decompose: conditioning needs x");
    qaoa_status s = dqaoa_draw_indices(Q, N, x, method, m, k, seed, cycle, idx);
    if (s) return s;
    build_subqubos(Q, N, x, m, k, idx, conditioned, Qsub);
    return QAOA_OK;
}

extern "C" qaoa_status dqaoa_subqubo_build(qaoa_ctx* c, const double* Q, int N, const uint8_t* x, int m,
                                           int k, const int32_t* idx, int conditioned, float* qsub,
                                           qaoa_stream_t stream) {
    if (!c || !Q || N < 1 || N > 40000 || m < 1 || k < 1 || k > N || k > 4096 || !idx || !qsub ||
        (conditioned && !x))
        return fail(QAOA_E_INVALID, "subqubo_build: bad arguments");
    CK(launch_subqubo(Q, N, x, m, k, idx, conditioned, qsub, (cudaStream_t)stream));
    return QAOA_OK;
}

extern "C" qaoa_status dqaoa_merge(const double* Q, int N, uint8_t* x, int m, int k, const int32_t* idx,
                                   int K, const uint64_t* cand, double* energy_out, int* accepted_out) {
    if (!Q || N < 1 || !x || m < 1 || k < 1 || k > 64 || K < 1 || !idx || !cand)
        return fail(QAOA_E_INVALID, "merge: bad arguments");
    for (int64_t t = 0; t < (int64_t)m * k; ++t)
        if (idx[t] < 0 || idx[t] >= N) return fail(QAOA_E_INVALID, "merge: index %d out of range", idx[t]);
    merge(Q, N, x, m, k, idx, K, cand, energy_out, accepted_out);
    return QAOA_OK;
}

// =============================================================================================
// DQAOA session: one cycle per call
// =============================================================================================

struct dqaoa_session {
    qaoa_ctx* ctx = nullptr;
    int N = 0, m = 0, k = 0, p = 0, K = 0, method = 0, conditioned = 1;
    void* dev = nullptr;          // Q, x, idx, qsub, params, expect, top-k
    double* Q_dev = nullptr;
    uint8_t* x_dev = nullptr;
    int32_t* idx_dev = nullptr;
    float* qsub = nullptr;
    double* qblk = nullptr;       // raw FP64 blocks Q[S_j, S_j] for the merge
    double* mh = nullptr;         // merge set-up on the device: h = Qx, column sums of |Q|, scratch
    double* mca = nullptr;
    double* mscr = nullptr;
    float* params = nullptr;
    double* expect = nullptr;
    uint64_t* topk = nullptr;
    void* host = nullptr;         // pinned staging
    int32_t* idx_h = nullptr;
    uint8_t* x_h = nullptr;
    double* expect_h = nullptr;
    double* qblk_h = nullptr;
    double* mh_h = nullptr;       // h and the column sums from the device set-up
    double* mca_h = nullptr;
    // the sub-QUBOs are solved in chunks, one plan each, so that the host merges chunk c while
    // the device solves chunk c + 1 (the merge is sequential over sub-QUBOs in index order)
    int chunks = 1;
    int chunk_start[3] = {0, 0, 0};
    qaoa_plan* plans[2] = {nullptr, nullptr};
    cudaEvent_t chunk_solved[2] = {nullptr, nullptr};   // chunk's kernels done (main stream)
    cudaEvent_t chunk_done[2] = {nullptr, nullptr};     // chunk's results on the host (side stream)
    cudaEvent_t dev_begin = nullptr, dev_end = nullptr;   // device part of the last cycle
    // the FP64 blocks go to the host on a side stream, beside the first chunk's kernels
    cudaStream_t side = nullptr;
    cudaEvent_t sub_done = nullptr, qblk_done = nullptr, setup_done = nullptr;
    cudaStream_t solve2 = nullptr;  // the second chunk's solve
    // per chunk one packed block (pair terms, candidates, <C>, status word) on the device and its
    // pinned copy: one copy per chunk brings back everything the merge reads
    char* pk_dev = nullptr;
    char* pk_h = nullptr;
    size_t pk_off[2] = {0, 0};
    bool last_sampled = false;      // the last cycle was dqaoa_session_cycle_sampled
    cudaEvent_t solve_begin = nullptr, solve_end = nullptr;   // span of the chunk solves
    double t_decompose = 0.0, t_merge = 0.0, t_cycle = 0.0; // host ms of the last cycle
    MergeCache cache;             // h = Qx and E(x) after the last merge
    StrongGraph graph;            // BFS / PFS strong-interaction graph of the current Q
    bool graph_valid = false;
    std::vector<uint8_t> x_last;  // the solution the cache belongs to
    // random index sets of the next cycle, drawn on the host while the device works
    std::vector<int32_t> next_idx;
    bool next_valid = false;
    uint64_t next_seed = 0, next_cycle = 0;
    // sampled cycles (dqaoa_session_cycle_sampled), set up on first use: one plan over all m
    // sub-QUBOs that returns their states, then shots and the best shot of each on the device
    qaoa_plan* s_plan = nullptr;
    void* s_dev = nullptr;        // states (m * 2^k complex64), FP64 diagonals, sampler scratch
    void* s_shot_dev = nullptr;   // uniforms, shots (m * s_shots each), best shots (m)
    int s_shots = 0;              // shots per sub-QUBO the buffers hold
    int s_last_shots = 0;         // shots per sub-QUBO of the last sampled cycle (0: none yet)
    void* s_psi = nullptr;
    double* s_qdiag = nullptr;
    double* s_scratch = nullptr;
    double* s_u = nullptr;
    uint64_t* s_z = nullptr;
    uint64_t* s_best = nullptr;
    uint64_t* s_best_h = nullptr; // pinned, with the plan's status word after it
    unsigned* s_status_h = nullptr;
};

extern "C" qaoa_status dqaoa_session_create(qaoa_ctx* c, int N, int m, int k, int p, int K, int method,
                                            int conditioned, const double* gamma, const double* beta,
                                            dqaoa_session** out) {
    if (!c || !out || N < 1 || m < 1 || k < 1 || k > N || k > NMAX || p < 1 || p > PMAX || K < 1 ||
        K > KMAX || (uint64_t)K > (1ull << k) || !gamma || !beta || (method & ~63) || (method & 15) > DQAOA_PFS ||
        (method & 31) == (DQAOA_RANDOM | DQAOA_SIGNED_IMPACT))
        return fail(QAOA_E_INVALID, "session_create: bad arguments");
    const bool paper_mixer = (method & DQAOA_PAPER_MIXER) != 0;
    method &= 31;
    if ((method & 15) == DQAOA_IFD && m + k - 1 > N) return fail(QAOA_E_INVALID, "IFD needs m + k - 1 <= N");
    if (((method & 15) == DQAOA_BFS || (method & 15) == DQAOA_PFS) && m > N)
        return fail(QAOA_E_INVALID, "BFS / PFS need m <= N");
    *out = nullptr;
    CK(cudaSetDevice(c->device));
    dqaoa_session* s = new dqaoa_session();
    s->ctx = c; s->N = N; s->m = m; s->k = k; s->p = p; s->K = K; s->method = method;
    s->conditioned = conditioned;
    size_t o = 0;
    const size_t oQ = o; o = align256(o + (size_t)N * N * sizeof(double));
    const size_t ox = o; o = align256(o + (size_t)N);
    const size_t oi = o; o = align256(o + (size_t)m * k * sizeof(int32_t));
    const size_t oq = o; o = align256(o + (size_t)m * k * k * sizeof(float));
    const size_t ob = o; o = align256(o + (size_t)m * k * k * sizeof(double));
    const size_t op = o; o = align256(o + (size_t)2 * p * sizeof(float));
    const size_t oe = o; o = align256(o + (size_t)m * sizeof(double));
    const size_t ot = o; o = align256(o + (size_t)m * K * sizeof(uint64_t));
    const size_t omh = o; o = align256(o + (size_t)N * sizeof(double));
    const size_t omc = o; o = align256(o + (size_t)N * sizeof(double));
    const size_t oms = o; o = align256(o + (size_t)2 * merge_setup_blocks(N) * N * sizeof(double));
    cudaError_t e = cudaMalloc(&s->dev, o);
    if (e != cudaSuccess) { delete s; return fail(QAOA_E_NOMEM, "session cudaMalloc: %s", cudaGetErrorString(e)); }
    char* b = static_cast<char*>(s->dev);
    s->Q_dev = reinterpret_cast<double*>(b + oQ);
    s->x_dev = reinterpret_cast<uint8_t*>(b + ox);
    s->idx_dev = reinterpret_cast<int32_t*>(b + oi);
    s->qsub = reinterpret_cast<float*>(b + oq);
    s->qblk = reinterpret_cast<double*>(b + ob);
    s->params = reinterpret_cast<float*>(b + op);
    s->expect = reinterpret_cast<double*>(b + oe);
    s->topk = reinterpret_cast<uint64_t*>(b + ot);
    s->mh = reinterpret_cast<double*>(b + omh);
    s->mca = reinterpret_cast<double*>(b + omc);
    s->mscr = reinterpret_cast<double*>(b + oms);
    size_t h = 0;
    // x then the index sets, spaced as on the device (ox, oi): one copy moves both
    const size_t hx = h; h = align256(h + (size_t)N);
    const size_t hi = h; h = align256(h + (size_t)m * k * sizeof(int32_t));
    const size_t he = h; h = align256(h + (size_t)m * sizeof(double));
    const size_t hb2 = h; h = align256(h + (size_t)m * k * k * sizeof(double));
    const size_t hmh = h; h = align256(h + (size_t)N * sizeof(double));
    const size_t hmc = h; h = align256(h + (size_t)N * sizeof(double));
    e = cudaMallocHost(&s->host, h);
    if (e != cudaSuccess) { cudaFree(s->dev); delete s; return fail(QAOA_E_NOMEM, "session cudaMallocHost"); }
    char* hb = static_cast<char*>(s->host);
    s->idx_h = reinterpret_cast<int32_t*>(hb + hi);
    s->x_h = reinterpret_cast<uint8_t*>(hb + hx);
    if (reinterpret_cast<char*>(s->idx_h) - reinterpret_cast<char*>(s->x_h) !=
        reinterpret_cast<char*>(s->idx_dev) - reinterpret_cast<char*>(s->x_dev)) {
        dqaoa_session_destroy(s);
        return fail(QAOA_E_INVALID, "session_create: staging layout mismatch");
    }
    s->expect_h = reinterpret_cast<double*>(hb + he);
    s->qblk_h = reinterpret_cast<double*>(hb + hb2);
    s->mh_h = reinterpret_cast<double*>(hb + hmh);
    s->mca_h = reinterpret_cast<double*>(hb + hmc);
    std::vector<float> par(2 * p);
    // the paper's mixer H_X = -sum X is this library's mixer at -beta
    for (int l = 0; l < p; ++l) { par[l] = (float)gamma[l]; par[p + l] = (float)(paper_mixer ? -beta[l] : beta[l]); }
    e = cudaMemcpy(s->params, par.data(), par.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { dqaoa_session_destroy(s); return cuda_fail(e, "session params upload"); }
    // Two chunks from m = 128 on, so that the host merges the first while the device solves the
    // second. Streaming tier: about two thirds, rounded up to whole waves (instances whose tiles
    // give every block of a launch one tile; measured on GB300 for 256 sub-QUBOs of n = 16: 190 /
    // 66 beat 152 / 104, 128 / 128 and 114 / 142 by 4-8%). Cluster-streaming tier, whose two
    // chunk launches overlap on the device: 11/16 of m for N <= 4096 (measured for 256
    // sub-QUBOs at N = 1000: splits from 128 to 216 within 4%, 176 best, 232 8% slower), 9/16
    // above (at N = 10^4 the merge costs about 0.8 of the solve).
    s->chunks = m >= 128 ? 2 : 1;
    int m0 = m;
    if (s->chunks == 2) {
        const int tier = eff_tier(c, k, p);
        if (k >= CS_NMIN && k <= CS_NMAX && tier == QAOA_TIER_CSTREAM && cstream_usable(c, k)) {
            // the first chunk's merge should end before the second chunk's solve does: with the
            // merge's cost growing with N (the update of h per flipped variable), a larger N
            // takes a smaller first chunk
            m0 = N <= 4096 ? (m * 11) / 16 : (m * 9) / 16;
        } else {
            int w = 1;
            if (k >= 16 && (k > 18 || tier == QAOA_TIER_STREAM)) {
                const int tiles = 1 << (k - stream_tile_bits(false));
                w = std::max(1, 2 * c->nsm / tiles);
            }
            m0 = (m * 13 + 19) / 20;
            m0 = (m0 + w - 1) / w * w;
        }
        m0 = std::max(1, std::min(m - 1, m0));
    }
    s->chunk_start[1] = m0;
    s->chunk_start[2] = m;
    for (int ch = 0; ch < s->chunks; ++ch) {
        const int j0 = s->chunk_start[ch], mc = s->chunk_start[ch + 1] - j0;
        std::vector<qaoa_inst> d(mc);
        for (int j = 0; j < mc; ++j) d[j] = qaoa_inst{k, p, K, 0, (int64_t)(j0 + j) * k * k, 0, -1, -1};
        qaoa_batch_io io{};
        io.q = s->qsub;
        io.params = s->params;
        io.expect = s->expect + j0;
        io.topk_idx = s->topk + (size_t)j0 * K;
        io.k_stride = K;
        qaoa_status st = qaoa_plan_create(c, d.data(), mc, &io, 0, &s->plans[ch]);
        if (st == QAOA_OK && (cudaEventCreateWithFlags(&s->chunk_done[ch], cudaEventDisableTiming) != cudaSuccess ||
                              cudaEventCreateWithFlags(&s->chunk_solved[ch], cudaEventDisableTiming) != cudaSuccess))
            st = fail(QAOA_E_CUDA, "session event");
        if (st) { dqaoa_session_destroy(s); return st; }
    }
    {
        size_t pk = 0;
        for (int ch = 0; ch < s->chunks; ++ch) {
            s->pk_off[ch] = pk;
            pk += cand_pack_bytes(s->chunk_start[ch + 1] - s->chunk_start[ch], K);
        }
        if (cudaMalloc(&s->pk_dev, pk) != cudaSuccess) {
            s->pk_dev = nullptr;
            dqaoa_session_destroy(s);
            return fail(QAOA_E_NOMEM, "session cudaMalloc (result blocks)");
        }
        if (cudaMallocHost(&s->pk_h, pk) != cudaSuccess) {
            s->pk_h = nullptr;
            dqaoa_session_destroy(s);
            return fail(QAOA_E_NOMEM, "session cudaMallocHost (result blocks)");
        }
    }
    if (cudaEventCreate(&s->dev_begin) != cudaSuccess || cudaEventCreate(&s->dev_end) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->sub_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->qblk_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->setup_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&s->solve_begin) != cudaSuccess || cudaEventCreate(&s->solve_end) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->solve2, cudaStreamNonBlocking) != cudaSuccess) {
        dqaoa_session_destroy(s);
        return fail(QAOA_E_CUDA, "session events");
    }
    *out = s;
    return QAOA_OK;
}

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Decomposition step of a cycle (Section V-A): the index sets on the host (random sets drawn
// ahead during the previous cycle when seed and cycle match), Q (when changed), x and the index
// sets to the device, then the matrices of the first `rows` sub-QUBOs on the device (with their
// FP64 diagonals when qdiag is given); the caller builds the others. dev_begin is recorded
// before the first per-cycle copy.
qaoa_status session_decompose(dqaoa_session* s, const double* Q, int q_changed, const uint8_t* x, uint64_t seed,
                              uint64_t cycle, cudaStream_t st, double* qdiag, int rows) {
    const int N = s->N, m = s->m, k = s->k;
    if (q_changed) CK(cudaMemcpyAsync(s->Q_dev, Q, (size_t)N * N * sizeof(double), cudaMemcpyHostToDevice, st));
    qaoa_status r = QAOA_OK;
    if (s->method == DQAOA_RANDOM && s->next_valid && s->next_seed == seed && s->next_cycle == cycle)
        std::memcpy(s->idx_h, s->next_idx.data(), (size_t)m * k * sizeof(int32_t));
    else if ((s->method & 15) == DQAOA_BFS || (s->method & 15) == DQAOA_PFS) {
        if (q_changed || !s->graph_valid) {
            build_strong_graph(Q, N, k, &s->graph);
            s->graph_valid = true;
        }
        draw_graph(Q, N, x, s->method & 15, m, k, s->idx_h, &s->graph, (s->method & DQAOA_SIGNED_IMPACT) != 0);
    } else
        r = dqaoa_draw_indices(Q, N, x, s->method, m, k, seed, cycle, s->idx_h);
    s->next_valid = false;
    if (r) return r;
    std::memcpy(s->x_h, x, (size_t)N);
    CK(cudaEventRecord(s->dev_begin, st));
    CK(cudaMemcpyAsync(s->x_dev, s->x_h,
                       (size_t)(reinterpret_cast<char*>(s->idx_h) - reinterpret_cast<char*>(s->x_h)) +
                           (size_t)m * k * sizeof(int32_t),
                       cudaMemcpyHostToDevice, st));
    CK(launch_subqubo(s->Q_dev, N, s->x_dev, rows, k, s->idx_dev, s->conditioned, s->qsub, st, s->qblk, qdiag));
    return QAOA_OK;
}

}  // namespace

extern "C" qaoa_status dqaoa_session_cycle(dqaoa_session* s, const double* Q, int q_changed, uint8_t* x,
                                           uint64_t seed, uint64_t cycle, double* energy_out,
                                           int* accepted_out, qaoa_stream_t stream) {
    if (!s || !Q || !x) return fail(QAOA_E_INVALID, "session_cycle: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = s->N, m = s->m, k = s->k, K = s->K;
    const double t0 = now_ms();
    // h = Qx from the last merge stays valid while Q is unchanged and x is the solution that
    // merge left; else the device sets it up (beside the solve, on the side stream)
    const bool need_setup = !(s->cache.valid && !q_changed && s->x_last.size() == (size_t)N &&
                              std::memcmp(s->x_last.data(), x, (size_t)N) == 0);
    qaoa_status r = session_decompose(s, Q, q_changed, x, seed, cycle, st, nullptr, m);
    if (r) return r;
    CK(cudaEventRecord(s->sub_done, st));
    // the second chunk's solve runs on its own stream: its clusters take the SMs the first
    // chunk's clusters leave while that chunk's last instances finish
    if (s->chunks == 2) CK(cudaStreamWaitEvent(s->solve2, s->sub_done, 0));
    CK(cudaStreamWaitEvent(s->side, s->sub_done, 0));
    CK(cudaMemcpyAsync(s->qblk_h, s->qblk, (size_t)m * k * k * sizeof(double), cudaMemcpyDeviceToHost, s->side));
    CK(cudaEventRecord(s->qblk_done, s->side));
    if (need_setup) {
        CK(launch_merge_setup(s->Q_dev, N, s->x_dev, s->mscr, s->mh, s->mca, s->side));
        CK(cudaMemcpyAsync(s->mh_h, s->mh, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, s->side));
        CK(cudaMemcpyAsync(s->mca_h, s->mca, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, s->side));
        CK(cudaEventRecord(s->setup_done, s->side));
    }
    // solve the sub-QUBOs chunk by chunk; each chunk's results come back behind its own event
    CK(cudaEventRecord(s->solve_begin, st));
    for (int ch = 0; ch < s->chunks; ++ch) {
        const int j0 = s->chunk_start[ch], mc = s->chunk_start[ch + 1] - j0;
        cudaStream_t cs = ch == 0 ? st : s->solve2;
        r = qaoa_plan_launch(s->plans[ch], (qaoa_stream_t)cs);
        if (r) return r;
        CK(cudaEventRecord(s->chunk_solved[ch], cs));
        // the pair terms of the chunk's candidates against the cycle's starting x, packed with
        // the chunk's results into one block that one copy brings back (on the chunk's stream:
        // the next chunk's solve runs on the other one)
        CK(launch_cand_pair(mc, k, K, s->idx_dev + (size_t)j0 * k, s->x_dev, s->qblk + (size_t)j0 * k * k,
                            s->topk + (size_t)j0 * K, reinterpret_cast<double*>(s->pk_dev + s->pk_off[ch]), cs,
                            s->expect + j0,
                            reinterpret_cast<const unsigned*>(static_cast<char*>(s->plans[ch]->dev) +
                                                              PLAN_STATUS_SLOT * sizeof(int))));
        CK(cudaMemcpyAsync(s->pk_h + s->pk_off[ch], s->pk_dev + s->pk_off[ch], cand_pack_bytes(mc, K),
                           cudaMemcpyDeviceToHost, cs));
        CK(cudaEventRecord(s->chunk_done[ch], cs));
    }
    for (int ch = 0; ch < s->chunks; ++ch) CK(cudaStreamWaitEvent(s->side, s->chunk_done[ch], 0));
    CK(cudaEventRecord(s->dev_end, s->side));
    if (s->chunks == 2) CK(cudaStreamWaitEvent(st, s->chunk_solved[1], 0));   // the caller's stream covers the cycle
    CK(cudaEventRecord(s->solve_end, st));
    CK(cudaStreamWaitEvent(st, s->dev_end, 0));
    const double t1 = now_ms();
    if (s->method == DQAOA_RANDOM) {   // overlaps the device work of this cycle
        s->next_idx.resize((size_t)m * k);
        draw_random(N, m, k, seed, cycle + 1, s->next_idx.data());
        s->next_valid = true;
        s->next_seed = seed;
        s->next_cycle = cycle + 1;
    }
    // aggregate chunk by chunk in sub-QUBO order; merging chunk c overlaps the device work of
    // chunk c + 1
    int accepted = 0;
    double t_merge = 0.0;
    CK(cudaEventSynchronize(s->qblk_done));
    if (need_setup) {
        CK(cudaEventSynchronize(s->setup_done));
        const double ts = now_ms();
        merge_setup_from(N, x, s->mh_h, s->mca_h, &s->cache);
        t_merge += now_ms() - ts;
    }
    s->cache.chg.assign((size_t)N, 0);
    for (int ch = 0; ch < s->chunks; ++ch) {
        CK(cudaEventSynchronize(s->chunk_done[ch]));
        const int mcc = s->chunk_start[ch + 1] - s->chunk_start[ch];
        const double* pair_c = reinterpret_cast<const double*>(s->pk_h + s->pk_off[ch]);
        const uint64_t* cand_c = reinterpret_cast<const uint64_t*>(pair_c + (size_t)mcc * K);
        const unsigned status_c = *reinterpret_cast<const unsigned*>(reinterpret_cast<const double*>(cand_c + (size_t)mcc * K) + mcc);
        if (status_c) {
            // a device-side wait of this chunk ran out: its results are not valid, x is left as is
            cudaStreamSynchronize(st);
            return fail(QAOA_E_TIMEOUT, "session_cycle: a device-side wait of chunk %d ran out of time", ch);
        }
        const double tm = now_ms();
        const int j0 = s->chunk_start[ch], mc = s->chunk_start[ch + 1] - j0;
        int acc = 0;
        merge(Q, N, x, mc, k, s->idx_h + (size_t)j0 * k, K, cand_c, energy_out, &acc, &s->cache,
              s->qblk_h + (size_t)j0 * k * k, pair_c);
        accepted += acc;
        t_merge += now_ms() - tm;
    }
    CK(cudaStreamSynchronize(st));
    if (accepted_out) *accepted_out = accepted;
    s->last_sampled = false;
    s->x_last.assign(x, x + N);
    s->t_decompose = t1 - t0;
    s->t_merge = t_merge;
    s->t_cycle = now_ms() - t0;
    return QAOA_OK;
}

extern "C" qaoa_status dqaoa_session_timing(dqaoa_session* s, double* out) {
    if (!s || !out) return fail(QAOA_E_INVALID, "session_timing: NULL argument");
    float dev = 0.0f;
    CK(cudaEventElapsedTime(&dev, s->dev_begin, s->dev_end));
    out[0] = s->t_decompose;
    out[1] = dev;
    out[2] = s->t_merge;
    out[3] = s->t_cycle;
    return QAOA_OK;
}

extern "C" qaoa_status dqaoa_session_solve_ms(dqaoa_session* s, double* ms) {
    if (!s || !ms) return fail(QAOA_E_INVALID, "session_solve_ms: NULL argument");
    float v = 0.0f;
    CK(cudaEventElapsedTime(&v, s->solve_begin, s->solve_end));
    *ms = v;
    return QAOA_OK;
}

extern "C" qaoa_status dqaoa_session_results(dqaoa_session* s, double* expect, uint64_t* topk) {
    if (!s) return fail(QAOA_E_INVALID, "session is NULL");
    if (expect && s->last_sampled) std::memcpy(expect, s->expect_h, (size_t)s->m * sizeof(double));
    for (int ch = 0; ch < s->chunks; ++ch) {
        // the packed block of each chunk: pair terms, candidates, <C>
        const int j0 = s->chunk_start[ch], mc = s->chunk_start[ch + 1] - j0;
        const double* pair_c = reinterpret_cast<const double*>(s->pk_h + s->pk_off[ch]);
        const uint64_t* cand_c = reinterpret_cast<const uint64_t*>(pair_c + (size_t)mc * s->K);
        const double* ex_c = reinterpret_cast<const double*>(cand_c + (size_t)mc * s->K);
        if (expect && !s->last_sampled) std::memcpy(expect + j0, ex_c, (size_t)mc * sizeof(double));
        if (topk) std::memcpy(topk + (size_t)j0 * s->K, cand_c, (size_t)mc * s->K * sizeof(uint64_t));
    }
    return QAOA_OK;
}

namespace {

// Buffers of the sampled cycles: the plan and the state pool once, the shot buffers again when a
// call asks for more shots than they hold.
qaoa_status session_sampling_setup(dqaoa_session* s, int shots) {
    const int m = s->m, k = s->k, p = s->p;
    if (!s->s_plan) {
        size_t o = 0;
        const size_t ops = o; o = align256(o + ((size_t)m << k) * 8);
        const size_t odg = o; o = align256(o + (size_t)m * k * sizeof(double));
        const size_t osc = o; o = align256(o + (size_t)m * sample_scratch_bytes(k));
        cudaError_t e = cudaMalloc(&s->s_dev, o);
        if (e != cudaSuccess) { s->s_dev = nullptr; return fail(QAOA_E_NOMEM, "sampled cycle: cudaMalloc: %s", cudaGetErrorString(e)); }
        char* b = static_cast<char*>(s->s_dev);
        s->s_psi = b + ops;
        s->s_qdiag = reinterpret_cast<double*>(b + odg);
        s->s_scratch = reinterpret_cast<double*>(b + osc);
        e = cudaMallocHost(&s->s_best_h, (size_t)m * sizeof(uint64_t) + 16);
        if (e != cudaSuccess) { s->s_best_h = nullptr; return fail(QAOA_E_NOMEM, "sampled cycle: cudaMallocHost"); }
        s->s_status_h = reinterpret_cast<unsigned*>(s->s_best_h + m);
        std::vector<qaoa_inst> d(m);
        for (int j = 0; j < m; ++j) d[j] = qaoa_inst{k, p, 0, 0, (int64_t)j * k * k, 0, (int64_t)j << k, -1};
        qaoa_batch_io io{};
        io.q = s->qsub;
        io.params = s->params;
        io.psi = s->s_psi;
        io.expect = s->expect;
        qaoa_status st = qaoa_plan_create(s->ctx, d.data(), m, &io, 0, &s->s_plan);
        if (st) { s->s_plan = nullptr; return st; }
    }
    if (shots > s->s_shots) {
        cudaFree(s->s_shot_dev);
        s->s_shot_dev = nullptr;
        s->s_shots = 0;
        size_t o = 0;
        const size_t ou = o; o = align256(o + (size_t)m * shots * sizeof(double));
        const size_t oz = o; o = align256(o + (size_t)m * shots * sizeof(uint64_t));
        const size_t ob = o; o = align256(o + (size_t)m * sizeof(uint64_t));
        cudaError_t e = cudaMalloc(&s->s_shot_dev, o);
        if (e != cudaSuccess) { s->s_shot_dev = nullptr; return fail(QAOA_E_NOMEM, "sampled cycle: cudaMalloc: %s", cudaGetErrorString(e)); }
        char* b = static_cast<char*>(s->s_shot_dev);
        s->s_u = reinterpret_cast<double*>(b + ou);
        s->s_z = reinterpret_cast<uint64_t*>(b + oz);
        s->s_best = reinterpret_cast<uint64_t*>(b + ob);
        s->s_shots = shots;
    }
    return QAOA_OK;
}

}  // namespace

extern "C" qaoa_status dqaoa_session_cycle_sampled(dqaoa_session* s, const double* Q, int q_changed, uint8_t* x,
                                                   uint64_t seed, uint64_t cycle, int shots, const double* u,
                                                   double* energy_out, int* accepted_out, qaoa_stream_t stream) {
    if (!s || !Q || !x || !u || shots < 1 || shots > (1 << 20))
        return fail(QAOA_E_INVALID, "session_cycle_sampled: bad arguments");
    if (s->m > 65535) return fail(QAOA_E_INVALID, "session_cycle_sampled: m > 65535");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = s->N, m = s->m, k = s->k;
    CK(cudaSetDevice(s->ctx->device));
    qaoa_status r = session_sampling_setup(s, shots);
    if (r) return r;
    const double t0 = now_ms();
    r = session_decompose(s, Q, q_changed, x, seed, cycle, st, s->s_qdiag, m);
    if (r) return r;
    CK(cudaMemcpyAsync(s->s_u, u, (size_t)m * shots * sizeof(double), cudaMemcpyHostToDevice, st));
    r = qaoa_plan_launch(s->s_plan, stream);
    if (r) return r;
    CK(launch_sample(k, s->s_psi, m, shots, s->s_u, s->s_z, s->s_scratch, st));
    CK(launch_best_shot(m, k, shots, s->qblk, s->s_qdiag, s->s_z, s->s_best, st));
    CK(cudaMemcpyAsync(s->s_best_h, s->s_best, (size_t)m * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(s->qblk_h, s->qblk, (size_t)m * k * k * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(s->expect_h, s->expect, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(s->s_status_h, static_cast<char*>(s->s_plan->dev) + PLAN_STATUS_SLOT * sizeof(int),
                       sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(s->dev_end, st));
    const double t1 = now_ms();
    CK(cudaStreamSynchronize(st));
    s->s_last_shots = shots;
    s->last_sampled = true;
    if (*s->s_status_h) return fail(QAOA_E_TIMEOUT, "session_cycle_sampled: a device-side wait ran out of time");
    s->cache.valid = s->cache.valid && !q_changed && s->x_last.size() == (size_t)N &&
                     std::memcmp(s->x_last.data(), x, (size_t)N) == 0;
    const double tm = now_ms();
    int acc = 0;
    merge(Q, N, x, m, k, s->idx_h, 1, s->s_best_h, energy_out, &acc, &s->cache, s->qblk_h);
    if (accepted_out) *accepted_out = acc;
    s->x_last.assign(x, x + N);
    s->t_decompose = t1 - t0;
    s->t_merge = now_ms() - tm;
    s->t_cycle = now_ms() - t0;
    return QAOA_OK;
}

extern "C" qaoa_status dqaoa_session_shots(dqaoa_session* s, uint64_t* shots_out, uint64_t* best_out,
                                           void* psi_out) {
    if (!s) return fail(QAOA_E_INVALID, "session is NULL");
    if (!s->s_plan || !s->s_last_shots) return fail(QAOA_E_INVALID, "session_shots: no sampled cycle has run");
    CK(cudaSetDevice(s->ctx->device));
    const size_t m = (size_t)s->m;
    if (shots_out) CK(cudaMemcpy(shots_out, s->s_z, m * s->s_last_shots * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (best_out) std::memcpy(best_out, s->s_best_h, m * sizeof(uint64_t));
    if (psi_out) CK(cudaMemcpy(psi_out, s->s_psi, (m << s->k) * 8, cudaMemcpyDeviceToHost));
    return QAOA_OK;
}

extern "C" qaoa_plan* dqaoa_session_plan(dqaoa_session* s, int i) {
    return (s && i >= 0 && i < s->chunks) ? s->plans[i] : nullptr;
}

extern "C" void dqaoa_session_destroy(dqaoa_session* s) {
    if (!s) return;
    cudaSetDevice(s->ctx->device);
    for (int ch = 0; ch < 2; ++ch) {
        qaoa_plan_destroy(s->plans[ch]);
        if (s->chunk_done[ch]) cudaEventDestroy(s->chunk_done[ch]);
        if (s->chunk_solved[ch]) cudaEventDestroy(s->chunk_solved[ch]);
    }
    if (s->dev_begin) cudaEventDestroy(s->dev_begin);
    if (s->dev_end) cudaEventDestroy(s->dev_end);
    if (s->sub_done) cudaEventDestroy(s->sub_done);
    if (s->qblk_done) cudaEventDestroy(s->qblk_done);
    if (s->setup_done) cudaEventDestroy(s->setup_done);
    if (s->solve_begin) cudaEventDestroy(s->solve_begin);
    if (s->solve_end) cudaEventDestroy(s->solve_end);
    if (s->solve2) cudaStreamDestroy(s->solve2);
    if (s->side) cudaStreamDestroy(s->side);
    qaoa_plan_destroy(s->s_plan);
    cudaFree(s->pk_dev);
    if (s->pk_h) cudaFreeHost(s->pk_h);
    cudaFree(s->s_dev);
    cudaFree(s->s_shot_dev);
    if (s->s_best_h) cudaFreeHost(s->s_best_h);
    cudaFreeHost(s->host);
    cudaFree(s->dev);
    delete s;
}
