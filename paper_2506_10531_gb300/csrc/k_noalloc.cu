// k_noalloc.cu -- <C> and top-k of a complex64 state with no allocation at all: the standalone
// reduction kernels of k_stream.cu run on a fixed scratch array that lives in this file, in
// device memory reserved when the library is loaded (every GPU that loads the library holds it
// until the process exits). The paper has no counterpart; this is an interface addition for
// callers that cannot allocate device memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/qaoa.h"
#include "qaoa_kernels.h"
#include "qaoa_stream.h"

namespace {

constexpr int kMaxParts = 1024;
constexpr int kMaxK = 16;
static_assert(qaoa::reduce_parts(30) <= kMaxParts && qaoa::reduce_parts(1) >= 1,
              "the fixed scratch must hold the partials of every accepted n (1..30)");

// Per-block partial sums and per-block top-k lists of one reduction (about 200 KB).
struct ReduceScratch {
    double expect[kMaxParts];
    double prob[kMaxParts * kMaxK];
    uint32_t idx[kMaxParts * kMaxK];
};

static __device__ __align__(256) ReduceScratch g_reduce_scratch;

// Device address of g_reduce_scratch per CUDA device, looked up with that device current once per
// context: the unique id of the current context is kept with the address, so that after a
// cudaDeviceReset (a new primary context, the module loaded again, the array possibly elsewhere)
// the next call looks the address up again instead of using a stale one.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
ReduceScratch* g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current context, or 0 when the driver cannot say (then every call
// looks the address up, which is always correct).
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_cur || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

}  // namespace

extern "C" qaoa_status qaoa_expect_topk_static(int n, const void* psi, const float* E, int k,
                                               double* expect, uint64_t* idx, double* prob,
                                               qaoa_stream_t stream) {
    if (n < 1 || n > 30) return qaoa::report(QAOA_E_INVALID, "expect_topk_static: n must be 1..30");
    if (k < 0 || k > kMaxK || (uint64_t)k > (1ull << n))
        return qaoa::report(QAOA_E_INVALID, "expect_topk_static: k must be 0..16 and <= 2^n");
    if (!psi || (expect && !E) || (k > 0 && !idx) || (!expect && k == 0))
        return qaoa::report(QAOA_E_INVALID, "expect_topk_static: NULL pointer or nothing to compute");
    if (qaoa::reduce_parts(n) > kMaxParts)
        return qaoa::report(QAOA_E_INVALID, "expect_topk_static: state too large for the fixed scratch");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return qaoa::report(QAOA_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return qaoa::report(QAOA_E_UNSUPPORTED, "expect_topk_static: device index >= 64");
    ReduceScratch* scr = nullptr;
    {
        // cudaGetSymbolAddress also creates the device's context on a first call, so the id is
        // read after it when nothing is cached yet
        std::lock_guard<std::mutex> lock(g_mu);
        unsigned long long id = g_addr[dev] ? current_ctx_id() : 0;
        if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_reduce_scratch);
            if (e != cudaSuccess) return qaoa::report(QAOA_E_CUDA, cudaGetErrorString(e));
            g_addr[dev] = static_cast<ReduceScratch*>(p);
            g_ctx_id[dev] = current_ctx_id();
        }
        scr = g_addr[dev];
    }
    // every slot the kernels read is written earlier in the same call: nothing to clear
    e = qaoa::launch_reduce_state(false, n, psi, expect ? E : nullptr, k, scr->expect, scr->prob,
                                  scr->idx, expect, idx, prob, (cudaStream_t)stream);
    if (e != cudaSuccess) return qaoa::report(QAOA_E_CUDA, cudaGetErrorString(e));
    return QAOA_OK;
}
