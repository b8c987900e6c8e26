// qaoa_kernels.h -- internal interface between the C-ABI layer (qaoa_api.cu) and the kernel
// translation units of libqaoa. Not installed; the public interface is include/qaoa.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qaoa.h"

namespace qaoa {

// Record `msg` as the calling thread's last error (qaoa_last_error) and return s.
qaoa_status report(qaoa_status s, const char* msg);

enum InstFlags : int {
    F_GRAD = 1,       // run the adjoint sweep (d<C>/d gamma, d<C>/d beta)
    F_INIT_PSI = 2,   // start from psi_in instead of |+>
};

// One instance of the batched forward (and optional adjoint) computation. All pointers are
// device pointers; optional outputs are nullptr when not wanted.
template <typename T>
struct InstDesc {
    int n, p, k, flags;
    const T* Q;          // n x n row-major QUBO (energies are built from it), or nullptr
    const T* E_in;       // 2^n energies when Q is nullptr
    const T* gamma;      // p values
    const T* beta;       // p values
    const void* psi_in;  // initial state (F_INIT_PSI), complex of T
    void* psi_out;       // final state, complex of T
    T* E_out;            // energies
    double* expect;      // <C>
    uint64_t* topk_idx;  // k indices
    double* topk_prob;   // k probabilities
    double* dgamma;      // p values (F_GRAD)
    double* dbeta;       // p values (F_GRAD)
};

// ---- resident tier: one CTA per instance, whole state in shared memory -----------------
// Largest n the resident tier holds (forward / adjoint), per real type.
constexpr int RES_NMAX_F = 14, RES_NMAX_F_ADJ = 13;
constexpr int RES_NMAX_D = 13, RES_NMAX_D_ADJ = 12;

// rmax: widest forward register window (qubits) a launch uses; the block has 2^(n - window)
// threads (32..512), so a narrower window means more threads per instance.
constexpr int RES_RMAX = 8;   // no narrowing
size_t resident_smem_bytes(bool dbl, int n, int p, bool grad, int rmax = RES_RMAX);
int resident_threads(bool dbl, int n, int rmax = RES_RMAX);
// Launch a resident-tier kernel over `count` device descriptors (all with the same n).
// queue: device int zeroed by the caller before the launch (work counter). With desc ==
// nullptr the host descriptor `one` is passed by value and run by one block.
cudaError_t launch_resident(bool dbl, const void* desc, int count, int n, int pmax, bool grad,
                            int* queue, int grid, cudaStream_t st, const void* one = nullptr,
                            int rmax = RES_RMAX);
int resident_max_blocks_per_sm(bool dbl, int n, int pmax, bool grad, int rmax = RES_RMAX);

// ---- cluster tier: one cluster of 2^(n-L) CTAs per complex64 instance (15 <= n <= 18) ----
constexpr int CL_NMIN = 15, CL_NMAX = 18;
size_t cluster_smem_bytes(int n, int L, int p);
// With max_clusters != nullptr nothing is launched: the occupancy limit of active clusters is
// returned there instead. desc: device array of `count` descriptors of the same n.
cudaError_t launch_cluster(const void* desc, int count, int n, int L, int pmax, int clusters,
                           cudaStream_t st, int* max_clusters);

}  // namespace qaoa
