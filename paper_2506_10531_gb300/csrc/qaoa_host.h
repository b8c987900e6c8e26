// qaoa_host.h -- internal host functions of the DQAOA steps (dqaoa_host.cpp).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace qaoa {
int draw_random(int N, int m, int k, uint64_t seed, uint64_t cycle, int32_t* idx);
int draw_ifd(const double* Q, int N, const uint8_t* x, int m, int k, int32_t* idx, bool signed_rank = false);
// Strong-interaction graph of the BFS / PFS decompositions for (Q, k), CSR form.
struct StrongGraph {
    int N = 0, k = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> nbr;
    int words = 0;                // > 0: rows also as bitsets of `words` 64-bit words (dense graphs)
    std::vector<uint64_t> bits;
};
void build_strong_graph(const double* Q, int N, int k, StrongGraph* g);
int draw_graph(const double* Q, int N, const uint8_t* x, int method, int m, int k, int32_t* idx,
               const StrongGraph* g = nullptr, bool signed_rank = false);
void build_subqubos(const double* Q, int N, const uint8_t* x, int m, int k, const int32_t* idx,
                    int conditioned, double* Qsub);
// State the merge can carry from one call to the next on the same Q: h = Qx, E(x), tau.
struct MergeCache {
    std::vector<double> h;
    double energy = 0.0, tau = 0.0;
    bool valid = false;
    // variables flipped since the cycle began (merges of one cycle may come in chunks): a
    // candidate's precomputed pair term holds only while no variable of its sub-QUBO has flipped
    std::vector<uint8_t> chg;
};
// h = Qx, tau = 1e-12 sum |Q| and E(x) for a merge without a cached h: rows in blocks of MERGE_RB,
// each block's rows added in ascending order, the blocks added in ascending order (the order the
// device set-up uses, so both give the same bits); tau from the column sums of |Q| added in
// ascending column order; E(x) = sum over x_i = 1 of h_i, ascending.
constexpr int MERGE_RB = 64;   // rows per block of the merge set-up (device and host)
void merge_setup_host(const double* Q, int N, const uint8_t* x, MergeCache* cache);
// The same from the device set-up's h and column sums.
void merge_setup_from(int N, const uint8_t* x, const double* h, const double* colabs, MergeCache* cache);
// qblk (optional): the m raw FP64 blocks Q[S_j, S_j] (k*k each, row-major), read instead of
// gathering the entries from Q (same values, contiguous). pair (optional, with a cache whose chg
// marks the flips of this cycle): candidate c of sub-QUBO j has pair term pair[j*K + c] against
// the x the cycle began with; it is used while no variable of S_j has flipped.
int merge(const double* Q, int N, uint8_t* x, int m, int k, const int32_t* idx, int K,
          const uint64_t* cand, double* energy_out, int* accepted_out, MergeCache* cache = nullptr,
          const double* qblk = nullptr, const double* pair = nullptr);
int merge_setup_blocks(int N);
// device set-up: scratch holds 2 * merge_setup_blocks(N) * N doubles; h, colabs: N doubles each
cudaError_t launch_merge_setup(const double* Q, int N, const uint8_t* x, double* scratch, double* h,
                               double* colabs, cudaStream_t st);
// pair terms of m*K candidates against x (device): idx m*k, qblk m*k*k, cand m*K, pair m*K.
// With expect and status given, pair is the start of a packed block: m*K pair terms, then the
// m*K candidates, the m <C> values (copied from expect) and the status word (from *status).
cudaError_t launch_cand_pair(int m, int k, int K, const int32_t* idx, const uint8_t* x, const double* qblk,
                             const uint64_t* cand, double* pair, cudaStream_t st, const double* expect = nullptr,
                             const unsigned* status = nullptr);
// bytes of the packed block of m sub-QUBOs with K candidates each
inline size_t cand_pack_bytes(int m, int K) { return ((size_t)m * K * 16 + (size_t)m * 8 + 16 + 255) & ~(size_t)255; }
cudaError_t launch_subqubo(const double* Q, int N, const uint8_t* x, int m, int k,
                           const int32_t* idx, int conditioned, float* qsub, cudaStream_t st,
                           double* qblk = nullptr, double* qdiag = nullptr);
// the shot of lowest sub-QUBO energy per sub-QUBO (FP64: off-diagonal entries from qblk, the
// diagonal from qdiag as launch_subqubo writes them); ties go to the smaller bitstring
cudaError_t launch_best_shot(int m, int k, int shots, const double* qblk, const double* qdiag,
                             const uint64_t* z, uint64_t* best, cudaStream_t st);
cudaError_t launch_plain_layers(int n, int p, const float* gamma, const float* beta,
                                const float* E, float2* psi, int init_plus, cudaStream_t st,
                                int* kernels);
int sample_part_bits(int n);
size_t sample_scratch_bytes(int n);
// `count` states of 2^n amplitudes, one after the other from psi; state c draws `shots` shots
// with the uniforms u[c * shots ...] into out[c * shots ...]; scratch: count * sample_scratch_bytes(n)
cudaError_t launch_sample(int n, const void* psi, int count, int64_t shots, const double* u, uint64_t* out,
                          double* scratch, cudaStream_t st);
cudaError_t launch_adam(int count, float* theta, const double* grad, float* m, float* v, int step,
                        float lr, float b1, float b2, float eps, int minimise, cudaStream_t st);
}  // namespace qaoa

// Plans placed in caller memory (used by the serving loop; qaoa_api.cu).
#include "../../include/qaoa.h"
namespace qaoa {
size_t plan_inst_scratch_bytes(qaoa_ctx* c, int n, int p, int k, bool grad);
size_t plan_header_bound(int count);
qaoa_status plan_create_placed(qaoa_ctx* c, const qaoa_inst* desc, int count, const qaoa_batch_io* io,
                               void* base, size_t bytes, cudaStream_t st, void* staging,
                               size_t staging_bytes, qaoa_plan** out);
qaoa_status set_error(qaoa_status s, const char* msg);
}  // namespace qaoa
