// qaoa_stream.h -- internal types of the HBM-streaming tier of libqaoa.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qaoa {

// One HBM pass over all tiles of the instances of a launch (uniform for the launch).
struct StreamPass {
    int n;          // qubits of the instances of this launch
    int tb;         // tile bits
    int kind;       // 0: contiguous tile (qubits 0..tb-1); 1: c low + h high qubits [s, s+h)
    int c, s, h;
    int la, lb;     // layers covered (lb <= la + 1)
    int ph_first;   // the cost of layer la opens this pass
    int init;       // generate |+> instead of reading psi
    int fin;        // last pass: per-tile <C> partials and top-k candidates
    int k;          // top-k length when fin
    int need_e;     // the pass reads the energies
    int keep_frame; // fin pass of a gradient run: leave psi in the rotated frame for the adjoint
    int no_store;   // fin pass whose final state nobody reads: reductions only, no write-back
};

// One instance of a streaming launch (device pointers).
template <typename T>
struct StreamInst {
    int p;
    const T* Q;           // n x n QUBO the energies are built from (batched energy kernel)
    double amp0;          // 2^{-n/2}
    const T* gamma;
    const T* beta;
    void* psi;            // 2^n complex state in HBM (in/out)
    const T* E;           // 2^n energies in HBM
    double* part_expect;  // 2^(n - tb) tile partials
    double* part_topp;    // 2^(n - tb) * k
    uint32_t* part_topz;  // 2^(n - tb) * k
    double* expect;
    uint64_t* topk_idx;
    double* topk_prob;
    // adjoint (gradient runs only)
    void* lam;            // 2^n complex adjoint state in HBM
    double* part_grad;    // adjoint passes * 2^(n - adjoint tile bits) * 4 per-tile partials
    double* dgamma;       // p
    double* dbeta;        // p
};

int stream_tile_bits(bool dbl);
// Tile bits of the adjoint passes: one bit fewer than the forward tiles, so that two CTAs
// (psi, lam and E tiles each) share an SM.
int stream_adj_tile_bits(bool dbl);
// Fill the pass list of a p-layer run on n qubits with tiles of tb bits (tb < 0: the forward
// tile size); returns the number of passes or -1.
int stream_plan(bool dbl, int n, int p, int k, StreamPass* out, int max_out, int tb = -1);
size_t stream_smem_bytes(bool dbl);
// insts: device array of `count` instances, or nullptr to pass the host instance `one` by value.
cudaError_t launch_stream_pass(bool dbl, const StreamPass& P, const void* insts, int count,
                               int grid, cudaStream_t st, const void* one = nullptr);
// <C> and top-k of each instance from its tile partials; with many tiles and k > 0 a first
// merge level runs as its own kernel (stream_finalize_two_level: two launches instead of one).
cudaError_t launch_stream_finalize(bool dbl, const void* insts, int count, uint64_t ntiles, int k,
                                   cudaStream_t st, const void* one = nullptr);
bool stream_finalize_two_level(uint64_t ntiles, int k);
// Adjoint pass `si` (pass P of the adjoint plan, i.e. stream_plan with the adjoint tile bits,
// run backwards on psi and lam): lam_first forms lam = E psi on load, store == 0 skips writing
// the states back (last adjoint pass).
cudaError_t launch_stream_adj_pass(bool dbl, const StreamPass& P, int si, bool lam_first, bool store,
                                   const void* insts, int count, int grid, cudaStream_t st,
                                   const void* one = nullptr);
// Sum the per-tile gradient partials of the S passes into dgamma / dbeta (fixed order).
cudaError_t launch_stream_grad_reduce(bool dbl, const StreamPass* passes, int S, const void* insts,
                                      int count, uint64_t ntiles, cudaStream_t st,
                                      const void* one = nullptr);
size_t stream_adj_smem_bytes(bool dbl);
cudaError_t launch_energy(bool dbl, int n, const void* Q, void* E, cudaStream_t st);
// Energies of `count` streaming instances (E written through insts[i].E from insts[i].Q).
cudaError_t launch_energy_batch(bool dbl, int n, const void* insts, int count, cudaStream_t st);
// Blocks of the standalone reduction of a 2^n state: one per 8192 amplitudes, 1 to 1024.
constexpr int reduce_parts(int n) {
    return (int)(((1ull << n) + 256 * 32 - 1) / (256 * 32) > 1024 ? 1024
                 : ((1ull << n) + 256 * 32 - 1) / (256 * 32) < 1 ? 1
                 : ((1ull << n) + 256 * 32 - 1) / (256 * 32));
}
cudaError_t launch_reduce_state(bool dbl, int n, const void* psi, const void* E, int k,
                                double* part_expect, double* part_topp, uint32_t* part_topz,
                                double* expect, uint64_t* topk_idx, double* topk_prob,
                                cudaStream_t st);

}  // namespace qaoa
