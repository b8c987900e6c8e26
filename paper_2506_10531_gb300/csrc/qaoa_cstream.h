// qaoa_cstream.h -- internal interface of the cluster-streaming tier (k_cstream.cu): complex64
// forward runs of CS_NMIN..CS_NMAX qubits, one thread-block cluster per instance, tiles of
// 2^CS_TILE_BITS amplitudes moved between L2 and shared memory by TMA.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace qaoa {

constexpr int CS_TILE_BITS = 13;
constexpr int CS_NMIN = 15, CS_NMAX = 17;
constexpr size_t CS_MAPS_BYTES = 4 * 128;   // four CUtensorMap per instance, 64-byte aligned

// The driver's tensor-map encoder could be found.
bool cstream_available();
// Size of one device descriptor (plan header entry).
size_t cstream_inst_bytes();
// CTAs per cluster for n qubits.
int cstream_cluster_size(int n);
// Occupancy limit of active clusters for n qubits (0 when none fits).
cudaError_t cstream_max_clusters(int n, int* out);
// Encode the four tensor maps of an instance (state and energies at psi / E, 16-byte aligned)
// into maps_out (host memory, CS_MAPS_BYTES, 64-byte aligned). False if the driver refuses.
bool cstream_encode_maps(int n, void* psi, void* E, void* maps_out);
// Host image of one device descriptor; maps_dev is the device address of its four maps.
void cstream_fill_inst(void* out, int n, int p, int k, bool out_psi, const float* Q, const float* gamma,
                       const float* beta, double* expect, uint64_t* topk_idx, double* topk_prob,
                       const void* maps_dev);
// One launch over `count` descriptors (device array, same n): `clusters` clusters walk them
// round-robin; a bounded wait that ran out sets bit 0 of *status.
cudaError_t launch_cstream(int n, const void* insts, int count, int clusters, unsigned* status, cudaStream_t st);

}  // namespace qaoa
