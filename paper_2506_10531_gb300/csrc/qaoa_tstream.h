// qaoa_tstream.h -- internal interface of the TMA streaming passes (k_tstream.cu): the forward
// and adjoint passes of the HBM tier for complex64, with tiles moved by TMA.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "qaoa_stream.h"

namespace qaoa {

// Shape of the tensor map of a pass (TMA coordinates of a tile): kind A; kind B with h <= 8 and
// qubits above the chunk (5-D) or without (4-D); kind B with h = 9, whose 512 high values are
// split over two box dimensions (at most 256 each), 5-D or 4-D.
enum : int { TS_A = 0, TS_B5 = 1, TS_B4 = 2, TS_B9_5 = 3, TS_B9_4 = 4, TS_A3 = 5 };   // TS_A3: kind A of
// the adjoint's 12-bit tiles, 3-D
// Tile bits of the adjoint passes (the adjoint plan of stream_plan with stream_adj_tile_bits).
constexpr int TSA_TB = 12;

struct TsPass {
    int bmode;          // TS_*
    int midbits;        // kind B: tile-index bits below the chunk (s - c)
    int map;            // index of this pass's state map among an instance's maps
    int emap;           // index of its energy map
    int maps_per_inst;  // maps per instance in the plan's map array
};

constexpr size_t TS_MAP_BYTES = 128;   // one CUtensorMap, 64-byte aligned

// The driver's tensor-map encoder could be found.
bool tstream_available();
size_t tstream_smem_bytes();
TsPass tstream_pass_geometry(const StreamPass& P, int map, int emap, int maps_per_inst);
// Encode the tensor maps of pass P (any pass of the same kind and chunk gives the same maps) for
// a state at psi and its energies at E (both 16-byte aligned) into psi_map / e_map (host,
// 64-byte aligned).
bool tstream_encode_maps(const StreamPass& P, void* psi, void* E, void* psi_map, void* e_map);
// One pass over `count` instances (device array of StreamInst<float>) whose maps start at `maps`
// (device); a bounded wait that ran out sets bit 0 of *status.
cudaError_t launch_tstream_pass(const StreamPass& P, const TsPass& T, const void* insts, int count,
                                const void* maps, int grid, unsigned* status, cudaStream_t st);

// Adjoint passes (tiles of TSA_TB bits, kind-B chunks of h <= 8 high qubits): per pass shape
// three maps (state psi, adjoint state lam, energies) at indices T.map, T.map + 1, T.map + 2.
size_t tstream_adj_smem_bytes();
TsPass tstream_adj_geometry(const StreamPass& P, int map, int maps_per_inst);
bool tstream_encode_adj_maps(const StreamPass& P, void* psi, void* lam, void* E, void* maps3);
// Adjoint pass `si` of the adjoint plan over `count` instances (see launch_stream_adj_pass).
cudaError_t launch_tstream_adj_pass(const StreamPass& P, const TsPass& T, int si, bool lam_first, bool store,
                                    const void* insts, int count, const void* maps, int grid, unsigned* status,
                                    cudaStream_t st);

}  // namespace qaoa
