// msf_tiled.h -- host-visible declarations of the tiled (temporally blocked)
// ghost-state and interface-velocity extensions of two-dimensional grids
// (FP32-bulk form): one launch runs all K sweeps of a 16 x 16 tile in shared
// memory over the tile plus a K-cell halo. The ghost-state sweeps repeat the
// one-sweep kernel's arithmetic; the velocity sweeps sum in the bulk type.
#pragma once
#include <cuda_runtime.h>

#include "msf_types.cuh"

namespace msf {

constexpr int TILED_T = 16;       // tile edge (cells)
constexpr int TILED_MAX_SWEEPS = 8;  // larger sweep counts use the one-sweep kernels

struct TiledOps {
  // K ghost-state sweeps from (Win, fin) to (Wout, fout); Wout != Win
  cudaError_t (*extend)(const Grid&, const Bufs&, const void* Win, void* Wout, const uint8_t* fin, uint8_t* fout,
                        int K, cudaStream_t);
  // K interface-velocity sweeps from (vin, fin) to (vout, fout), sums in the
  // bulk type; vout != vin
  cudaError_t (*extend_vel)(const Grid&, const Bufs&, const double* vin, double* vout, const uint8_t* fin,
                            uint8_t* fout, int K, cudaStream_t);
};
const TiledOps* tiled_ops_f32();

}  // namespace msf
