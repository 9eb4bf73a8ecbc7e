// msf_tiled.h -- host-visible declaration of the tiled (temporally blocked)
// ghost-state extension of two-dimensional grids: one launch runs all K
// sweeps of a 16 x 16 tile in shared memory over the tile plus a K-cell halo;
// every cell's arithmetic is that of the one-sweep kernel, in the same order,
// so the results are identical.
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
};
const TiledOps* tiled_ops_f32();

}  // namespace msf
