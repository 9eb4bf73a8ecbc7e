// msf_adjoint.h -- host-visible declarations of the adjoint kernels of one
// TVD-RK3 step at frozen interface evolution (the replay of a recorded step).
#pragma once
#include <cuda_runtime.h>

#include "msf_types.cuh"

namespace msf {

// adjoint workspace of one instance (device arrays; ncell = padded cells)
struct AdjBufs {
  double* LA;        // [N][NV][ncell] adjoint of the stage output, then of the stage input
  double* LN;        // [N][NV][ncell] accumulated adjoint of Q^n
  double* LU;        // [N][NV][ncell] adjoint of the stencil states (interior and halo cells)
  double* LQ;        // [N][NV][ncell] adjoint of Q^(s) through the band states
  double *LW0, *LW1; // [N][NV][ncell] adjoint of the primitive states (extension sweeps)
  uint8_t* lvl;      // [N][ncell] sweep that filled a ghost state (0: real, 0xff: never)
  double* mixt;      // [nbmax][N][NV] band scratch of the mixing adjoint
  uint8_t* mixn[3];  // mixing records of each stage (as Bufs::mixn / mixoff / mixbeta)
  uint8_t* mixoff[3];
  double* mixbeta[3];
  double* mixT[3];
  double* aband[4];  // [nbmax][N] band volume fractions after each geometry: 0 step start, s+1 after stage s
  double* deos;      // [MAXM][2] d/d(gamma_m, pinf_m)
  double* dinf;      // [3][2][5] d/d(inflow primitive state)
};

// launchers whose stencil-state type depends on the precision of the context
struct AdjOps {
  void (*flux)(const Grid&, const Bufs&, const AdjBufs&, const double* Qs, double omb_dt, cudaStream_t);
  void (*interface)(const Grid&, const Bufs&, const AdjBufs&, const double* Qs, double omb_dt, int nblk,
                    cudaStream_t);
  void (*cons)(const Grid&, const Bufs&, const AdjBufs&, const void* W, const uint8_t* f, double* lw, int nblk,
               cudaStream_t);
};
const AdjOps* adj_ops_f64();
const AdjOps* adj_ops_f32();

// precision-independent adjoint kernels (FP64 unit)
void launch_adj_begin(const Bufs&, const double* tape_dt, cudaStream_t);
void launch_adj_level(const Grid&, const Bufs&, const AdjBufs&, const uint8_t* f, int k, int nblk, cudaStream_t);
void launch_adj_ext(const Grid&, const Bufs&, const AdjBufs&, const double* lin, double* lout, int k, int nblk,
                    cudaStream_t);
void launch_adj_prim(const Grid&, const Bufs&, const AdjBufs&, const double* Qs, const double* lw, int nblk,
                     cudaStream_t);
void launch_adj_mix(const Grid&, const Bufs&, const AdjBufs&, int stage, const uint8_t* chi_next, int nblk,
                    cudaStream_t);
void launch_adj_bc(const Grid&, const Bufs&, const AdjBufs&, cudaStream_t);
void launch_adj_combine(const Grid&, const Bufs&, const AdjBufs&, double beta, double omb, int last_stage,
                        cudaStream_t);
void launch_adj_alpha(const Grid&, const Bufs&, double* aband, int save, int nblk, cudaStream_t);
void launch_adj_io(const Grid&, const AdjBufs&, const double* lam_out, double* lam_in, int dir, cudaStream_t);
void launch_adj_end(const Bufs&, const double* tape_t, cudaStream_t);

}  // namespace msf
