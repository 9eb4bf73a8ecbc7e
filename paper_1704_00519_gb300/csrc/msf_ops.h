// msf_ops.h -- host-side launch table shared by the runtime and the two
// kernel translation units (FP64 strict, FP32 bulk).
#pragma once
#include <cuda_runtime.h>

#include "msf_types.cuh"

namespace msf {
struct BatchEntry;

// launchers of the kernels whose bulk arithmetic type depends on the precision
struct Ops {
  size_t tsize;  // sizeof(T)
  void (*prim)(const Grid&, const Bufs&, const double* Qs, int nblk, cudaStream_t);
  void (*extend)(const Grid&, const Bufs&, const void* Win, void* Wout, const uint8_t* fin, uint8_t* fout, int nblk,
                 cudaStream_t);
  void (*cons)(const Grid&, const Bufs&, const double* Qs, const void* W, const uint8_t* f, int nblk, cudaStream_t);
  void (*bc_uhat)(const Grid&, const Bufs&, const double* Qs, cudaStream_t);
  void (*dt)(const Grid&, const Bufs&, const double* Qs, cudaStream_t);
  void (*interface)(const Grid&, const Bufs&, const double* Qs, int stage, int nblk, cudaStream_t);
  // Qsf: FP32 copy of Qs for the bulk staging (null: convert Qs); Qof: FP32
  // copy of Qout to write (null: none); both ignored in FP64 contexts
  cudaError_t (*flux)(const Grid&, const Bufs&, const double* Qs, const double* Qn, double* Qout, double beta,
                      double omb, const BndBase&, const float* Qsf, float* Qof, cudaStream_t);
  // FP32-bulk form: Q[0] rounded into its FP32 copy Qf[0], for the band
  // cells of the step (band_only = 1, at the end of a step) or for every cell
  // (after a host-side write of Q[0]); nothing in FP64 contexts
  void (*qf_copy)(const Grid&, const Bufs&, int band_only, int nblk, cudaStream_t);
  // n_steps steps of every 1D instance of a batch, one CTA of bs threads per instance
  cudaError_t (*batched)(const BatchEntry* tab, const int* order, int n_inst, int n_steps, int bs, cudaStream_t);
};
void launch_set_tend_all(const BatchEntry* tab, int n, double t_end, cudaStream_t);
const Ops* ops_f64();
const Ops* ops_f32();

// precision-independent (FP64) kernels, compiled in the strict FP64 unit
void launch_step_begin(const Bufs&, cudaStream_t);
void launch_bc_phichi(const Grid&, const Bufs&, cudaStream_t);
void launch_masks(const Grid&, const Bufs&, cudaStream_t);
void launch_geometry(const Grid&, const Bufs&, const double* Qs, const double* mass, int nblk, cudaStream_t);
void launch_band_save(const Grid&, const Bufs&, int nblk, cudaStream_t);
void launch_dt_finalize(const Grid&, const Bufs&, cudaStream_t);
void launch_step_end(const Bufs&, cudaStream_t);
void launch_extend_vel(const Grid&, const Bufs&, const double* vin, double* vout, const uint8_t* fin, uint8_t* fout,
                       int nblk, cudaStream_t);
void launch_ledger(const Grid&, const Bufs&, int nbnd, double w, cudaStream_t);
void launch_levelset(const Grid&, const Bufs&, const double* vel, double beta, double omb, int nblk, cudaStream_t);
void launch_scatter_phichi(const Grid&, const Bufs&, int nblk, cudaStream_t);
void launch_mix(const Grid&, const Bufs&, double* Qc, int nblk, cudaStream_t);
void launch_scale_sep(const Grid&, const Bufs&, int nblk, cudaStream_t);
void launch_reinit(const Grid&, const Bufs&, int nblk, cudaStream_t);
void launch_totals(const Grid&, const double* Q, double* out, cudaStream_t);
// start-up and state transfer
void launch_init_levelset(const Grid&, const Bufs&, const double* phi_in, const int32_t* chi_in, cudaStream_t);
void launch_init_mass(const Grid&, const Bufs&, const double* prim_in, double* mass, cudaStream_t);
void launch_init_state(const Grid&, const Bufs&, const double* prim_in, cudaStream_t);
// free-surface ambient held at alpha (fs_rho, 0, p(t)): k = -2 at t = 0, -1 at
// the step's start, k >= 0 at the time of stage k
void launch_hold_ambient(const Grid&, const Bufs&, double* Qc, int k, cudaStream_t);
void launch_gather(const Grid&, const Bufs&, int which, double* out, int32_t* iout, cudaStream_t);
void launch_scatter_state(const Grid&, const Bufs&, const double* Q, const double* phi, const int32_t* chi,
                          cudaStream_t);
void launch_check_inputs(const Grid&, const double* phi, const int32_t* chi, const double* prim, unsigned* flag,
                         cudaStream_t);
}  // namespace msf
