// msf_f64.cu -- strict FP64 unit (compiled with -fmad=false): the FP64
// instantiation of the precision-dependent kernels plus every kernel whose
// arithmetic is FP64 in both precision modes (geometry, correction, level set,
// mixing, scale separation, band maintenance, totals) and the start-up and
// state-transfer kernels.
#include "msf_kernels.cuh"
#include "msf_ops.h"
#include "msf_prec.inc"
#include "msf_adjoint_common.cuh"

namespace msf {

const Ops* ops_f64() {
  static const Ops ops = make_ops<double>();
  return &ops;
}
const AdjOps* adj_ops_f64() {
  static const AdjOps ops = make_adj_ops<double>();
  return &ops;
}

static int grid_blocks(long long n) {
  long long b = (n + NTHREADS - 1) / NTHREADS;
  if (b > 1216) b = 1216;  // 152 SMs x 8 resident CTAs of 256 threads
  if (b < 1) b = 1;
  return (int)b;
}

// ------------------------------------------------------------ start-up
__global__ void k_init_levelset(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* phi_in, const int32_t* chi_in) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.n_interior;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, idx);
    double ph = phi_in[idx];
    if (ph > g.cap) ph = g.cap;
    b.phi[c] = ph;
    b.chi[c] = (uint8_t)chi_in[idx];
  }
}
__global__ void k_init_mass(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* prim, double* mass) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.n_interior;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, idx);
    for (int m = 0; m < g.N; m++)
      mass[qidx(g, m, 0, c)] = alpha_of(g, b, c, m) * prim[((long long)m * g.NV) * g.n_interior + idx];
  }
}
__global__ void k_init_state(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* prim) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.n_interior;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, idx);
    for (int m = 0; m < g.N; m++) {
      const double a = alpha_of(g, b, c, m);
      double w[5], u[5];
      for (int v = 0; v < g.NV; v++) w[v] = prim[((long long)m * g.NV + v) * g.n_interior + idx];
      prim_to_cons<double>(g, m, g.D, w, u);
      for (int v = 0; v < g.NV; v++) b.Q[0][qidx(g, m, v, c)] = a > 0.0 ? a * u[v] : 0.0;
    }
  }
}
__global__ void k_check_inputs(const __grid_constant__ Grid g, const double* phi, const int32_t* chi, const double* prim, unsigned* flag) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.n_interior;
       idx += (long long)gridDim.x * blockDim.x) {
    unsigned f = 0;
    if (phi) {
      const double p = phi[idx];
      if (!(p >= 0.0) || !isfinite(p)) f |= 1u;
    }
    if (chi) {
      if (chi[idx] < 0 || chi[idx] >= g.N) f |= 2u;
    }
    if (prim)
      for (int m = 0; m < g.N; m++) {
        const double rho = prim[((long long)m * g.NV) * g.n_interior + idx];
        const double p = prim[((long long)m * g.NV + g.NV - 1) * g.n_interior + idx];
        bool fin = true;
        for (int v = 0; v < g.NV; v++) fin = fin && isfinite(prim[((long long)m * g.NV + v) * g.n_interior + idx]);
        if (!fin || !(rho > 0.0) || !(p + g.pinf[m] > 0.0)) f |= 4u;
      }
    if (f) atomicOr(flag, f);
  }
}

// -------------------------------------------------------- state transfer
__global__ void k_gather(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, int which, double* out, int32_t* iout) {
  const int N = g.N, NV = g.NV;
  const long long ni = g.n_interior;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ni;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, idx);
    const bool inb = b.bandidx[c] >= 0;
    switch (which) {
      case 0:  // Q
        for (int m = 0; m < N; m++)
          for (int v = 0; v < NV; v++) out[((long long)m * NV + v) * ni + idx] = b.Q[0][qidx(g, m, v, c)];
        break;
      case 1:  // alpha
        for (int m = 0; m < N; m++) out[(long long)m * ni + idx] = alpha_of(g, b, c, m);
        break;
      case 2:
        out[idx] = b.phi[c];
        break;
      case 3:
        iout[idx] = b.chi[c];
        break;
      case 11:  // exchange flux
        for (int m = 0; m < N; m++)
          for (int v = 0; v < NV; v++)
            out[((long long)m * NV + v) * ni + idx] = (inb && (b.gflag[c] & GF_CUT)) ? b.X[qidx(g, m, v, c)] : 0.0;
        break;
      case 13:
        out[idx] = (b.gflag[c] & GF_MIXED) ? 1.0 : 0.0;
        break;
      case 14:
        out[idx] = (double)b.smask[c];
        break;
      default:
        break;
    }
  }
}
// stencil state of the last stage: band cells from Uh, bulk cells from the
// stage's Q (the material of the cell) or NaN
template <typename T>
__global__ void k_gather_uh(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qs, double* out) {
  const int N = g.N, NV = g.NV;
  const long long ni = g.n_interior;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ni;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, idx);
    for (int m = 0; m < N; m++) {
      T u[5];
      interior_uhat<T>(g, b, Qs, c, m, u);
      for (int v = 0; v < NV; v++) out[((long long)m * NV + v) * ni + idx] = (double)u[v];
    }
  }
}
__global__ void k_gather_vel(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* vel, double* out) {
  const long long ni = g.n_interior;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ni;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, idx);
    for (int d = 0; d < 3; d++) out[d * ni + idx] = (b.bandidx[c] >= 0 && d < g.D) ? vel[d * g.ncell + c] : 0.0;
  }
}
__global__ void k_scatter_state(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Q, const double* phi, const int32_t* chi) {
  const long long ni = g.n_interior;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ni;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, idx);
    for (int m = 0; m < g.N; m++)
      for (int v = 0; v < g.NV; v++) b.Q[0][qidx(g, m, v, c)] = Q[((long long)m * g.NV + v) * ni + idx];
    b.phi[c] = phi[idx];
    b.chi[c] = (uint8_t)chi[idx];
  }
}

// ------------------------------------------------------------ launchers
void launch_step_begin(const Bufs& b, cudaStream_t s) { k_step_begin<<<1, 1, 0, s>>>(b); }
void launch_bc_phichi(const Grid& g, const Bufs& b, cudaStream_t s) {
  long long nh = g.ncell - g.n_interior;
  k_bc_phichi<<<grid_blocks(nh), NTHREADS, 0, s>>>(g, b);
}
void launch_masks(const Grid& g, const Bufs& b, cudaStream_t s) {
  const int nb = grid_blocks(g.ncell);
  k_xs<<<nb, NTHREADS, 0, s>>>(g, b);
  // dilate xs -> mtmp (x) -> xsS used as scratch (y) -> mtmp (z)
  const uint8_t* src = b.xs;
  uint8_t* bufs[2] = {b.mtmp, b.xsS};
  int w = 0;
  for (int d = 0; d < g.D; d++) {
    k_dilate<<<nb, NTHREADS, 0, s>>>(g, b, src, bufs[w], d);
    src = bufs[w];
    w ^= 1;
  }
  k_band<<<nb, NTHREADS, 0, s>>>(g, b, src);
}
void launch_geometry(const Grid& g, const Bufs& b, const double* Qs, const double* mass, int nblk, cudaStream_t s) {
  if (g.D == 3) cudaMemsetAsync(&b.ctl->geom_count, 0, sizeof(unsigned), s);
  cudaMemsetAsync(&b.ctl->ls_count, 0, sizeof(unsigned), s);
  k_geom_mat<<<nblk, BAND_THREADS, 0, s>>>(g, b);
  if (g.D == 3) k_geom_cut<<<nblk, BAND_THREADS, 0, s>>>(g, b);
  k_geom_cell<<<nblk, BAND_THREADS, 0, s>>>(g, b, Qs, mass);
}
void launch_band_save(const Grid& g, const Bufs& b, int nblk, cudaStream_t s) {
  k_band_save<<<nblk, BAND_THREADS, 0, s>>>(g, b);
}
void launch_dt_finalize(const Grid& g, const Bufs& b, cudaStream_t s) { k_dt_finalize<<<1, 1, 0, s>>>(g, b); }
void launch_step_end(const Bufs& b, cudaStream_t s) { k_step_end<<<1, 1, 0, s>>>(b); }
void launch_extend_vel(const Grid& g, const Bufs& b, const double* vin, double* vout, const uint8_t* fin,
                       uint8_t* fout, int nblk, cudaStream_t s) {
  k_extend_vel<<<nblk, BAND_THREADS, 0, s>>>(g, b, vin, vout, fin, fout);
}
void launch_set_tend_all(const BatchEntry* tab, int n, double t_end, cudaStream_t s) {
  k_set_tend_all<<<(n + 255) / 256, 256, 0, s>>>(tab, n, t_end);
}
void launch_ledger(const Grid& g, const Bufs& b, int nbnd, double w, cudaStream_t s) {
  const int nparts = (nbnd + NTHREADS - 1) / NTHREADS;
  if (nparts > 0) k_ledger_partial<<<nparts, NTHREADS, 0, s>>>(g, b, nbnd);
  k_ledger<<<1, NTHREADS, 0, s>>>(g, b, nparts, w);
}
void launch_levelset(const Grid& g, const Bufs& b, const double* vel, double beta, double omb, int nblk,
                     cudaStream_t s) {
  k_levelset<<<nblk, BAND_THREADS, 0, s>>>(g, b, vel, beta, omb);
  k_levelset_R<<<nblk, BAND_THREADS, 0, s>>>(g, b);
}
void launch_scatter_phichi(const Grid& g, const Bufs& b, int nblk, cudaStream_t s) {
  k_scatter_phichi<<<nblk, BAND_THREADS, 0, s>>>(g, b);
}
void launch_mix(const Grid& g, const Bufs& b, double* Qc, int nblk, cudaStream_t s) {
  k_mix_mark<<<nblk, BAND_THREADS, 0, s>>>(g, b, Qc);
  k_mix_weights<<<nblk, BAND_THREADS, 0, s>>>(g, b);
  k_mix_compute<<<nblk, BAND_THREADS, 0, s>>>(g, b, Qc);
  k_mix_scatter<<<nblk, BAND_THREADS, 0, s>>>(g, b, Qc);
}
void launch_scale_sep(const Grid& g, const Bufs& b, int nblk, cudaStream_t s) {
  k_scale_sep<<<nblk, BAND_THREADS, 0, s>>>(g, b, b.Q[0]);
  k_scatter_phichi<<<nblk, BAND_THREADS, 0, s>>>(g, b);
}
void launch_reinit(const Grid& g, const Bufs& b, int nblk, cudaStream_t s) {
  k_reinit<<<nblk, BAND_THREADS, 0, s>>>(g, b);
  k_scatter_phichi<<<nblk, BAND_THREADS, 0, s>>>(g, b);
}
void launch_totals(const Grid& g, const double* Q, double* out, cudaStream_t s) {
  k_totals<<<g.N * g.NV, NTHREADS, 0, s>>>(g, Q, out);
}
void launch_init_levelset(const Grid& g, const Bufs& b, const double* phi_in, const int32_t* chi_in, cudaStream_t s) {
  k_init_levelset<<<grid_blocks(g.n_interior), NTHREADS, 0, s>>>(g, b, phi_in, chi_in);
}
void launch_init_mass(const Grid& g, const Bufs& b, const double* prim_in, double* mass, cudaStream_t s) {
  k_init_mass<<<grid_blocks(g.n_interior), NTHREADS, 0, s>>>(g, b, prim_in, mass);
}
void launch_hold_ambient(const Grid& g, const Bufs& b, double* Qc, int k, cudaStream_t s) {
  k_hold_ambient<<<grid_blocks(g.n_interior), NTHREADS, 0, s>>>(g, b, Qc, k);
}
void launch_init_state(const Grid& g, const Bufs& b, const double* prim_in, cudaStream_t s) {
  k_init_state<<<grid_blocks(g.n_interior), NTHREADS, 0, s>>>(g, b, prim_in);
}
void launch_check_inputs(const Grid& g, const double* phi, const int32_t* chi, const double* prim, unsigned* flag,
                         cudaStream_t s) {
  k_check_inputs<<<grid_blocks(g.n_interior), NTHREADS, 0, s>>>(g, phi, chi, prim, flag);
}
void launch_gather(const Grid& g, const Bufs& b, int which, double* out, int32_t* iout, cudaStream_t s) {
  const int nb = grid_blocks(g.n_interior);
  if (which == 20) {
    k_gather_uh<double><<<nb, NTHREADS, 0, s>>>(g, b, b.Q[2], out);
  } else if (which == 21) {
    k_gather_uh<float><<<nb, NTHREADS, 0, s>>>(g, b, b.Q[2], out);
  } else if (which == 30) {
    k_gather_vel<<<nb, NTHREADS, 0, s>>>(g, b, b.vel0, out);
  } else if (which == 31) {
    k_gather_vel<<<nb, NTHREADS, 0, s>>>(g, b, b.vel1, out);
  } else {
    k_gather<<<nb, NTHREADS, 0, s>>>(g, b, which, out, iout);
  }
}
void launch_scatter_state(const Grid& g, const Bufs& b, const double* Q, const double* phi, const int32_t* chi,
                          cudaStream_t s) {
  k_scatter_state<<<grid_blocks(g.n_interior), NTHREADS, 0, s>>>(g, b, Q, phi, chi);
}

}  // namespace msf
