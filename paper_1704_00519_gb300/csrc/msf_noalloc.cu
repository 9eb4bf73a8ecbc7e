// msf_noalloc.cu -- CFL time step of one material's state with no device
// allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs inside a region another
// framework has reserved (a caching allocator that owns all device memory, so
// a raw cudaMalloc fails or fragments it), real-time loops that must not hit
// the implicit device synchronisation of cudaMalloc/cudaFree, and embedded
// users with a fixed device-memory budget. For them this entry point keeps its
// only scratch -- one partial maximum per thread block -- in a fixed array
// that lives in the library image on every device that loads it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/msf.h"

extern "C" void msf_internal_set_error(const char* msg);  // defined with the other entry points

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = MSF_NOALLOC_MAX_CELLS / kThreads;

// per-block partial maxima of the wave-speed bound; shared by every call on a device
static __device__ __align__(256) double g_partial_max[kMaxBlocks];

struct CflArgs {
  int dim;
  double gamma, pinf, gm1, gpi, rh[3];
};

// maximum that keeps a NaN: a non-physical cell must not vanish in the reduction
__device__ inline double max_keep_nan(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }

// one thread per cell: sum_d (|u_d| + c) / h_d of the state, block maximum to
// scratch; a cell with rho <= 0, c^2 <= 0 or a non-finite value gives NaN
__global__ void k_cfl_partial(const double* U, long long cells, CflArgs a, double* partial) {
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  double s = 0.0;
  if (i < cells) {
    const int D = a.dim;
    const double rho = U[i];
    double vel[3] = {0.0, 0.0, 0.0};
    double q = 0.0;
    for (int d = 0; d < D; d++) vel[d] = U[(long long)(1 + d) * cells + i] / rho;
    for (int d = 0; d < D; d++) q += vel[d] * vel[d];
    const double ke = 0.5 * rho * q;
    const double p = a.gm1 * (U[(long long)(D + 1) * cells + i] - ke) - a.gpi;
    const double c2 = (a.gamma * (p + a.pinf)) / rho;
    if (!(rho > 0.0) || !(c2 > 0.0)) {
      s = __longlong_as_double(0x7ff8000000000000LL);
    } else {
      const double c = sqrt(c2);
      for (int d = 0; d < D; d++) s += (fabs(vel[d]) + c) * a.rh[d];
      if (!isfinite(s)) s = __longlong_as_double(0x7ff8000000000000LL);
    }
  }
  __shared__ double red[kThreads];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = kThreads / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] = max_keep_nan(red[threadIdx.x], red[threadIdx.x + k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// one block: maximum over the partials of this call, then dt = cfl / max; a
// NaN partial (a non-physical cell) or a zero bound gives dt = NaN
__global__ void k_cfl_final(const double* partial, int nblocks, double cfl, double* dt_out) {
  double m = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += kThreads) m = max_keep_nan(m, partial[k]);
  __shared__ double red[kThreads];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int k = kThreads / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] = max_keep_nan(red[threadIdx.x], red[threadIdx.x + k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *dt_out = red[0] > 0.0 ? cfl / red[0] : __longlong_as_double(0x7ff8000000000000LL);
}

std::mutex g_mu;
double* g_scratch[256] = {};  // device address of g_partial_max per device ordinal

}  // namespace

extern "C" msf_status msf_cfl_dt_noalloc(const double* U, int64_t cells, int32_t dim, const msf_eos* eos,
                                         const double* h, double cfl, double* dt_out, void* stream) {
  if (!U || !eos || !h || !dt_out) {
    msf_internal_set_error("msf_cfl_dt_noalloc: NULL argument");
    return MSF_EINVAL;
  }
  if (dim < 1 || dim > 3 || cells < 1) {
    msf_internal_set_error("msf_cfl_dt_noalloc: dim must be 1..3 and cells >= 1");
    return MSF_EINVAL;
  }
  if (cells > MSF_NOALLOC_MAX_CELLS) {
    msf_internal_set_error("msf_cfl_dt_noalloc: more cells than MSF_NOALLOC_MAX_CELLS (4194304); "
                           "use msf_step / msf_last_dt for larger states");
    return MSF_EINVAL;
  }
  if (eos->kind != MSF_EOS_STIFFENED || !(eos->gamma > 1.0) || !(eos->pinf >= 0.0) || !(cfl > 0.0 && cfl <= 1.0)) {
    msf_internal_set_error("msf_cfl_dt_noalloc: need a stiffened gas with gamma > 1, pinf >= 0, 0 < cfl <= 1");
    return MSF_EINVAL;
  }
  CflArgs a;
  a.dim = dim;
  a.gamma = eos->gamma;
  a.pinf = eos->pinf;
  a.gm1 = eos->gamma - 1.0;
  a.gpi = eos->gamma * eos->pinf;
  for (int d = 0; d < 3; d++) a.rh[d] = 0.0;
  for (int d = 0; d < dim; d++) {
    if (!(h[d] > 0.0) || !std::isfinite(h[d])) {
      msf_internal_set_error("msf_cfl_dt_noalloc: cell sizes must be finite and > 0");
      return MSF_EINVAL;
    }
    a.rh[d] = 1.0 / h[d];
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    msf_internal_set_error("msf_cfl_dt_noalloc: no current CUDA device");
    return MSF_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // Device address of the scratch array, looked up with this device current.
  // The first call on a device does it; later calls look it up again unless
  // the stream is being captured (the module may have been reloaded at a new
  // address after a context reset), and a capturing call uses the address the
  // last call outside capture found.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
  if (capturing) cudaGetLastError();  // clear a refused query
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!capturing) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_partial_max);
      if (e != cudaSuccess || !p) {
        msf_internal_set_error("msf_cfl_dt_noalloc: cudaGetSymbolAddress failed");
        return MSF_ECUDA;
      }
      g_scratch[dev] = (double*)p;
    } else if (!g_scratch[dev]) {
      msf_internal_set_error("msf_cfl_dt_noalloc: the first call on a device must come before any stream capture");
      return MSF_ESTATE;
    }
    scratch = g_scratch[dev];
  }
  const int nblocks = (int)((cells + kThreads - 1) / kThreads);
  k_cfl_partial<<<nblocks, kThreads, 0, s>>>(U, cells, a, scratch);
  k_cfl_final<<<1, kThreads, 0, s>>>(scratch, nblocks, cfl, dt_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    msf_internal_set_error("msf_cfl_dt_noalloc: kernel launch failed");
    return MSF_ECUDA;
  }
  return MSF_OK;
}
