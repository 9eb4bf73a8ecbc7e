// msf_capi.cu -- host runtime and C ABI (include/msf.h) of the GB300 build of
// the conservative sharp-interface multi-material method (arXiv:1704.00519).
//
// The runtime owns every device allocation of a context, enqueues one
// TVD-RK3 step as a fixed kernel sequence per instance on the context's
// stream, captures that sequence once as a CUDA graph and replays it. Time,
// time step, the end time and every branch on them live on the device, so a
// replayed graph needs no host round trip; the only readback of msf_step is
// the 4-byte error word when the caller asks for synchronisation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/msf.h"
#include "msf_types.cuh"
#include "msf_ops.h"
#include "msf_adjoint.h"
#include "msf_tiled.h"

using namespace msf;

namespace {

struct Inst {
  Grid g;
  Bufs b;
  BndBase bb;
  int nbnd = 0;
  int nblk_band = 1;
  void* Fface = nullptr;     // batched stepping: face fluxes of a stage
  double* Aface = nullptr;   // batched stepping: face apertures of a stage
};

}  // namespace

struct msf_ctx {
  int dim = 0, N = 0, ninst = 0;
  msf_options opt{};
  cudaStream_t stream = nullptr;
  std::vector<Inst> inst;
  std::vector<void*> allocs;
  const Ops* ops = nullptr;
  const TiledOps* tops = nullptr;
  Ctl* h_ctl = nullptr;  // pinned readback of one control block
  unsigned* d_flag = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool graph_tried = false;
  long long graph_kernels = -1;  // kernel nodes of the captured step graph
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  long long launches = 0;  // kernel launches of the last enqueued step
  void* arena = nullptr;   // every device array of every instance
  bool batched = false;    // persistent one-CTA-per-instance stepping
  BatchEntry* d_tab = nullptr;
  int* d_order = nullptr;
  int bs = 0;              // autotuned CTA size of the batched kernel (0: not tuned yet)
  cudaEvent_t tev[2] = {nullptr, nullptr};
  bool sticky = false;
  std::string err;
  // adjoint workspace (allocated by the first taped, replayed or adjoint step)
  const AdjOps* aops = nullptr;
  AdjBufs adj{};
  bool adj_ready = false;
  double* h_pin = nullptr;  // pinned readback of dt / t and the gradient accumulators
};

static thread_local std::string g_create_err = "";

static msf_status fail(msf_ctx* c, msf_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_err = msg;
  return s;
}
#define CUDA_TRY(ctx, call)                                                                      \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(ctx, MSF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static void* dalloc(msf_ctx* c, size_t bytes, cudaError_t* err) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  *err = cudaMalloc(&p, bytes);
  if (*err != cudaSuccess) return nullptr;
  c->allocs.push_back(p);
  cudaMemsetAsync(p, 0, bytes, c->stream);
  return p;
}

extern "C" msf_status msf_default_options(int32_t dim, msf_options* opt) {
  if (!opt || dim < 1 || dim > 3) return MSF_EINVAL;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = MSF_FP64;
  opt->cfl = 0.6;
  opt->weno_eps = 1e-6;
  opt->mix_alpha = 0.5;
  opt->ext_sweeps = dim + 3;
  opt->vel_sweeps = 6;
  opt->reinit_iters = 6;
  opt->scale_sep = 1;
  opt->reinit = 1;
  opt->scale_eps_h = 0.0;
  opt->phi_cap_h = 8.0;
  opt->use_graph = 1;
  opt->profile = 0;
  opt->batch_mode = 0;
  opt->stream = nullptr;
  opt->rk_stages = 3;
  opt->literal_reduced = 0;
  opt->literal_normal = 0;
  opt->positivity = 0;
  return MSF_OK;
}

static int band_blocks(const Grid& g) {
  // band kernels stride over (band cell, material) items with 64-thread
  // blocks: up to 16 blocks per SM of the 152 SMs
  long long b = (g.n_interior * g.N + BAND_THREADS - 1) / BAND_THREADS;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

extern "C" msf_status msf_create(const msf_grid* grids, int32_t n_instances, int32_t n_mat, const msf_eos* eos,
                                 const msf_options* opt, msf_ctx** out) {
  if (!out) return fail(nullptr, MSF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grids || !eos || !opt) return fail(nullptr, MSF_EINVAL, "NULL argument");
  if (n_instances < 1) return fail(nullptr, MSF_EINVAL, "n_instances < 1");
  if (n_mat < 1 || n_mat > MSF_MAXMAT) return fail(nullptr, MSF_EINVAL, "n_mat outside [1, 8]");
  const int dim = grids[0].dim;
  if (dim < 1 || dim > 3) return fail(nullptr, MSF_EINVAL, "dim outside [1, 3]");
  if (opt->precision != MSF_FP64 && opt->precision != MSF_FP32_BULK) return fail(nullptr, MSF_EINVAL, "precision");
  if (!(opt->cfl > 0.0 && opt->cfl <= 1.0) || !(opt->weno_eps > 0.0) || !(opt->mix_alpha >= 0.0 && opt->mix_alpha < 1.0) ||
      opt->ext_sweeps < 1 || opt->ext_sweeps > 64 || opt->vel_sweeps < 0 || opt->vel_sweeps > 64 ||
      opt->reinit_iters < 0 || opt->reinit_iters > 64 || !(opt->phi_cap_h >= 4.0) || !(opt->scale_eps_h >= 0.0) ||
      (opt->rk_stages != 2 && opt->rk_stages != 3) || (opt->literal_reduced != 0 && opt->literal_reduced != 1) ||
      (opt->literal_normal != 0 && opt->literal_normal != 1) || (opt->positivity != 0 && opt->positivity != 1))
    return fail(nullptr, MSF_EINVAL, "option out of range");
  for (int i = 0; i < n_instances; i++) {
    const msf_grid& gr = grids[i];
    if (gr.dim != dim) return fail(nullptr, MSF_EINVAL, "instances must share dim");
    for (int d = 0; d < dim; d++) {
      if (gr.n[d] < 1 || gr.n[d] > (1 << 24)) return fail(nullptr, MSF_EINVAL, "grid size");
      if (!std::isfinite(gr.lo[d]) || !std::isfinite(gr.hi[d]) || !(gr.hi[d] > gr.lo[d]))
        return fail(nullptr, MSF_EINVAL, "domain box");
      for (int s = 0; s < 2; s++) {
        if (gr.bc[d][s] < 0 || gr.bc[d][s] > 2) return fail(nullptr, MSF_EINVAL, "bc type");
        if (gr.bc[d][s] == 2) {
          const int m = gr.inflow_mat[d][s];
          if (m < 0 || m >= n_mat) return fail(nullptr, MSF_EINVAL, "inflow material");
          const double rho = gr.inflow_prim[d][s][0], p = gr.inflow_prim[d][s][dim + 1];
          const msf_eos& em = eos[i * n_mat + m];
          const double pinf_eff = em.kind == MSF_EOS_TAIT ? em.tait_B - em.tait_p0 : em.pinf;
          if (!(rho > 0.0) || !(p + pinf_eff > 0.0)) return fail(nullptr, MSF_EINVAL, "inflow state");
        }
      }
    }
    if (gr.geom != MSF_GEOM_CARTESIAN &&
        !(gr.geom == MSF_GEOM_CYLINDRICAL && dim == 1 && gr.lo[0] >= 0.0))
      return fail(nullptr, MSF_EINVAL, "geom: cylindrical grids have one dimension and lo >= 0");
    if (gr.free_surface != 0) {
      if (gr.free_surface != 1 || gr.fs_mat < 0 || gr.fs_mat >= n_mat) return fail(nullptr, MSF_EINVAL, "fs_mat");
      const msf_eos& ef = eos[i * n_mat + gr.fs_mat];
      const double pinf_eff = ef.kind == MSF_EOS_TAIT ? ef.tait_B - ef.tait_p0 : ef.pinf;
      if (!(gr.fs_rho > 0.0) || !std::isfinite(gr.fs_rho) || !(gr.fs_t1 > gr.fs_t0) || !std::isfinite(gr.fs_t0) ||
          !std::isfinite(gr.fs_t1) || !(gr.fs_p0 + pinf_eff > 0.0) || !(gr.fs_p1 + pinf_eff > 0.0) ||
          !std::isfinite(gr.fs_p0) || !std::isfinite(gr.fs_p1))
        return fail(nullptr, MSF_EINVAL, "free-surface ambient state or drive");
    }
    long long cells = 1;
    for (int d = 0; d < dim; d++) cells *= (long long)(gr.n[d] + 2 * G);
    if (cells > (1LL << 31) - 1) return fail(nullptr, MSF_EINVAL, "grid too large");
    for (int m = 0; m < n_mat; m++) {
      const msf_eos& e = eos[i * n_mat + m];
      if (e.kind != MSF_EOS_STIFFENED && e.kind != MSF_EOS_TAIT) return fail(nullptr, MSF_EINVAL, "EOS kind");
      if (!(e.gamma > 1.0) || !std::isfinite(e.gamma)) return fail(nullptr, MSF_EINVAL, "EOS parameters");
      if (e.kind == MSF_EOS_STIFFENED && (!(e.pinf >= 0.0) || !std::isfinite(e.pinf)))
        return fail(nullptr, MSF_EINVAL, "EOS parameters");
      if (e.kind == MSF_EOS_TAIT && (!(e.tait_B > 0.0) || !(e.tait_rho0 > 0.0) || !std::isfinite(e.tait_B) ||
                                     !std::isfinite(e.tait_rho0) || !std::isfinite(e.tait_p0)))
        return fail(nullptr, MSF_EINVAL, "Tait parameters");
    }
  }

  msf_ctx* c = new msf_ctx();
  c->dim = dim;
  c->N = n_mat;
  c->ninst = n_instances;
  c->opt = *opt;
  c->stream = (cudaStream_t)opt->stream;
  c->ops = opt->precision == MSF_FP32_BULK ? ops_f32() : ops_f64();
  c->tops = opt->precision == MSF_FP32_BULK ? tiled_ops_f32() : nullptr;
  const size_t ts = c->ops->tsize;
  cudaError_t ce = cudaSuccess;
#define ALLOC(ptr, type, count)                                        \
  do {                                                                 \
    ptr = (type*)dalloc(c, sizeof(type) * (size_t)(count), &ce);       \
    if (!ptr) {                                                        \
      msf_destroy(c);                                                  \
      return fail(nullptr, MSF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(ce)); \
    }                                                                  \
  } while (0)
  ce = cudaMallocHost((void**)&c->h_ctl, sizeof(Ctl));
  if (ce != cudaSuccess) {
    delete c;
    return fail(nullptr, MSF_ENOMEM, "cudaMallocHost");
  }
  ALLOC(c->d_flag, unsigned, 4);
  if (opt->profile)
    for (int k = 0; k < 6; k++)
      if (cudaEventCreate(&c->ev[k]) != cudaSuccess) {
        msf_destroy(c);
        return fail(nullptr, MSF_ECUDA, "cudaEventCreate");
      }
  c->inst.resize(n_instances);
  for (int i = 0; i < n_instances; i++) {
    Inst& in = c->inst[i];
    Grid& g = in.g;
    std::memset(&g, 0, sizeof(g));
    const msf_grid& gr = grids[i];
    g.D = dim;
    g.N = n_mat;
    g.NV = dim + 2;
    for (int d = 0; d < 3; d++) {
      const bool act = d < dim;
      g.n[d] = act ? gr.n[d] : 1;
      g.pn[d] = act ? gr.n[d] + 2 * G : 1;
      g.off[d] = act ? G : 0;
      g.lo[d] = act ? gr.lo[d] : 0.0;
      g.h[d] = act ? (gr.hi[d] - gr.lo[d]) / (double)gr.n[d] : 1.0;
      g.rh[d] = 1.0 / g.h[d];
      g.rh2[d] = 0.5 * g.rh[d];
      g.ih2[d] = g.rh[d] * g.rh[d];
      for (int s = 0; s < 2; s++) {
        g.bc[d][s] = act ? gr.bc[d][s] : 0;
        g.inflow_mat[d][s] = gr.inflow_mat[d][s];
        for (int v = 0; v < 5; v++) g.inflow_prim[d][s][v] = gr.inflow_prim[d][s][v];
      }
    }
    g.st[0] = 1;
    g.st[1] = g.pn[0];
    g.st[2] = (long long)g.pn[0] * g.pn[1];
    g.ncell = (long long)g.pn[0] * g.pn[1] * g.pn[2];
    g.n_interior = (long long)g.n[0] * g.n[1] * g.n[2];
    g.V = 1.0;
    for (int d = 0; d < dim; d++) g.V = g.V * g.h[d];
    g.rV = 1.0 / g.V;
    for (int d = 0; d < dim; d++) g.farea[d] = g.V / g.h[d];
    g.hmin = g.h[0];
    for (int d = 1; d < dim; d++) g.hmin = std::fmin(g.hmin, g.h[d]);
    const double ce_h = opt->scale_eps_h > 0.0 ? opt->scale_eps_h : (dim == 1 ? 0.5 : (dim == 2 ? 0.75 : 0.9));
    g.eps_ss = ce_h * g.hmin;
    g.cap = opt->phi_cap_h * g.hmin;
    for (int m = 0; m < n_mat; m++) {
      const msf_eos& e = eos[i * n_mat + m];
      g.gamma[m] = e.gamma;
      g.eos_kind[m] = e.kind;
      g.tait_B[m] = e.kind == MSF_EOS_TAIT ? e.tait_B : 0.0;
      g.tait_rho0[m] = e.kind == MSF_EOS_TAIT ? e.tait_rho0 : 0.0;
      g.tait_p0[m] = e.kind == MSF_EOS_TAIT ? e.tait_p0 : 0.0;
      g.pinf[m] = e.kind == MSF_EOS_TAIT ? e.tait_B - e.tait_p0 : e.pinf;
      g.gm1[m] = g.gamma[m] - 1.0;
      g.gpi[m] = g.gamma[m] * g.pinf[m];
    }
    g.cfl = opt->cfl;
    g.weno_eps = opt->weno_eps;
    g.mix_alpha = opt->mix_alpha;
    g.ext_sweeps = opt->ext_sweeps;
    g.vel_sweeps = opt->vel_sweeps;
    g.reinit_iters = opt->reinit_iters;
    g.scale_sep = opt->scale_sep;
    g.reinit = opt->reinit;
    g.literal = (opt->literal_reduced ? 1 : 0) | (opt->literal_normal ? 2 : 0);
    g.positivity = opt->positivity;
    // Shu-Osher TVD Runge-Kutta in the beta form; the ledger weight of stage s
    // is the coefficient of dt L(Q^(s)) in Q^{n+1}
    g.rk = opt->rk_stages;
    if (g.rk == 2) {
      g.rk_beta[0] = 0.0; g.rk_beta[1] = 0.5; g.rk_beta[2] = 0.0;
      g.rk_lw[0] = 0.5; g.rk_lw[1] = 0.5; g.rk_lw[2] = 0.0;
      g.rk_c[0] = 0.0; g.rk_c[1] = 1.0; g.rk_c[2] = 1.0; g.rk_c[3] = 1.0;
    } else {
      g.rk_beta[0] = 0.0; g.rk_beta[1] = 0.75; g.rk_beta[2] = 1.0 / 3.0;
      g.rk_lw[0] = 1.0 / 6.0; g.rk_lw[1] = 1.0 / 6.0; g.rk_lw[2] = 2.0 / 3.0;
      g.rk_c[0] = 0.0; g.rk_c[1] = 1.0; g.rk_c[2] = 0.5; g.rk_c[3] = 1.0;
    }
    // axisymmetric grid and free-surface ambient (Case II)
    g.geom = gr.geom;
    g.fs_mat = gr.free_surface ? gr.fs_mat : -1;
    g.fs_rho = gr.fs_rho;
    g.fs_p0 = gr.fs_p0;
    g.fs_t0 = gr.fs_t0;
    g.fs_t1 = gr.fs_t1;
    g.fs_p1 = gr.fs_p1;
    // boundary faces, numbered per (axis, side)
    long long nb = 0;
    for (int d = 0; d < dim; d++)
      for (int s = 0; s < 2; s++) {
        in.bb.base[2 * d + s] = nb;
        nb += g.n_interior / g.n[d];
      }
    in.nbnd = (int)nb;
    in.nblk_band = band_blocks(g);
  }
#undef ALLOC
  // all arrays of all instances carved from one allocation (two passes: size, then assign)
  const bool batched = n_instances > 1 && dim == 1 && opt->batch_mode == 0;
  c->batched = batched;
  size_t total = 0;
  for (int pass = 0; pass < 2; pass++) {
    char* base = pass == 0 ? nullptr : (char*)c->arena;
    size_t off = 0;
    auto carve = [&](size_t bytes) -> void* {
      off = (off + 255) & ~(size_t)255;
      void* p = base ? (void*)(base + off) : nullptr;
      off += bytes ? bytes : 16;
      return p;
    };
    for (int i = 0; i < n_instances; i++) {
      Inst& in = c->inst[i];
      const Grid& g = in.g;
      const long long nc = g.ncell, N = n_mat, NV = g.NV, nbmax = g.n_interior;
      Bufs& b = in.b;
      for (int k = 0; k < 3; k++) b.Q[k] = (double*)carve(8 * N * NV * nc);
      // FP32 copies of the stage states (FP32-bulk grid contexts; the
      // batched kernel stages its states itself)
      for (int k = 0; k < 3; k++) b.Qf[k] = ts == 4 && !batched ? (float*)carve(4 * N * NV * nc) : nullptr;
      b.phi = (double*)carve(8 * nc);
      b.phin = (double*)carve(8 * nc);
      b.chi = (uint8_t*)carve(nc);
      b.chin = (uint8_t*)carve(nc);
      b.xs = (uint8_t*)carve(nc);
      b.mtmp = (uint8_t*)carve(nc);
      b.smask = (uint8_t*)carve(nc);
      b.xsS = (uint8_t*)carve(nc);
      b.gflag = (uint8_t*)carve(nc);
      b.nrm = (double*)carve(8 * N * 3 * nc);
      b.alpha = (double*)carve(8 * N * nc);
      b.Alo = (double*)carve(8 * dim * N * nc);
      b.Ahi = (double*)carve(8 * dim * N * nc);
      b.W0 = carve(ts * N * NV * nc);
      b.W1 = carve(ts * N * NV * nc);
      b.Uh = carve(ts * N * NV * nc);
      b.f0 = (uint8_t*)carve(N * nc);
      b.f1 = (uint8_t*)carve(N * nc);
      b.isreal = (uint8_t*)carve(N * nc);
      b.X = (double*)carve(8 * N * NV * nc);
      b.vel0 = (double*)carve(8 * 3 * nc);
      b.vel1 = (double*)carve(8 * 3 * nc);
      b.vf0 = (uint8_t*)carve(nc);
      b.vf1 = (uint8_t*)carve(nc);
      b.band = (int*)carve(4 * nbmax);
      b.bandidx = (int*)carve(4 * nc);
      b.phit = (double*)carve(8 * nbmax);
      b.chit = (uint8_t*)carve(nbmax);
      b.mixq = (double*)carve(8 * nbmax * N * NV);
      b.mixmerge = (unsigned*)carve(4 * nbmax);
      b.mixn = (uint8_t*)carve(nbmax * N);
      b.mixoff = (uint8_t*)carve(nbmax * N * MIX_MAXT);
      b.mixbeta = (double*)carve(8 * nbmax * N * MIX_MAXT);
      b.mixin = (unsigned*)carve(4 * nbmax * N);
      b.mixT = (double*)carve(8 * nbmax * N);
      b.mixlist = (int*)carve(4 * nbmax * N);
      b.geomlist = (int*)carve(4 * nbmax * N);
      b.lslist = (int*)carve(4 * nbmax * N);
      b.mixtouch = (uint8_t*)carve(nbmax);
      b.phir = (double*)carve(8 * nbmax * N);
      b.bflux = (double*)carve(8 * std::max<long long>(1, in.nbnd) * N * NV);
      b.lpart = (double*)carve(8 * ((std::max<long long>(1, in.nbnd) + NTHREADS - 1) / NTHREADS) * N * NV);
      b.ctl = (Ctl*)carve(sizeof(Ctl));
      if (batched) {
        in.Fface = carve(ts * N * NV * (g.n[0] + 1));
        in.Aface = (double*)carve(8 * N * (g.n[0] + 1));
      }
    }
    if (pass == 0) {
      total = off;
      ce = cudaMalloc(&c->arena, total);
      if (ce != cudaSuccess) {
        msf_destroy(c);
        return fail(nullptr, MSF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(ce));
      }
      cudaMemsetAsync(c->arena, 0, total, c->stream);
    }
  }
  for (Inst& in : c->inst) cudaMemsetAsync(in.b.bandidx, 0xff, sizeof(int) * in.g.ncell, c->stream);
  if (batched) {
    // instance table and largest-first order for the persistent kernel
    std::vector<BatchEntry> tab(n_instances);
    std::vector<int> order(n_instances);
    for (int i = 0; i < n_instances; i++) {
      Inst& in = c->inst[i];
      tab[i].g = in.g;
      tab[i].b = in.b;
      tab[i].bb = in.bb;
      tab[i].Fface = in.Fface;
      tab[i].Aface = in.Aface;
      tab[i].nbnd = in.nbnd;
      order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int bb) { return c->inst[a].g.n_interior > c->inst[bb].g.n_interior; });
    ce = cudaMalloc((void**)&c->d_tab, sizeof(BatchEntry) * n_instances);
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&c->d_order, sizeof(int) * n_instances);
    if (ce == cudaSuccess) {
      c->allocs.push_back(c->d_tab);
      c->allocs.push_back(c->d_order);
      ce = cudaMemcpy(c->d_tab, tab.data(), sizeof(BatchEntry) * n_instances, cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess) ce = cudaMemcpy(c->d_order, order.data(), sizeof(int) * n_instances, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaEventCreate(&c->tev[0]);
    if (ce == cudaSuccess) ce = cudaEventCreate(&c->tev[1]);
    if (ce != cudaSuccess) {
      msf_destroy(c);
      return fail(nullptr, MSF_ECUDA, std::string("batch table: ") + cudaGetErrorString(ce));
    }
  }
  ce = cudaStreamSynchronize(c->stream);
  if (ce != cudaSuccess) {
    msf_destroy(c);
    return fail(nullptr, MSF_ECUDA, std::string("create: ") + cudaGetErrorString(ce));
  }
  *out = c;
  return MSF_OK;
}

extern "C" msf_status msf_destroy(msf_ctx* c) {
  if (!c) return MSF_OK;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (int k = 0; k < 2; k++)
    if (c->tev[k]) cudaEventDestroy(c->tev[k]);
  if (c->arena) cudaFree(c->arena);
  for (int k = 0; k < 6; k++)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  for (void* p : c->allocs) cudaFree(p);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  delete c;
  return MSF_OK;
}

// ---------------------------------------------------------------- stepping
// the FP32-bulk form runs the ghost-state sweeps of two-dimensional grids
// tiled (one launch for K sweeps)
static bool tiled_ext(const msf_ctx* c, const Grid& g) {
  return c->tops && g.D == 2 && g.ext_sweeps >= 1 && g.ext_sweeps <= TILED_MAX_SWEEPS;
}
static bool tiled_vel(const msf_ctx* c, const Grid& g) {
  return c->tops && g.D == 2 && g.vel_sweeps >= 1 && g.vel_sweeps <= TILED_MAX_SWEEPS;
}

// kernels one step enqueues (keep in step with enqueue_step)
static long long count_launches(const msf_ctx* c) {
  long long n = 0;
  for (const Inst& in : c->inst) {
    const Grid& g = in.g;
    const long long ext = tiled_ext(c, g) ? 1 : g.ext_sweeps;
    const long long vel = tiled_vel(c, g) ? 1 : g.vel_sweeps, re = 2LL * g.reinit_iters;
    // prim, ext, cons, bc_uhat, interface, vel, flux, ledger (2), level set (2),
    // bc_phichi, geometry (2), mixing (4)
    const long long per_stage = 1 + ext + 1 + 1 + 1 + vel + 1 + 2 + 2 + 1 + 2 + 4;
    n += 1 + 1 + (2 + g.D) + 2 + 1 + g.rk * per_stage + 2 + 1;
    if (g.D == 3) n += 1 + g.rk;  // the cut-item pass of every geometry launch
    if (in.b.Qf[0]) n += 1;
    if (g.fs_mat >= 0) n += 1 + g.rk;
    if (g.scale_sep) n += 2 + 1;
    if (g.reinit) n += re + 1;
  }
  return n;
}

// replay tape of one step (device memory, caller-owned): header (t, dt of the
// step), Q^n, and phi / chi after the boundary fill at the start of each
// stage and after the level-set stage of the last stage
struct TapeLayout {
  size_t q, phi, chi, total;
};
static TapeLayout tape_layout(const Grid& g) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t nc = (size_t)g.ncell;
  TapeLayout L;
  size_t off = 256;
  L.q = off;
  off = up(off + sizeof(double) * g.N * g.NV * nc);
  L.phi = off;
  off = up(off + sizeof(double) * 4 * nc);
  L.chi = off;
  off = up(off + 4 * nc);
  L.total = off;
  return L;
}
static void tape_slot_save(const Inst& in, char* tape, int slot, cudaStream_t s) {
  const TapeLayout L = tape_layout(in.g);
  const size_t nc = (size_t)in.g.ncell;
  cudaMemcpyAsync(tape + L.phi + sizeof(double) * nc * slot, in.b.phi, sizeof(double) * nc, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(tape + L.chi + nc * slot, in.b.chi, nc, cudaMemcpyDeviceToDevice, s);
}
static void tape_slot_load(const Inst& in, const char* tape, int slot, cudaStream_t s) {
  const TapeLayout L = tape_layout(in.g);
  const size_t nc = (size_t)in.g.ncell;
  cudaMemcpyAsync(in.b.phi, tape + L.phi + sizeof(double) * nc * slot, sizeof(double) * nc, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(in.b.chi, tape + L.chi + nc * slot, nc, cudaMemcpyDeviceToDevice, s);
}

static msf_status enqueue_step(msf_ctx* c, char* tape = nullptr) {
  const cudaStream_t s = c->stream;
  for (Inst& in : c->inst) {
    const Grid& g = in.g;
    const Bufs& b = in.b;
    const int nb = in.nblk_band;
    launch_step_begin(b, s);
    launch_bc_phichi(g, b, s);
    if (tape) {
      cudaMemcpyAsync(tape, &b.ctl->t, sizeof(double), cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(tape + tape_layout(g).q, b.Q[0], sizeof(double) * g.N * g.NV * g.ncell,
                      cudaMemcpyDeviceToDevice, s);
      tape_slot_save(in, tape, 0, s);
    }
    launch_masks(g, b, s);
    launch_geometry(g, b, b.Q[0], nullptr, nb, s);
    if (g.fs_mat >= 0) launch_hold_ambient(g, b, b.Q[0], -1, s);
    launch_band_save(g, b, nb, s);
    for (int st = 0; st < g.rk; st++) {
      const double beta = g.rk_beta[st];
      double* Qs = b.Q[st];
      double* Qo = st == g.rk - 1 ? b.Q[0] : b.Q[st + 1];
      c->ops->prim(g, b, Qs, nb, s);
      void* W[2] = {b.W0, b.W1};
      uint8_t* F[2] = {b.f0, b.f1};
      int cur = 0;
      if (tiled_ext(c, g)) {
        cudaError_t te = c->tops->extend(g, b, W[0], W[1], F[0], F[1], g.ext_sweeps, s);
        if (te != cudaSuccess) return fail(c, MSF_ECUDA, std::string("tiled extension: ") + cudaGetErrorString(te));
        cur = 1;
      } else {
        for (int k = 0; k < g.ext_sweeps; k++) {
          c->ops->extend(g, b, W[cur], W[cur ^ 1], F[cur], F[cur ^ 1], nb, s);
          cur ^= 1;
        }
      }
      c->ops->cons(g, b, Qs, W[cur], F[cur], nb, s);
      c->ops->bc_uhat(g, b, Qs, s);
      // the exchange of stage 0 comes first: the bound of the step reads the
      // free-surface velocities it sets
      c->ops->interface(g, b, Qs, st, nb, s);
      if (st == 0) {
        c->ops->dt(g, b, Qs, s);
        launch_dt_finalize(g, b, s);
        if (tape) cudaMemcpyAsync(tape + sizeof(double), &b.ctl->dt, sizeof(double), cudaMemcpyDeviceToDevice, s);
      }
      double* V[2] = {b.vel0, b.vel1};
      uint8_t* VF[2] = {b.vf0, b.vf1};
      int vc = 0;
      if (tiled_vel(c, g)) {
        cudaError_t te = c->tops->extend_vel(g, b, V[0], V[1], VF[0], VF[1], g.vel_sweeps, s);
        if (te != cudaSuccess) return fail(c, MSF_ECUDA, std::string("tiled velocity: ") + cudaGetErrorString(te));
        vc = 1;
      } else {
        for (int k = 0; k < g.vel_sweeps; k++) {
          launch_extend_vel(g, b, V[vc], V[vc ^ 1], VF[vc], VF[vc ^ 1], nb, s);
          vc ^= 1;
        }
      }
      const bool prof = c->ev[0] && &in == &c->inst[0];
      if (prof) cudaEventRecord(c->ev[2 * st], s);
      // FP32-bulk form: every stage stages its bulk states from the FP32 copy
      // of its state (Q^n rounded at the end of the step before, Q^(s) written
      // by the update of the stage before) and writes the copy of its output
      const float* Qsf = b.Qf[st];
      float* Qof = b.Qf[(st + 1) % g.rk];
      cudaError_t fe = c->ops->flux(g, b, Qs, b.Q[0], Qo, beta, 1.0 - beta, in.bb, Qsf, Qof, s);
      if (fe != cudaSuccess) return fail(c, MSF_ECUDA, std::string("flux launch: ") + cudaGetErrorString(fe));
      if (prof) cudaEventRecord(c->ev[2 * st + 1], s);
      launch_ledger(g, b, in.nbnd, g.rk_lw[st], s);
      launch_levelset(g, b, V[vc], beta, 1.0 - beta, nb, s);
      launch_bc_phichi(g, b, s);
      if (tape) tape_slot_save(in, tape, st + 1, s);
      launch_geometry(g, b, Qo, nullptr, nb, s);
      if (g.fs_mat >= 0) launch_hold_ambient(g, b, Qo, st + 1, s);
      launch_mix(g, b, Qo, nb, s);
    }
    launch_step_end(b, s);
    if (g.scale_sep) {
      launch_scale_sep(g, b, nb, s);
      launch_bc_phichi(g, b, s);
    }
    if (g.reinit) {
      for (int k = 0; k < g.reinit_iters; k++) launch_reinit(g, b, nb, s);
      launch_bc_phichi(g, b, s);
    }
    // the band cells' states changed after the last update wrote their FP32 copy
    c->ops->qf_copy(g, b, 1, nb, s);
  }
  // kernels enqueued above (keep in step with the sequence)
  c->launches = count_launches(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, MSF_ECUDA, std::string("step launch: ") + cudaGetErrorString(e));
  return MSF_OK;
}

__global__ void k_set_tend(Ctl* ctl, double t_end) { ctl->t_end = t_end; }

static msf_status read_error(msf_ctx* c) {
  unsigned bits = 0;
  for (Inst& in : c->inst) {
    cudaError_t e = cudaMemcpyAsync(c->h_ctl, in.b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, MSF_ECUDA, std::string("step: ") + cudaGetErrorString(e));
    bits |= c->h_ctl->err;
  }
  if (!bits) return MSF_OK;
  c->sticky = true;
  if (bits & ERR_BAND) return fail(c, MSF_EBAND, "a flux stencil reached a cell without a state of that material");
  if (bits & ERR_NEGATIVE) return fail(c, MSF_ENEGATIVE, "non-positive density or p + pinf in a used state");
  return fail(c, MSF_ENONFINITE, "non-finite conserved value");
}

extern "C" msf_status msf_step(msf_ctx* c, int32_t n_steps, double t_end, int32_t sync) {
  if (!c) return MSF_EINVAL;
  if (c->sticky) return fail(c, MSF_ESTATE, "context holds a device-detected error; reset with msf_set_state");
  if (n_steps < 0 || std::isnan(t_end)) return fail(c, MSF_EINVAL, "n_steps < 0 or t_end NaN");
  if (n_steps == 0) return MSF_OK;
  if (c->batched) {
    launch_set_tend_all(c->d_tab, c->ninst, t_end, c->stream);
    int left = n_steps;
    if (c->bs == 0) {
      // autotune the CTA size on live steps (results do not depend on it)
      const int cand[3] = {128, 256, 512};
      float best = 0.0f;
      int bestbs = 256;
      for (int k = 0; k < 3 && left > 0; k++, left--) {
        CUDA_TRY(c, cudaEventRecord(c->tev[0], c->stream));
        CUDA_TRY(c, c->ops->batched(c->d_tab, c->d_order, c->ninst, 1, cand[k], c->stream));
        CUDA_TRY(c, cudaEventRecord(c->tev[1], c->stream));
        CUDA_TRY(c, cudaEventSynchronize(c->tev[1]));
        float ms = 0.0f;
        CUDA_TRY(c, cudaEventElapsedTime(&ms, c->tev[0], c->tev[1]));
        if (k == 0 || ms < best) {
          best = ms;
          bestbs = cand[k];
        }
      }
      c->bs = bestbs;
    }
    if (left > 0) CUDA_TRY(c, c->ops->batched(c->d_tab, c->d_order, c->ninst, left, c->bs, c->stream));
    c->launches = 2;
    if (sync) return read_error(c);
    return MSF_OK;
  }
  for (Inst& in : c->inst) k_set_tend<<<1, 1, 0, c->stream>>>(in.b.ctl, t_end);
  bool use_graph = c->opt.use_graph != 0 && c->ninst == 1;
  if (use_graph && !c->graph && !c->graph_tried) {
    c->graph_tried = true;
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      msf_status st = enqueue_step(c);
      cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
      if (st == MSF_OK && e == cudaSuccess) {
        size_t nn = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess) {
          std::vector<cudaGraphNode_t> nodes(nn);
          if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess) {
            long long nk = 0;
            for (size_t k = 0; k < nn; k++) {
              cudaGraphNodeType ty;
              if (cudaGraphNodeGetType(nodes[k], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) nk++;
            }
            c->graph_kernels = nk;
          }
        }
        if (cudaGraphInstantiate(&c->graph, graph, 0) != cudaSuccess) c->graph = nullptr;
        cudaGraphDestroy(graph);
      }
    }
    cudaGetLastError();
  }
  for (int k = 0; k < n_steps; k++) {
    if (use_graph && c->graph) {
      CUDA_TRY(c, cudaGraphLaunch(c->graph, c->stream));
    } else {
      msf_status st = enqueue_step(c);
      if (st != MSF_OK) return st;
    }
  }
  if (sync) return read_error(c);
  return MSF_OK;
}

// ------------------------------------------------------------ data movement
static msf_status check_instance(msf_ctx* c, int32_t i) {
  if (!c) return MSF_EINVAL;
  if (i < 0 || i >= c->ninst) return fail(c, MSF_EINVAL, "instance out of range");
  return MSF_OK;
}

// device staging copy of a caller array (host or device)
static msf_status stage_in(msf_ctx* c, const void* src, size_t bytes, int32_t mem, void** dst) {
  cudaError_t e = cudaMalloc(dst, bytes ? bytes : 16);
  if (e != cudaSuccess) return fail(c, MSF_ENOMEM, "staging allocation");
  e = cudaMemcpyAsync(*dst, src, bytes, mem == MSF_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      c->stream);
  if (e != cudaSuccess) {
    cudaFree(*dst);
    return fail(c, MSF_ECUDA, "staging copy");
  }
  return MSF_OK;
}

// control-block setters that leave the ledger and the counters alone
__global__ void k_ctl_activate(Ctl* ctl) {
  ctl->active = 1;
  ctl->nband = 0;
}
__global__ void k_ctl_restart(Ctl* ctl, double t) {
  ctl->t = t;
  ctl->dt = 0.0;
  ctl->err = 0;
  ctl->active = 0;
  ctl->last = 0;
}

static msf_status finish_geometry(msf_ctx* c, Inst& in) {
  // boundary fill and narrow band of the current (phi, chi)
  const cudaStream_t s = c->stream;
  k_ctl_activate<<<1, 1, 0, s>>>(in.b.ctl);
  launch_bc_phichi(in.g, in.b, s);
  launch_masks(in.g, in.b, s);
  return MSF_OK;
}

extern "C" msf_status msf_set_levelset(msf_ctx* c, int32_t i, const double* phi, const int32_t* chi,
                                       const double* prim, int32_t mem) {
  msf_status st = check_instance(c, i);
  if (st != MSF_OK) return st;
  if (!phi || !chi || !prim) return fail(c, MSF_EINVAL, "NULL array");
  if (mem != MSF_HOST && mem != MSF_DEVICE) return fail(c, MSF_EINVAL, "mem");
  Inst& in = c->inst[i];
  const Grid& g = in.g;
  const long long ni = g.n_interior;
  const int N = g.N, NV = g.NV;
  if (mem == MSF_HOST) {
    for (long long k = 0; k < ni; k++) {
      if (!(phi[k] >= 0.0) || !std::isfinite(phi[k])) return fail(c, MSF_EINVAL, "phi must be finite and >= 0");
      if (chi[k] < 0 || chi[k] >= N) return fail(c, MSF_EINVAL, "chi out of range");
    }
    for (int m = 0; m < N; m++)
      for (long long k = 0; k < ni; k++) {
        for (int v = 0; v < NV; v++)
          if (!std::isfinite(prim[((long long)m * NV + v) * ni + k])) return fail(c, MSF_EINVAL, "non-finite prim");
        if (!(prim[((long long)m * NV) * ni + k] > 0.0)) return fail(c, MSF_EINVAL, "rho <= 0 in prim");
        if (!(prim[((long long)m * NV + NV - 1) * ni + k] + g.pinf[m] > 0.0))
          return fail(c, MSF_EINVAL, "p + pinf <= 0 in prim");
      }
  }
  void *dphi = nullptr, *dchi = nullptr, *dprim = nullptr;
  if ((st = stage_in(c, phi, sizeof(double) * ni, mem, &dphi)) != MSF_OK) return st;
  if ((st = stage_in(c, chi, sizeof(int32_t) * ni, mem, &dchi)) != MSF_OK) return st;
  if ((st = stage_in(c, prim, sizeof(double) * ni * N * NV, mem, &dprim)) != MSF_OK) return st;
  const cudaStream_t s = c->stream;
  if (mem == MSF_DEVICE) {
    unsigned flag = 0;
    cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned), s);
    launch_check_inputs(g, (const double*)dphi, (const int32_t*)dchi, (const double*)dprim, c->d_flag, s);
    cudaMemcpyAsync(&flag, c->d_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (flag) {
      cudaFree(dphi); cudaFree(dchi); cudaFree(dprim);
      return fail(c, MSF_EINVAL, "invalid device inputs (phi < 0, chi out of range or bad prim)");
    }
  }
  Bufs& b = in.b;
  for (int k = 0; k < 3; k++) cudaMemsetAsync(b.Q[k], 0, sizeof(double) * N * NV * g.ncell, s);
  launch_init_levelset(g, b, (const double*)dphi, (const int32_t*)dchi, s);
  if ((st = finish_geometry(c, in)) != MSF_OK) return st;
  // raw volume fractions, masses alpha rho, then the corrected fractions
  launch_geometry(g, b, nullptr, nullptr, in.nblk_band, s);
  launch_init_mass(g, b, (const double*)dprim, b.Q[1], s);
  launch_geometry(g, b, nullptr, b.Q[1], in.nblk_band, s);
  cudaMemsetAsync(b.Q[1], 0, sizeof(double) * N * NV * g.ncell, s);
  launch_init_state(g, b, (const double*)dprim, s);
  if (g.fs_mat >= 0) launch_hold_ambient(g, b, b.Q[0], -2, s);
  c->ops->qf_copy(g, b, 0, 0, s);
  Ctl h{};
  h.t_end = INFINITY;
  CUDA_TRY(c, cudaMemcpyAsync(b.ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(dphi);
  cudaFree(dchi);
  cudaFree(dprim);
  if (e != cudaSuccess) return fail(c, MSF_ECUDA, std::string("set_levelset: ") + cudaGetErrorString(e));
  c->sticky = false;
  return MSF_OK;
}

static msf_status gather_out(msf_ctx* c, Inst& in, int which, void* dst, size_t bytes, int32_t mem, bool integer) {
  void* tmp = nullptr;
  if (cudaMalloc(&tmp, bytes ? bytes : 16) != cudaSuccess) return fail(c, MSF_ENOMEM, "staging allocation");
  launch_gather(in.g, in.b, which, integer ? nullptr : (double*)tmp, integer ? (int32_t*)tmp : nullptr, c->stream);
  cudaError_t e = cudaMemcpyAsync(dst, tmp, bytes, mem == MSF_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(c, MSF_ECUDA, std::string("gather: ") + cudaGetErrorString(e));
  return MSF_OK;
}

extern "C" msf_status msf_get_state(msf_ctx* c, int32_t i, double* Q, double* alpha, double* phi, int32_t* chi,
                                    double* t, int32_t mem) {
  msf_status st = check_instance(c, i);
  if (st != MSF_OK) return st;
  Inst& in = c->inst[i];
  const long long ni = in.g.n_interior;
  if (Q && (st = gather_out(c, in, 0, Q, sizeof(double) * ni * in.g.N * in.g.NV, mem, false)) != MSF_OK) return st;
  if (alpha && (st = gather_out(c, in, 1, alpha, sizeof(double) * ni * in.g.N, mem, false)) != MSF_OK) return st;
  if (phi && (st = gather_out(c, in, 2, phi, sizeof(double) * ni, mem, false)) != MSF_OK) return st;
  if (chi && (st = gather_out(c, in, 3, chi, sizeof(int32_t) * ni, mem, true)) != MSF_OK) return st;
  if (t) {
    CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, in.b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *t = c->h_ctl->t;
  }
  return MSF_OK;
}

extern "C" msf_status msf_set_state(msf_ctx* c, int32_t i, const double* Q, const double* phi, const int32_t* chi,
                                    double t, int32_t mem) {
  msf_status st = check_instance(c, i);
  if (st != MSF_OK) return st;
  if (!Q || !phi || !chi || !std::isfinite(t)) return fail(c, MSF_EINVAL, "NULL array or non-finite t");
  Inst& in = c->inst[i];
  const Grid& g = in.g;
  const long long ni = g.n_interior;
  if (mem == MSF_HOST)
    for (long long k = 0; k < ni; k++) {
      if (!(phi[k] >= 0.0) || !std::isfinite(phi[k])) return fail(c, MSF_EINVAL, "phi must be finite and >= 0");
      if (chi[k] < 0 || chi[k] >= g.N) return fail(c, MSF_EINVAL, "chi out of range");
    }
  void *dQ = nullptr, *dphi = nullptr, *dchi = nullptr;
  if ((st = stage_in(c, Q, sizeof(double) * ni * g.N * g.NV, mem, &dQ)) != MSF_OK) return st;
  if ((st = stage_in(c, phi, sizeof(double) * ni, mem, &dphi)) != MSF_OK) return st;
  if ((st = stage_in(c, chi, sizeof(int32_t) * ni, mem, &dchi)) != MSF_OK) return st;
  const cudaStream_t s = c->stream;
  launch_scatter_state(g, in.b, (const double*)dQ, (const double*)dphi, (const int32_t*)dchi, s);
  if ((st = finish_geometry(c, in)) != MSF_OK) return st;
  launch_geometry(g, in.b, in.b.Q[0], nullptr, in.nblk_band, s);
  c->ops->qf_copy(g, in.b, 0, 0, s);
  // keep the ledger and counters, set t, clear the error
  k_ctl_restart<<<1, 1, 0, s>>>(in.b.ctl, t);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(dQ);
  cudaFree(dphi);
  cudaFree(dchi);
  if (e != cudaSuccess) return fail(c, MSF_ECUDA, std::string("set_state: ") + cudaGetErrorString(e));
  c->sticky = false;
  return MSF_OK;
}

extern "C" msf_status msf_totals(msf_ctx* c, int32_t i, double* totals, double* ledger) {
  msf_status st = check_instance(c, i);
  if (st != MSF_OK) return st;
  Inst& in = c->inst[i];
  const int NMV = in.g.N * in.g.NV;
  double* tmp = nullptr;
  if (cudaMalloc(&tmp, sizeof(double) * NMV) != cudaSuccess) return fail(c, MSF_ENOMEM, "totals staging");
  launch_totals(in.g, in.b.Q[0], tmp, c->stream);
  std::vector<double> h(NMV);
  cudaError_t e = cudaMemcpyAsync(h.data(), tmp, sizeof(double) * NMV, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_ctl, in.b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(c, MSF_ECUDA, std::string("totals: ") + cudaGetErrorString(e));
  for (int m = 0; m < in.g.N; m++)
    for (int v = 0; v < in.g.NV; v++) {
      if (totals) totals[m * in.g.NV + v] = h[m * in.g.NV + v];
      if (ledger) ledger[m * in.g.NV + v] = c->h_ctl->ledger[m][v];
    }
  return MSF_OK;
}

extern "C" msf_status msf_stats(msf_ctx* c, int64_t* counters) {
  if (!c || !counters) return MSF_EINVAL;
  for (int k = 0; k < MSF_NSTATS; k++) counters[k] = 0;
  for (Inst& in : c->inst) {
    CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, in.b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < MSF_NSTATS; k++) counters[k] += (int64_t)c->h_ctl->cnt[k];
  }
  return MSF_OK;
}

extern "C" msf_status msf_last_dt(msf_ctx* c, int32_t i, double* dt) {
  msf_status st = check_instance(c, i);
  if (st != MSF_OK) return st;
  if (!dt) return fail(c, MSF_EINVAL, "dt is NULL");
  CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, c->inst[i].b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *dt = c->h_ctl->dt;
  return MSF_OK;
}

extern "C" msf_status msf_debug_field(msf_ctx* c, int32_t i, int32_t which, double* out) {
  msf_status st = check_instance(c, i);
  if (st != MSF_OK) return st;
  if (!out) return fail(c, MSF_EINVAL, "out is NULL");
  Inst& in = c->inst[i];
  const long long ni = in.g.n_interior;
  const int N = in.g.N, NV = in.g.NV;
  switch (which) {
    case 0: return gather_out(c, in, 1, out, sizeof(double) * ni * N, MSF_HOST, false);
    case 1: return gather_out(c, in, c->ops->tsize == 8 ? 20 : 21, out, sizeof(double) * ni * N * NV, MSF_HOST, false);
    case 2: return gather_out(c, in, 11, out, sizeof(double) * ni * N * NV, MSF_HOST, false);
    case 3: {
      const int which_vel = (in.g.vel_sweeps % 2 == 0) ? 30 : 31;
      return gather_out(c, in, which_vel, out, sizeof(double) * ni * 3, MSF_HOST, false);
    }
    case 4: return gather_out(c, in, 13, out, sizeof(double) * ni, MSF_HOST, false);
    case 5: return gather_out(c, in, 14, out, sizeof(double) * ni, MSF_HOST, false);
    default: return fail(c, MSF_EINVAL, "which");
  }
}

extern "C" msf_status msf_launches_per_step(msf_ctx* c, int64_t* n) {
  if (!c || !n) return MSF_EINVAL;
  // batched: one persistent launch (plus the end-time kernel) covers every step of a call
  *n = c->batched ? 1 : count_launches(c);
  // the captured step graph holds the kernels one step actually enqueues
  if (!c->batched && c->graph && c->graph_kernels >= 0 && c->graph_kernels != *n)
    return fail(c, MSF_ESTATE, "kernel count of one step out of step with the captured graph");
  return MSF_OK;
}

extern "C" msf_status msf_instance_info(msf_ctx* c, int32_t i, double* t, int64_t* steps, int32_t* status) {
  msf_status st = check_instance(c, i);
  if (st != MSF_OK) return st;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, c->inst[i].b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const Ctl& h = *c->h_ctl;
  if (t) *t = h.t;
  if (steps) *steps = (int64_t)h.cnt[C_STEPS];
  if (status)
    *status = (h.err & ERR_BAND) ? MSF_EBAND
              : (h.err & ERR_NEGATIVE) ? MSF_ENEGATIVE
              : (h.err & ERR_NONFINITE) ? MSF_ENONFINITE : MSF_OK;
  return MSF_OK;
}

extern "C" msf_status msf_batch_block_size(msf_ctx* c, int32_t* block_size) {
  if (!c || !block_size) return MSF_EINVAL;
  *block_size = c->batched ? c->bs : 0;
  return MSF_OK;
}

extern "C" msf_status msf_profile_read(msf_ctx* c, double* flux_ms) {
  if (!c || !flux_ms) return MSF_EINVAL;
  if (!c->ev[0]) return fail(c, MSF_EINVAL, "profiling is off (msf_options.profile = 0)");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int st = 0; st < 3; st++) {
    float ms = 0.0f;
    if (st < c->inst[0].g.rk) CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev[2 * st], c->ev[2 * st + 1]));
    flux_ms[st] = ms;
  }
  return MSF_OK;
}

// ------------------------------------------------ tapes, replay, adjoint
static msf_status check_single(msf_ctx* c) {
  if (!c) return MSF_EINVAL;
  if (c->ninst != 1 || c->batched) return fail(c, MSF_EUNSUPPORTED, "tapes and the adjoint need a single-instance context");
  if (c->inst[0].g.geom != 0 || c->inst[0].g.fs_mat >= 0)
    return fail(c, MSF_EUNSUPPORTED, "tapes and the adjoint take Cartesian grids without a free surface");
  if (c->inst[0].g.literal != 0 || c->inst[0].g.positivity != 0)
    return fail(c, MSF_EUNSUPPORTED, "tapes and the adjoint take the default scheme (literal options and positivity off)");
  if (c->sticky) return fail(c, MSF_ESTATE, "context holds a device-detected error; reset with msf_set_state");
  return MSF_OK;
}

static msf_status ensure_adjoint(msf_ctx* c) {
  if (c->adj_ready) return MSF_OK;
  Inst& in = c->inst[0];
  const Grid& g = in.g;
  const size_t nc = (size_t)g.ncell, N = g.N, NV = g.NV, nbmax = (size_t)g.n_interior;
  cudaError_t ce = cudaSuccess;
  AdjBufs& a = c->adj;
  auto take = [&](size_t bytes) -> void* {
    void* p = dalloc(c, bytes, &ce);
    return p;
  };
  a.LA = (double*)take(8 * N * NV * nc);
  a.LN = (double*)take(8 * N * NV * nc);
  a.LU = (double*)take(8 * N * NV * nc);
  a.LQ = (double*)take(8 * N * NV * nc);
  a.LW0 = (double*)take(8 * N * NV * nc);
  a.LW1 = (double*)take(8 * N * NV * nc);
  a.lvl = (uint8_t*)take(N * nc);
  a.mixt = (double*)take(8 * nbmax * N * NV);
  for (int k = 0; k < 3; k++) {
    a.mixn[k] = (uint8_t*)take(nbmax * N);
    a.mixoff[k] = (uint8_t*)take(nbmax * N * MIX_MAXT);
    a.mixbeta[k] = (double*)take(8 * nbmax * N * MIX_MAXT);
    a.mixT[k] = (double*)take(8 * nbmax * N);
  }
  for (int k = 0; k < 4; k++) a.aband[k] = (double*)take(8 * nbmax * N);
  a.deos = (double*)take(8 * MAXM * 2);
  a.dinf = (double*)take(8 * 3 * 2 * 5);
  if (ce != cudaSuccess) return fail(c, MSF_ENOMEM, std::string("adjoint workspace: ") + cudaGetErrorString(ce));
  if (!c->h_pin && cudaMallocHost((void**)&c->h_pin, sizeof(double) * 64) != cudaSuccess)
    return fail(c, MSF_ENOMEM, "cudaMallocHost");
  c->aops = c->ops->tsize == 8 ? adj_ops_f64() : adj_ops_f32();
  c->adj_ready = true;
  return MSF_OK;
}

static bool tape_aligned(const void* p) { return ((uintptr_t)p & 255u) == 0; }

extern "C" msf_status msf_tape_bytes(const msf_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return MSF_EINVAL;
  if (c->ninst != 1 || c->batched) return MSF_EUNSUPPORTED;
  if (c->inst[0].g.geom != 0 || c->inst[0].g.fs_mat >= 0 || c->inst[0].g.literal != 0 || c->inst[0].g.positivity != 0)
    return MSF_EUNSUPPORTED;
  *bytes = (int64_t)tape_layout(c->inst[0].g).total;
  return MSF_OK;
}

extern "C" msf_status msf_step_taped(msf_ctx* c, void* tape, double t_end) {
  msf_status st = check_single(c);
  if (st != MSF_OK) return st;
  if (!tape || !tape_aligned(tape)) return fail(c, MSF_EINVAL, "tape must be a 256-byte aligned device buffer");
  if (std::isnan(t_end)) return fail(c, MSF_EINVAL, "t_end NaN");
  Inst& in = c->inst[0];
  CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, in.b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (!(c->h_ctl->t < t_end)) return fail(c, MSF_EINVAL, "no step to take: t >= t_end");
  k_set_tend<<<1, 1, 0, c->stream>>>(in.b.ctl, t_end);
  if ((st = enqueue_step(c, (char*)tape)) != MSF_OK) return st;
  return read_error(c);
}

// one step of the recorded tape from the current Q[0]: the level set of
// every stage is loaded from the tape instead of advected, the time step is
// the tape's, band maintenance and scale separation are skipped. With rec,
// the band volume fractions after each geometry pass and the mixing records
// of each stage are kept in the adjoint workspace.
static void enqueue_replay(msf_ctx* c, const char* tape, bool rec) {
  const cudaStream_t s = c->stream;
  Inst& in = c->inst[0];
  const Grid& g = in.g;
  const Bufs& b = in.b;
  const int nb = in.nblk_band;
  AdjBufs& a = c->adj;
  launch_adj_begin(b, (const double*)(tape + sizeof(double)), s);
  tape_slot_load(in, tape, 0, s);
  launch_masks(g, b, s);
  launch_geometry(g, b, b.Q[0], nullptr, nb, s);
  launch_band_save(g, b, nb, s);
  if (rec) launch_adj_alpha(g, b, a.aband[0], 1, nb, s);
  for (int st = 0; st < g.rk; st++) {
    double* Qs = b.Q[st];
    double* Qo = st == g.rk - 1 ? b.Q[0] : b.Q[st + 1];
    c->ops->prim(g, b, Qs, nb, s);
    void* W[2] = {b.W0, b.W1};
    uint8_t* F[2] = {b.f0, b.f1};
    int cur = 0;
    for (int k = 0; k < g.ext_sweeps; k++) {
      c->ops->extend(g, b, W[cur], W[cur ^ 1], F[cur], F[cur ^ 1], nb, s);
      cur ^= 1;
    }
    c->ops->cons(g, b, Qs, W[cur], F[cur], nb, s);
    c->ops->bc_uhat(g, b, Qs, s);
    c->ops->interface(g, b, Qs, st, nb, s);
    c->ops->flux(g, b, Qs, b.Q[0], Qo, g.rk_beta[st], 1.0 - g.rk_beta[st], in.bb, nullptr, nullptr, s);
    launch_ledger(g, b, in.nbnd, g.rk_lw[st], s);
    tape_slot_load(in, tape, st + 1, s);
    launch_geometry(g, b, Qo, nullptr, nb, s);
    if (rec) {
      launch_adj_alpha(g, b, a.aband[st + 1], 1, nb, s);
      Bufs br = b;
      br.mixn = a.mixn[st];
      br.mixoff = a.mixoff[st];
      br.mixbeta = a.mixbeta[st];
      br.mixT = a.mixT[st];
      launch_mix(g, br, Qo, nb, s);
    } else {
      launch_mix(g, b, Qo, nb, s);
    }
  }
}

__global__ void k_replay_end(Ctl* ctl, const double* tape_t) {
  ctl->t = *tape_t + ctl->dt;
  ctl->cnt[C_STEPS] += 1;
}

extern "C" msf_status msf_replay_step(msf_ctx* c, const void* tape) {
  msf_status st = check_single(c);
  if (st != MSF_OK) return st;
  if (!tape || !tape_aligned(tape)) return fail(c, MSF_EINVAL, "tape must be a 256-byte aligned device buffer");
  if ((st = ensure_adjoint(c)) != MSF_OK) return st;
  enqueue_replay(c, (const char*)tape, false);
  k_replay_end<<<1, 1, 0, c->stream>>>(c->inst[0].b.ctl, (const double*)tape);
  c->ops->qf_copy(c->inst[0].g, c->inst[0].b, 0, 0, c->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, MSF_ECUDA, std::string("replay launch: ") + cudaGetErrorString(e));
  return read_error(c);
}

extern "C" msf_status msf_set_conserved(msf_ctx* c, int32_t i, const double* Q, int32_t mem) {
  msf_status st = check_instance(c, i);
  if (st != MSF_OK) return st;
  if (!Q) return fail(c, MSF_EINVAL, "Q is NULL");
  if (mem != MSF_HOST && mem != MSF_DEVICE) return fail(c, MSF_EINVAL, "mem");
  Inst& in = c->inst[i];
  const Grid& g = in.g;
  void* dQ = nullptr;
  if ((st = stage_in(c, Q, sizeof(double) * g.n_interior * g.N * g.NV, mem, &dQ)) != MSF_OK) return st;
  launch_adj_io(g, AdjBufs{}, (const double*)dQ, in.b.Q[0], 2, c->stream);
  c->ops->qf_copy(g, in.b, 0, 0, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  cudaFree(dQ);
  if (e != cudaSuccess) return fail(c, MSF_ECUDA, std::string("set_conserved: ") + cudaGetErrorString(e));
  return MSF_OK;
}

extern "C" msf_status msf_adjoint_step(msf_ctx* c, const void* tape_, const double* lam_out, double* lam_in,
                                       double* d_eos, double* d_inflow) {
  msf_status st = check_single(c);
  if (st != MSF_OK) return st;
  if (!tape_ || !tape_aligned(tape_)) return fail(c, MSF_EINVAL, "tape must be a 256-byte aligned device buffer");
  if (!lam_out || !lam_in) return fail(c, MSF_EINVAL, "NULL adjoint array");
  for (int m = 0; m < c->N; m++)
    if (c->inst[0].g.eos_kind[m] != MSF_EOS_STIFFENED)
      return fail(c, MSF_EUNSUPPORTED, "the adjoint step takes stiffened-gas materials only");
  if ((st = ensure_adjoint(c)) != MSF_OK) return st;
  const char* tape = (const char*)tape_;
  const cudaStream_t s = c->stream;
  Inst& in = c->inst[0];
  const Grid& g = in.g;
  const Bufs& b = in.b;
  const int nb = in.nblk_band;
  AdjBufs& a = c->adj;
  const TapeLayout L = tape_layout(g);
  const size_t qbytes = sizeof(double) * g.N * g.NV * g.ncell;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_pin, tape, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));
  const double dt = c->h_pin[1];
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, MSF_EINVAL, "tape holds no step");
  cudaMemsetAsync(a.deos, 0, sizeof(double) * MAXM * 2, s);
  cudaMemsetAsync(a.dinf, 0, sizeof(double) * 30, s);
  launch_adj_io(g, a, lam_out, nullptr, 0, s);
  // recompute the stages from the tape: Q^(1), Q^(2), band volume fractions, mixing records
  CUDA_TRY(c, cudaMemcpyAsync(b.Q[0], tape + L.q, qbytes, cudaMemcpyDeviceToDevice, s));
  enqueue_replay(c, tape, true);
  void* W[2] = {b.W0, b.W1};
  uint8_t* F[2] = {b.f0, b.f1};
  for (int sg = g.rk - 1; sg >= 0; sg--) {
    if (sg == 0) CUDA_TRY(c, cudaMemcpyAsync(b.Q[0], tape + L.q, qbytes, cudaMemcpyDeviceToDevice, s));
    const double* Qs = b.Q[sg];
    const double beta = g.rk_beta[sg], omb = 1.0 - g.rk_beta[sg];
    // stage-s geometry and states of the forward step
    tape_slot_load(in, tape, sg, s);
    launch_geometry(g, b, Qs, nullptr, nb, s);
    launch_adj_alpha(g, b, a.aband[sg], 0, nb, s);
    c->ops->prim(g, b, Qs, nb, s);
    launch_adj_level(g, b, a, b.f0, 0, nb, s);
    int cur = 0;
    for (int k = 1; k <= g.ext_sweeps; k++) {
      c->ops->extend(g, b, W[cur], W[cur ^ 1], F[cur], F[cur ^ 1], nb, s);
      cur ^= 1;
      launch_adj_level(g, b, a, F[cur], k, nb, s);
    }
    c->ops->cons(g, b, Qs, W[cur], F[cur], nb, s);
    c->ops->bc_uhat(g, b, Qs, s);
    c->ops->interface(g, b, Qs, sg, nb, s);
    // reverse: mixing, fluxes and exchange, boundary states, stencil states,
    // extension sweeps, primitive recovery, RK combination
    cudaMemsetAsync(a.LU, 0, qbytes, s);
    cudaMemsetAsync(a.LQ, 0, qbytes, s);
    cudaMemsetAsync(a.LW0, 0, qbytes, s);
    cudaMemsetAsync(a.LW1, 0, qbytes, s);
    launch_adj_mix(g, b, a, sg, (const uint8_t*)(tape + L.chi + (size_t)g.ncell * (sg + 1)), nb, s);
    c->aops->flux(g, b, a, Qs, omb * dt, s);
    c->aops->interface(g, b, a, Qs, omb * dt, nb, s);
    launch_adj_bc(g, b, a, s);
    c->aops->cons(g, b, a, W[cur], F[cur], a.LW0, nb, s);
    double* LW[2] = {a.LW0, a.LW1};
    int lc = 0;
    for (int k = g.ext_sweeps; k >= 1; k--) {
      launch_adj_ext(g, b, a, LW[lc], LW[lc ^ 1], k, nb, s);
      lc ^= 1;
    }
    launch_adj_prim(g, b, a, Qs, LW[lc], nb, s);
    launch_adj_combine(g, b, a, beta, omb, sg == g.rk - 1 ? 1 : 0, s);
  }
  launch_adj_io(g, a, nullptr, lam_in, 1, s);
  // back to the state at the start of the tape's step
  tape_slot_load(in, tape, 0, s);
  launch_masks(g, b, s);
  launch_geometry(g, b, b.Q[0], nullptr, nb, s);
  launch_adj_end(b, (const double*)tape, s);
  c->ops->qf_copy(g, b, 0, 0, s);
  CUDA_TRY(c, cudaMemcpyAsync(c->h_pin, a.deos, sizeof(double) * 2 * MAXM, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaMemcpyAsync(c->h_pin + 2 * MAXM, a.dinf, sizeof(double) * 30, cudaMemcpyDeviceToHost, s));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, MSF_ECUDA, std::string("adjoint launch: ") + cudaGetErrorString(e));
  if ((st = read_error(c)) != MSF_OK) return st;
  if (d_eos)
    for (int k = 0; k < 2 * g.N; k++) d_eos[k] += c->h_pin[k];
  if (d_inflow)
    for (int k = 0; k < 30; k++) d_inflow[k] += c->h_pin[2 * MAXM + k];
  return MSF_OK;
}

// message slot of calls without a context (used by msf_cfl_dt_noalloc)
extern "C" void msf_internal_set_error(const char* msg) { g_create_err = msg ? msg : ""; }

extern "C" const char* msf_last_error(const msf_ctx* c) {
  if (!c) return g_create_err.c_str();
  return c->err.c_str();
}
