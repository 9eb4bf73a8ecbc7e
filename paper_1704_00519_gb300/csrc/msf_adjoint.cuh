// msf_adjoint.cuh -- adjoint (reverse-mode) kernels of one TVD-RK3 step at
// frozen interface evolution.
//
// Frozen interface evolution: the level set of every stage, the time step and
// every discrete choice the step makes from the state (interface pair, the
// correction's material, small cells and their mixing targets) are those of
// a recorded forward step. What stays a function of the conserved state Q^n
// and of the EOS parameters (gamma_m, pinf_m) is the flow part of the step:
// primitive recovery, ghost extension (linear, Sec. 2.3.2), the reduced
// interface exchange (HLLC, Sec. 2.3.2), the aperture-weighted WENO5-LLF
// fluxes and the RK combination (Sec. 2.3, Eq. discretized_equ, Eq.
// local-advection) and conservative mixing (linear). These kernels pull an
// adjoint of the stage output back through each of these, in reverse order.
//
// Included after msf_kernels.cuh; T is the storage type of the stencil and
// primitive states (double or float), the adjoint accumulates in double.
#pragma once

#include "msf_adjoint.h"

namespace msf {
namespace {

// ------------------------------------------------------------- dual numbers
// forward-mode dual number with K partials; used for the local Jacobian of
// the HLLC interface state (ten inputs, two outputs)
template <int K>
struct Dual {
  double v;
  double d[K];
  __device__ Dual() {}
  __device__ Dual(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < K; i++) d[i] = 0.0;
  }
};
template <int K>
__device__ inline Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int K>
__device__ inline Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int K>
__device__ inline Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = -a.d[i];
  return r;
}
template <int K>
__device__ inline Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int K>
__device__ inline Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int K>
__device__ inline bool operator>(const Dual<K>& a, const Dual<K>& b) { return a.v > b.v; }
template <int K>
__device__ inline bool operator<(const Dual<K>& a, const Dual<K>& b) { return a.v < b.v; }
template <int K>
__device__ inline Dual<K> sqrt(const Dual<K>& a) {
  Dual<K> r;
  r.v = ::sqrt(a.v);
  const double s = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = a.d[i] * s;
  return r;
}
template <int K>
__device__ inline Dual<K> fmin(const Dual<K>& a, const Dual<K>& b) { return b.v < a.v ? b : a; }
template <int K>
__device__ inline Dual<K> fmax(const Dual<K>& a, const Dual<K>& b) { return b.v > a.v ? b : a; }

// ---------------------------------------------------- local derivatives
// gradient of the WENO5-JS value (weno5) with respect to its five arguments,
// in the arithmetic type A
template <typename A>
__device__ inline A weno5_grad(A a, A b, A c, A d, A e, A eps, A* gr) {
  const A r6 = A(1.0 / 6.0), k13 = A(13.0 / 12.0), k136 = A(13.0 / 6.0);
  const A q0 = (A(2) * a - A(7) * b + A(11) * c) * r6;
  const A q1 = (-b + A(5) * c + A(2) * d) * r6;
  const A q2 = (A(2) * c + A(5) * d - e) * r6;
  const A t00 = a - A(2) * b + c, t01 = a - A(4) * b + A(3) * c;
  const A t10 = b - A(2) * c + d, t11 = b - d;
  const A t20 = c - A(2) * d + e, t21 = A(3) * c - A(4) * d + e;
  const A s0 = k13 * t00 * t00 + A(0.25) * t01 * t01;
  const A s1 = k13 * t10 * t10 + A(0.25) * t11 * t11;
  const A s2 = k13 * t20 * t20 + A(0.25) * t21 * t21;
  const A b0 = eps + s0, b1 = eps + s1, b2 = eps + s2;
  const A a0 = A(0.1) / (b0 * b0), a1 = A(0.6) / (b1 * b1), a2 = A(0.3) / (b2 * b2);
  const A rA = A(1) / (a0 + a1 + a2);
  const A w0 = a0 * rA, w1 = a1 * rA, w2 = a2 * rA;
  const A out = w0 * q0 + w1 * q1 + w2 * q2;
  // d out / d s_k = (q_k - out) / A * d a_k / d s_k, d a_k / d s_k = -2 a_k / b_k
  const A c0 = (q0 - out) * rA * (A(-2) * a0 / b0);
  const A c1 = (q1 - out) * rA * (A(-2) * a1 / b1);
  const A c2 = (q2 - out) * rA * (A(-2) * a2 / b2);
  // linear parts
  gr[0] = w0 * A(2) * r6;
  gr[1] = w0 * A(-7) * r6 + w1 * A(-1) * r6;
  gr[2] = w0 * A(11) * r6 + w1 * A(5) * r6 + w2 * A(2) * r6;
  gr[3] = w1 * A(2) * r6 + w2 * A(5) * r6;
  gr[4] = w2 * A(-1) * r6;
  // smoothness indicators
  const A u00 = c0 * k136 * t00, u01 = c0 * A(0.5) * t01;
  gr[0] += u00 + u01;
  gr[1] += A(-2) * u00 - A(4) * u01;
  gr[2] += u00 + A(3) * u01;
  const A u10 = c1 * k136 * t10, u11 = c1 * A(0.5) * t11;
  gr[1] += u10 + u11;
  gr[2] += A(-2) * u10;
  gr[3] += u10 - u11;
  const A u20 = c2 * k136 * t20, u21 = c2 * A(0.5) * t21;
  gr[2] += u20 + A(3) * u21;
  gr[3] += A(-2) * u20 - A(4) * u21;
  gr[4] += u20 + u21;
  return out;
}

// reverse of cons_to_prim for material m: u -> w = (rho, vel, p); adds the
// pull-back of gw to gu and the EOS partials (d/dgamma, d/dpinf) to ge
__device__ inline void c2p_reverse(const Grid& g, int m, int D, const double* u, const double* gw, double* gu,
                                   double* ge) {
  const double rho = u[0];
  double vel[3] = {0, 0, 0}, qs = 0.0;
  for (int d = 0; d < D; d++) {
    vel[d] = u[1 + d] / rho;
    qs += vel[d] * vel[d];
  }
  const double ke = 0.5 * rho * qs;
  const double gp = gw[D + 1];
  gu[D + 1] += gp * g.gm1[m];
  const double gke = -gp * g.gm1[m];
  ge[0] += gp * (u[D + 1] - ke - g.pinf[m]);
  ge[1] += -gp * g.gamma[m];
  double grho = gw[0] + gke * 0.5 * qs;
  for (int d = 0; d < D; d++) {
    const double gv = gw[1 + d] + gke * rho * vel[d];
    gu[1 + d] += gv / rho;
    grho -= gv * vel[d] / rho;
  }
  gu[0] += grho;
}

// reverse of prim_to_cons for material m: w -> u; adds to gw and ge
__device__ inline void p2c_reverse(const Grid& g, int m, int D, const double* w, const double* gu, double* gw,
                                   double* ge) {
  const double rho = w[0];
  double qs = 0.0;
  for (int d = 0; d < D; d++) qs += w[1 + d] * w[1 + d];
  const double gE = gu[D + 1];
  double grho = gu[0] + gE * 0.5 * qs;
  for (int d = 0; d < D; d++) {
    grho += gu[1 + d] * w[1 + d];
    gw[1 + d] += gu[1 + d] * rho + gE * rho * w[1 + d];
  }
  gw[0] += grho;
  gw[D + 1] += gE / g.gm1[m];
  // E_int = (p + gamma pinf) / (gamma - 1)
  const double gm1 = g.gm1[m];
  ge[0] += gE * (g.pinf[m] / gm1 - (w[D + 1] + g.gpi[m]) / (gm1 * gm1));
  ge[1] += gE * g.gamma[m] / gm1;
}

// block-level accumulation of EOS partials: s_de[2 m + k]
__device__ inline void eos_block_flush(double* s_de, double* deos, int N) {
  __syncthreads();
  if (threadIdx.x < 2 * N && s_de[threadIdx.x] != 0.0) atomicAdd(&deos[threadIdx.x], s_de[threadIdx.x]);
}
__device__ inline void eos_block_init(double* s_de, int N) {
  if (threadIdx.x < 2 * MAXM) s_de[threadIdx.x] = 0.0;
  __syncthreads();
}

// adjoint of the stage update seen by the state of material m of cell c:
// omb dt lambda~ where the cell is updated, else 0
__device__ inline bool updated(const Grid& g, const Bufs& b, long long c, int m) {
  return interior_c(g, c) && ((b.smask[c] >> m) & 1u);
}

// ------------------------------------------------------------ flux adjoint
// faces of axis DIR: the face's flux F enters L of its upper cell with
// +A rh and of its lower cell with -A rh; g = A rh (mu_R - mu_L) is pulled
// back through WENO5 of the Lax-Friedrichs split fluxes to the six stencil
// states and the EOS of the material (the same stencil states as the forward
// flux: interior cells from interior_uhat, halo cells from Uh). The
// arithmetic is the stencil states' type T (the forward flux's), the
// accumulation FP64.
template <int D, typename T, int DIR>
__global__ void __launch_bounds__(NTHREADS) k_adj_flux(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                                                       const __grid_constant__ AdjBufs a, const double* Qs,
                                                       double omb_dt) {
  constexpr int NV = D + 2;
  __shared__ double s_de[2 * MAXM];
  eos_block_init(s_de, g.N);
  long long nf = (long long)(g.n[DIR] + 1);
  for (int e = 0; e < D; e++)
    if (e != DIR) nf *= g.n[e];
  const long long total = nf * g.N;
  const T eps = (T)g.weno_eps;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
       it += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(it / nf);
    long long r = it - (long long)m * nf;
    int q[3] = {0, 0, 0};
    for (int e = 0; e < D; e++) {
      const long long ne = e == DIR ? g.n[e] + 1 : g.n[e];
      q[e] = g.off[e] + (int)(r % ne);
      r /= ne;
    }
    const long long cR = cell_at(g, q[0], q[1], q[2]), cL = cR - g.st[DIR];
    const double Af = face_aperture(g, b, cL, cR, DIR, m);
    if (!(Af > 0.0)) continue;
    T gF[NV];
    const bool uL = updated(g, b, cL, m), uR = updated(g, b, cR, m);
    bool any = false;
    for (int v = 0; v < NV; v++) {
      const double muL = uL ? omb_dt * a.LA[qidx(g, m, v, cL)] : 0.0;
      const double muR = uR ? omb_dt * a.LA[qidx(g, m, v, cR)] : 0.0;
      gF[v] = (T)(Af * g.rh[DIR] * (muR - muL));
      any = any || gF[v] != T(0);
    }
    if (!any) continue;
    // stencil states
    T U[6][NV], un[6], pr[6], cs[6], vel[6][D];
    long long cq[6];
    bool ok = true;
    const T gm1 = (T)g.gm1[m], gpi = (T)g.gpi[m], gam = (T)g.gamma[m], pinf = (T)g.pinf[m];
    for (int k = 0; k < 6 && ok; k++) {
      const long long cc = cL + (long long)(k - 2) * g.st[DIR];
      cq[k] = cc;
      if (interior_c(g, cc)) {
        interior_uhat<T>(g, b, Qs, cc, m, U[k]);
      } else {
        const T* Uh = (const T*)b.Uh;
        for (int v = 0; v < NV; v++) U[k][v] = Uh[qidx(g, m, v, cc)];
      }
      if (isnan(U[k][0])) ok = false;
    }
    if (!ok) continue;
    for (int k = 0; k < 6; k++) {
      const T rho = U[k][0];
      T qs = T(0);
      for (int e = 0; e < D; e++) {
        vel[k][e] = U[k][1 + e] / rho;
        qs += vel[k][e] * vel[k][e];
      }
      pr[k] = gm1 * (U[k][D + 1] - T(0.5) * rho * qs) - gpi;
      const T c2 = gam * (pr[k] + pinf) / rho;
      cs[k] = c2 > T(0) ? ::sqrt(c2) : T(0);
      un[k] = vel[k][DIR];
    }
    T al = T(0);
    int kst = -1;
    for (int k = 0; k < 6; k++) {
      const T sp = fabs(un[k]) + cs[k];
      if (sp > al) {
        al = sp;
        kst = k;
      }
    }
    T gU[6][NV], gun[6], gpr[6], gcs[6];
    for (int k = 0; k < 6; k++) {
      gun[k] = gpr[k] = gcs[k] = T(0);
      for (int v = 0; v < NV; v++) gU[k][v] = T(0);
    }
    T gal = T(0);
    for (int v = 0; v < NV; v++) {
      if (gF[v] == T(0)) continue;
      T fp[6], fm[6];
      for (int k = 0; k < 6; k++) {
        const T uu = U[k][v];
        T F;
        if (v == 0) F = U[k][1 + DIR];
        else if (v == NV - 1) F = un[k] * (uu + pr[k]);
        else F = (v - 1 == DIR) ? uu * un[k] + pr[k] : uu * un[k];
        fp[k] = T(0.5) * (F + al * uu);
        fm[k] = T(0.5) * (F - al * uu);
      }
      T gp5[5], gm5[5];
      weno5_grad<T>(fp[0], fp[1], fp[2], fp[3], fp[4], eps, gp5);
      weno5_grad<T>(fm[5], fm[4], fm[3], fm[2], fm[1], eps, gm5);
      T gfp[6] = {T(0), T(0), T(0), T(0), T(0), T(0)}, gfm[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
      for (int k = 0; k < 5; k++) {
        gfp[k] = gF[v] * gp5[k];
        gfm[5 - k] = gF[v] * gm5[k];
      }
      for (int k = 0; k < 6; k++) {
        const T gFk = T(0.5) * (gfp[k] + gfm[k]);
        const T dpm = gfp[k] - gfm[k];
        gU[k][v] += T(0.5) * al * dpm;
        gal += T(0.5) * U[k][v] * dpm;
        if (gFk == T(0)) continue;
        if (v == 0) {
          gU[k][1 + DIR] += gFk;
        } else if (v == NV - 1) {
          gun[k] += gFk * (U[k][v] + pr[k]);
          gU[k][v] += gFk * un[k];
          gpr[k] += gFk * un[k];
        } else {
          gU[k][v] += gFk * un[k];
          gun[k] += gFk * U[k][v];
          if (v - 1 == DIR) gpr[k] += gFk;
        }
      }
    }
    if (kst >= 0) {
      gun[kst] += gal * (un[kst] > T(0) ? T(1) : (un[kst] < T(0) ? T(-1) : T(0)));
      gcs[kst] += gal;
    }
    T ge0 = T(0), ge1 = T(0);
    for (int k = 0; k < 6; k++) {
      const T rho = U[k][0];
      T gp = gpr[k], grho = T(0);
      T gvel[3] = {T(0), T(0), T(0)};
      gvel[DIR] += gun[k];
      if (gcs[k] != T(0) && cs[k] > T(0)) {
        const T c2 = cs[k] * cs[k];
        const T gc2 = gcs[k] * T(0.5) / cs[k];
        gp += gc2 * gam / rho;
        grho -= gc2 * c2 / rho;
        ge0 += gc2 * (pr[k] + pinf) / rho;
        ge1 += gc2 * gam / rho;
      }
      T qs = T(0);
      for (int e = 0; e < D; e++) qs += vel[k][e] * vel[k][e];
      const T ke = T(0.5) * rho * qs;
      gU[k][D + 1] += gp * gm1;
      const T gke = -gp * gm1;
      ge0 += gp * (U[k][D + 1] - ke - pinf);
      ge1 += -gp * gam;
      grho += gke * T(0.5) * qs;
      for (int e = 0; e < D; e++) {
        const T gv = gvel[e] + gke * rho * vel[k][e];
        gU[k][1 + e] += gv / rho;
        grho -= gv * vel[k][e] / rho;
      }
      gU[k][0] += grho;
      for (int v = 0; v < NV; v++)
        if (gU[k][v] != T(0)) atomicAdd(&a.LU[qidx(g, m, v, cq[k])], (double)gU[k][v]);
    }
    if (ge0 != T(0)) atomicAdd(&s_de[2 * m], (double)ge0);
    if (ge1 != T(0)) atomicAdd(&s_de[2 * m + 1], (double)ge1);
  }
  eos_block_flush(s_de, a.deos, g.N);
}

// ------------------------------------------------------- interface adjoint
// cut cells: X^m = p* (0, S^m, u* n.S^m) for the non-heaviest present
// materials and X^R = -sum; L += X rV. The pull-back of p*, u* goes through
// the HLLC state (dual numbers) and cons_to_prim of both materials.
template <typename T>
__global__ void k_adj_interface(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                                const __grid_constant__ AdjBufs a, const double* Qs, double omb_dt) {
  const int nb = b.ctl->nband, N = g.N, NV = g.NV, D = g.D;
  const T* Uh = (const T*)b.Uh;
  __shared__ double s_de[2 * MAXM];
  eos_block_init(s_de, N);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
    const long long c = b.band[k];
    if (!(b.gflag[c] & GF_CUT)) continue;
    int eta = -1, xi = -1;
    for (int m = 0; m < N; m++)
      if (present(g, b, c, m) && (eta < 0 || Qs[qidx(g, m, 0, c)] > Qs[qidx(g, eta, 0, c)])) eta = m;
    for (int m = 0; m < N; m++)
      if (m != eta && present(g, b, c, m) && (xi < 0 || Qs[qidx(g, m, 0, c)] > Qs[qidx(g, xi, 0, c)])) xi = m;
    if (xi < 0) continue;
    int L, R;
    if (Qs[qidx(g, xi, 0, c)] < Qs[qidx(g, eta, 0, c)]) { L = xi; R = eta; }
    else { L = eta; R = xi; }
    double n[3];
    stored_normal(g, b, c, R, n);
    double uL[5], uR[5], wL[5], wR[5];
    for (int v = 0; v < NV; v++) {
      uL[v] = (double)Uh[qidx(g, L, v, c)];
      uR[v] = (double)Uh[qidx(g, R, v, c)];
    }
    if (isnan(uL[0]) || isnan(uR[0])) continue;
    cons_to_prim<double>(g, L, D, uL, wL);
    cons_to_prim<double>(g, R, D, uR, wR);
    double unl = 0.0, unr = 0.0;
    for (int d = 0; d < D; d++) {
      unl += wL[1 + d] * n[d];
      unr += wR[1 + d] * n[d];
    }
    Dual<10> x[10];
    const double xv[10] = {wL[0], unl, wL[D + 1], g.gamma[L], g.pinf[L], wR[0], unr, wR[D + 1], g.gamma[R], g.pinf[R]};
    for (int i = 0; i < 10; i++) {
      x[i] = Dual<10>(xv[i]);
      x[i].d[i] = 1.0;
    }
    Dual<10> us, ps;
    hllc_star<Dual<10>>(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], x[8], x[9], &us, &ps);
    // adjoint of X
    double gXR[5] = {0, 0, 0, 0, 0};
    const bool updR = updated(g, b, c, R);
    for (int v = 1; v < NV; v++) gXR[v] = updR ? omb_dt * a.LA[qidx(g, R, v, c)] * g.rV : 0.0;
    double gps = 0.0, gus = 0.0;
    for (int m = 0; m < N; m++) {
      if (m == R || !present(g, b, c, m)) continue;
      const bool upd = updated(g, b, c, m);
      double S[3] = {0, 0, 0}, nS = 0.0;
      for (int d = 0; d < D; d++) S[d] = (b.Ahi[aidx(g, d, m, c)] - b.Alo[aidx(g, d, m, c)]) * g.farea[d];
      for (int d = 0; d < D; d++) nS += n[d] * S[d];
      for (int d = 0; d < D; d++) {
        const double gx = (upd ? omb_dt * a.LA[qidx(g, m, 1 + d, c)] * g.rV : 0.0) - gXR[1 + d];
        gps += gx * S[d];
      }
      const double ge = (upd ? omb_dt * a.LA[qidx(g, m, D + 1, c)] * g.rV : 0.0) - gXR[D + 1];
      gps += ge * us.v * nS;
      gus += ge * ps.v * nS;
    }
    if (gps == 0.0 && gus == 0.0) continue;
    double gx[10];
    for (int i = 0; i < 10; i++) gx[i] = gus * us.d[i] + gps * ps.d[i];
    double gwL[5] = {0, 0, 0, 0, 0}, gwR[5] = {0, 0, 0, 0, 0};
    gwL[0] = gx[0];
    gwL[D + 1] = gx[2];
    gwR[0] = gx[5];
    gwR[D + 1] = gx[7];
    for (int d = 0; d < D; d++) {
      gwL[1 + d] = gx[1] * n[d];
      gwR[1 + d] = gx[6] * n[d];
    }
    double geL[2] = {gx[3], gx[4]}, geR[2] = {gx[8], gx[9]};
    double guL[5] = {0, 0, 0, 0, 0}, guR[5] = {0, 0, 0, 0, 0};
    c2p_reverse(g, L, D, uL, gwL, guL, geL);
    c2p_reverse(g, R, D, uR, gwR, guR, geR);
    for (int v = 0; v < NV; v++) {
      a.LU[qidx(g, L, v, c)] += guL[v];
      a.LU[qidx(g, R, v, c)] += guR[v];
    }
    atomicAdd(&s_de[2 * L], geL[0]);
    atomicAdd(&s_de[2 * L + 1], geL[1]);
    atomicAdd(&s_de[2 * R], geR[0]);
    atomicAdd(&s_de[2 * R + 1], geR[1]);
  }
  eos_block_flush(s_de, a.deos, N);
}

// -------------------------------------------------- stencil-state adjoint
// band cells: real states u = Q / alpha -> LQ; filled ghost states
// u = prim_to_cons(W) -> adjoint of W (start of the reversed sweeps)
template <typename T>
__global__ void k_adj_cons(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                           const __grid_constant__ AdjBufs a, const void* Wfin, const uint8_t* ffin, double* lw) {
  const int nb = b.ctl->nband, N = g.N, NV = g.NV, D = g.D;
  const T* W = (const T*)Wfin;
  __shared__ double s_de[2 * MAXM];
  eos_block_init(s_de, N);
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nb * N; it += gridDim.x * blockDim.x) {
    const int m = it / nb, k = it - m * nb;
    const long long c = b.band[k];
    if (!((b.smask[c] >> m) & 1u)) continue;
    double gu[5];
    bool any = false;
    for (int v = 0; v < NV; v++) {
      gu[v] = a.LU[qidx(g, m, v, c)];
      any = any || gu[v] != 0.0;
    }
    if (!any) continue;
    if (b.isreal[midx(g, m, c)]) {
      const double al = b.alpha[midx(g, m, c)];
      for (int v = 0; v < NV; v++) a.LQ[qidx(g, m, v, c)] += gu[v] / al;
    } else if (ffin[midx(g, m, c)]) {
      double w[5], gw[5] = {0, 0, 0, 0, 0}, ge[2] = {0, 0};
      for (int v = 0; v < NV; v++) w[v] = (double)W[qidx(g, m, v, c)];
      p2c_reverse(g, m, D, w, gu, gw, ge);
      for (int v = 0; v < NV; v++) lw[qidx(g, m, v, c)] = gw[v];
      atomicAdd(&s_de[2 * m], ge[0]);
      atomicAdd(&s_de[2 * m + 1], ge[1]);
    }
  }
  eos_block_flush(s_de, a.deos, N);
}

}  // namespace

// ------------------------------------------------------------ launchers
template <typename T>
static void l_adj_flux(const Grid& g, const Bufs& b, const AdjBufs& a, const double* Qs, double omb_dt,
                       cudaStream_t s) {
  long long faces = 0;
  for (int d = 0; d < g.D; d++) {
    long long nf = g.n[d] + 1;
    for (int e = 0; e < g.D; e++)
      if (e != d) nf *= g.n[e];
    faces = nf > faces ? nf : faces;
  }
  long long blocks = (faces * g.N + NTHREADS - 1) / NTHREADS;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  const int nb = (int)blocks;
  if (g.D == 1) {
    k_adj_flux<1, T, 0><<<nb, NTHREADS, 0, s>>>(g, b, a, Qs, omb_dt);
  } else if (g.D == 2) {
    k_adj_flux<2, T, 0><<<nb, NTHREADS, 0, s>>>(g, b, a, Qs, omb_dt);
    k_adj_flux<2, T, 1><<<nb, NTHREADS, 0, s>>>(g, b, a, Qs, omb_dt);
  } else {
    k_adj_flux<3, T, 0><<<nb, NTHREADS, 0, s>>>(g, b, a, Qs, omb_dt);
    k_adj_flux<3, T, 1><<<nb, NTHREADS, 0, s>>>(g, b, a, Qs, omb_dt);
    k_adj_flux<3, T, 2><<<nb, NTHREADS, 0, s>>>(g, b, a, Qs, omb_dt);
  }
}
template <typename T>
static void l_adj_interface(const Grid& g, const Bufs& b, const AdjBufs& a, const double* Qs, double omb_dt,
                            int nblk, cudaStream_t s) {
  k_adj_interface<T><<<nblk, BAND_THREADS, 0, s>>>(g, b, a, Qs, omb_dt);
}
template <typename T>
static void l_adj_cons(const Grid& g, const Bufs& b, const AdjBufs& a, const void* W, const uint8_t* f, double* lw,
                       int nblk, cudaStream_t s) {
  k_adj_cons<T><<<nblk, BAND_THREADS, 0, s>>>(g, b, a, W, f, lw);
}
template <typename T>
static AdjOps make_adj_ops() {
  AdjOps o;
  o.flux = l_adj_flux<T>;
  o.interface = l_adj_interface<T>;
  o.cons = l_adj_cons<T>;
  return o;
}

}  // namespace msf
