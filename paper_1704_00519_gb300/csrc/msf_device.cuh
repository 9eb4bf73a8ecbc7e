// msf_device.cuh -- device building blocks of the cut-cell multi-material
// update (Pan, Han, Hu & Adams, arXiv:1704.00519): stiffened-gas EOS,
// WENO5-JS, the HLLC interface state, positive-part fractions of linear
// functions on simplices and the per-cell cut geometry.
//
// The FP64 kernels are compiled with -fmad=false so that every expression
// rounds exactly as written; the operation order below is part of the method
// definition (a fixed reading of the paper) and is kept stable on purpose.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace msf {

constexpr int G = 4;          // halo layers per side
constexpr int MAXM = 8;       // materials
constexpr int MIX_MAXT = 26;  // mixing targets per small cell

// error bits of the control block
constexpr unsigned ERR_NONFINITE = 1u, ERR_NEGATIVE = 2u, ERR_BAND = 4u;
// counters
enum { C_CUT = 0, C_MULTI, C_CORRECTED, C_SMALL, C_MIXFAIL, C_MERGE, C_ODDBALL, C_STEPS, NCOUNT };
// per-cell geometry flags
constexpr uint8_t GF_MIXED = 1, GF_CUT = 2;

// Everything a kernel needs to know about one instance's grid and materials.
struct Grid {
  int D, N, NV;
  int n[3], pn[3], off[3];
  long long st[3], ncell;
  double lo[3], h[3], rh[3], rh2[3], ih2[3], farea[3], V, rV, hmin, eps_ss, cap;
  int geom;    // 1: cylindrical grid of one dimension (x = radius)
  int fs_mat;  // held free-surface ambient, -1: none
  double fs_rho, fs_p0, fs_t0, fs_t1, fs_p1;
  double rk_c[4];  // time of stage s as a fraction of the step (s = rk: the step's end)
  double gamma[MAXM], pinf[MAXM], gm1[MAXM], gpi[MAXM];
  // Tait's equation per material (eos_kind 1): p = B (rho/rho0)^gamma - B + p0;
  // pinf holds B - p0 (sound speed and energy of the equivalent stiffened gas)
  int eos_kind[MAXM];
  double tait_B[MAXM], tait_rho0[MAXM], tait_p0[MAXM];
  double cfl, weno_eps, mix_alpha;
  int ext_sweeps, vel_sweeps, reinit_iters, scale_sep, reinit;
  int rk;                       // Runge-Kutta stages (2 or 3)
  int literal;                  // bit 0: printed reduced model, bit 1: |S| n area vectors
  int positivity;               // 1: positivity-preserving limiting of every face flux
  double rk_beta[3], rk_lw[3];  // beta_s of Eq. local-advection; ledger weight of stage s
  int bc[3][2], inflow_mat[3][2];
  double inflow_prim[3][2][5];
  long long n_interior;
};

// Device control block of one instance.
struct Ctl {
  double t, dt, t_end, lam;
  unsigned long long lam_bits;
  int active, last;
  unsigned err;
  int nband, nbnd;
  unsigned tile_ctr;  // next flux tile of the running flux-update launch
  unsigned mix_count; // (band cell, material) items of the running mixing pass that mix
  unsigned geom_count;  // 3D cut items listed by the running geometry pass
  unsigned ls_count;    // level-set items listed by the last geometry pass
  unsigned long long cnt[NCOUNT];
  double ledger[MAXM][5];
};

// ---------------------------------------------------------------- indexing
// cell counts are below 2^31 (checked at creation): 32-bit unsigned division
__host__ __device__ inline void coords(const Grid& g, long long c, int* q) {
  const unsigned cc = (unsigned)c, p0 = (unsigned)g.pn[0], p1 = (unsigned)g.pn[1];
  const unsigned t = cc / p0;
  q[0] = (int)(cc - t * p0);
  const unsigned z = t / p1;
  q[1] = (int)(t - z * p1);
  q[2] = (int)z;
}
// padded cell of the idx-th interior cell (interior order, x fastest)
__host__ __device__ inline long long interior_cell(const Grid& g, long long idx) {
  unsigned r = (unsigned)idx;
  int q[3] = {0, 0, 0};
  for (int d = 0; d < g.D; d++) {
    const unsigned nd = (unsigned)g.n[d], t = r / nd;
    q[d] = g.off[d] + (int)(r - t * nd);
    r = t;
  }
  return q[0] + g.st[1] * q[1] + g.st[2] * q[2];
}
__host__ __device__ inline long long cell_at(const Grid& g, int i, int j, int k) {
  return i + g.st[1] * j + g.st[2] * k;
}
__host__ __device__ inline bool in_array(const Grid& g, int i, int j, int k) {
  return i >= 0 && i < g.pn[0] && j >= 0 && j < g.pn[1] && k >= 0 && k < g.pn[2];
}
__host__ __device__ inline bool interior_q(const Grid& g, const int* q) {
  for (int d = 0; d < g.D; d++)
    if (q[d] < g.off[d] || q[d] >= g.off[d] + g.n[d]) return false;
  return true;
}
__host__ __device__ inline bool interior_c(const Grid& g, long long c) {
  int q[3];
  coords(g, c, q);
  return interior_q(g, q);
}
__host__ __device__ inline long long qidx(const Grid& g, int m, int v, long long c) {
  return ((long long)m * g.NV + v) * g.ncell + c;
}
__host__ __device__ inline long long midx(const Grid& g, int m, long long c) { return (long long)m * g.ncell + c; }
__host__ __device__ inline long long aidx(const Grid& g, int d, int m, long long c) {
  return ((long long)d * g.N + m) * g.ncell + c;
}
__device__ inline int popcount8(unsigned x) { return __popc(x & 0xffu); }

// ---------------------------------------------------------------- EOS (Sec. 2.1)
// Tait's equation (Sec. 2.1), evaluated in FP64: p = B (rho/rho0)^gamma - B + p0.
// Its pressure does not depend on the internal energy; the energy carried with
// it is that of the stiffened gas with pinf = B - p0 (prim_to_cons below).
__device__ inline double tait_pressure(const Grid& g, int m, double rho) {
  const double B = g.tait_B[m];
  return B * pow(rho / g.tait_rho0[m], g.gamma[m]) - B + g.tait_p0[m];
}
// conservative (rho, rho u, rho E) -> primitive (rho, u, p), in T, with the
// material's gamma - 1 and gamma pinf given in T
template <typename T>
__device__ inline void cons_to_prim_k(const Grid& g, int m, int D, const T* u, T* w, T gm1, T gpi) {
  T rho = u[0];
  T vel[3] = {T(0), T(0), T(0)};
  T q = T(0);
  for (int d = 0; d < D; d++) vel[d] = u[1 + d] / rho;
  for (int d = 0; d < D; d++) q += vel[d] * vel[d];
  T ke = T(0.5) * rho * q;
  w[0] = rho;
  for (int d = 0; d < D; d++) w[1 + d] = vel[d];
  w[D + 1] = g.eos_kind[m] == 1 ? (T)tait_pressure(g, m, (double)rho) : gm1 * (u[D + 1] - ke) - gpi;
}
template <typename T>
__device__ inline void cons_to_prim(const Grid& g, int m, int D, const T* u, T* w) {
  cons_to_prim_k<T>(g, m, D, u, w, T(g.gm1[m]), T(g.gpi[m]));
}
template <typename T>
__device__ inline void prim_to_cons(const Grid& g, int m, int D, const T* w, T* u) {
  T rho = w[0];
  T q = T(0);
  for (int d = 0; d < D; d++) q += w[1 + d] * w[1 + d];
  u[0] = rho;
  for (int d = 0; d < D; d++) u[1 + d] = rho * w[1 + d];
  u[D + 1] = (w[D + 1] + T(g.gpi[m])) / T(g.gm1[m]) + T(0.5) * rho * q;
}
// c = sqrt(gamma (p + pinf) / rho); flags a non-physical state; gamma and
// pinf given in T
template <typename T>
__device__ inline T sound_k(T gam, T pinf, T rho, T p, unsigned* err) {
  T c2 = (gam * (p + pinf)) / rho;
  if (!(rho > T(0)) || !(c2 > T(0))) {
    *err |= ERR_NEGATIVE;
    c2 = c2 > T(0) ? c2 : T(0);
  }
  return sqrt(c2);
}
template <typename T>
__device__ inline T sound(const Grid& g, int m, T rho, T p, unsigned* err) {
  return sound_k<T>(T(g.gamma[m]), T(g.pinf[m]), rho, p, err);
}

// -------------------------- axisymmetric grid and free surface (Sec. 3, Case II)
// A cylindrical grid of one dimension takes x as the radius: cell i has volume
// r_i h and its faces the areas r_f (per radian and unit length).
__device__ inline double face_r(const Grid& g, int i) { return g.lo[0] + (double)(i - g.off[0]) * g.h[0]; }
__device__ inline double cell_r(const Grid& g, int i) { return g.lo[0] + ((double)(i - g.off[0]) + 0.5) * g.h[0]; }
// volume of cell c over the Cartesian cell volume (1 on Cartesian grids)
__device__ inline double vfac(const Grid& g, long long c) { return g.geom == 1 ? cell_r(g, (int)(c % g.pn[0])) : 1.0; }
// pressure of the free-surface ambient at time t: fs_p0 up to fs_t0, linear to
// fs_p1 at fs_t1, fs_p1 after
__device__ inline double fs_pressure(const Grid& g, double t) {
  if (t <= g.fs_t0) return g.fs_p0;
  if (t >= g.fs_t1) return g.fs_p1;
  return g.fs_p0 - (g.fs_p0 - g.fs_p1) * (t - g.fs_t0) / (g.fs_t1 - g.fs_t0);
}
// velocity jump across the wave of material m at (rho, pK) that takes its
// pressure to p, on the two-shock approximation of the Riemann problem
// (Toro, Riemann Solvers, Sec. 9.4.2): (p - pK) sqrt(A / (p + pinf + B)),
// A = 2 / ((gamma + 1) rho), B = (gamma - 1) / (gamma + 1) (pK + pinf)
template <typename T>
__device__ inline T fs_wave(const Grid& g, int m, T rho, T pK, T p) {
  const T ga = (T)g.gamma[m], pi = (T)g.pinf[m];
  const T A = T(2) / ((ga + T(1)) * rho), B = (ga - T(1)) / (ga + T(1)) * (pK + pi);
  return (p - pK) * sqrt(A / (p + pi + B));
}

// ---------------------------------------------------------------- WENO5-JS
// value at i+1/2 from cell values i-2..i+2 (Jiang & Shu weights 1/10, 6/10, 3/10)
template <typename T>
__device__ inline T weno5(T a, T b, T c, T d, T e, T eps) {
  const T r6 = T(1.0 / 6.0), k13 = T(13.0 / 12.0);
  T q0 = (T(2) * a - T(7) * b + T(11) * c) * r6;
  T q1 = (-b + T(5) * c + T(2) * d) * r6;
  T q2 = (T(2) * c + T(5) * d - e) * r6;
  T t = a - T(2) * b + c;
  T s0 = k13 * t * t;
  t = a - T(4) * b + T(3) * c;
  s0 = s0 + T(0.25) * t * t;
  t = b - T(2) * c + d;
  T s1 = k13 * t * t;
  t = b - d;
  s1 = s1 + T(0.25) * t * t;
  t = c - T(2) * d + e;
  T s2 = k13 * t * t;
  t = T(3) * c - T(4) * d + e;
  s2 = s2 + T(0.25) * t * t;
  T b0 = eps + s0, b1 = eps + s1, b2 = eps + s2;
  // Jiang & Shu's weights d_k / (eps + beta_k)^2, normalised by their sum
  const T a0 = T(0.1) / (b0 * b0);
  const T a1 = T(0.6) / (b1 * b1);
  const T a2 = T(0.3) / (b2 * b2);
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// ---------------------------------------------------------------- HLLC (Sec. 2.3.2)
// interface velocity and pressure of the two-state problem along n, for states
// (rho, u_n, p) of two stiffened gases or Tait materials (tl, tr; pinf = B - p0);
// wave speeds with Roe-averaged Psi, Upsilon and p/rho (c^2 = Psi + Upsilon p/rho:
// stiffened gas Psi = (p + gamma pinf)/rho, Upsilon = gamma - 1; Tait
// Psi = gamma (p + pinf)/rho, Upsilon = 0)
template <typename T>
__device__ inline void hllc_star(T rl, T ul, T pl, T gl, T pil, T rr, T ur, T pr, T gr, T pir, T* ustar, T* pstar,
                                 bool tl = false, bool tr = false) {
  T c2l = (gl * (pl + pil)) / rl, c2r = (gr * (pr + pir)) / rr;
  T cl = sqrt(c2l > T(0) ? c2l : T(0)), cr = sqrt(c2r > T(0) ? c2r : T(0));
  T psil = tl ? (gl * (pl + pil)) / rl : (pl + gl * pil) / rl;
  T psir = tr ? (gr * (pr + pir)) / rr : (pr + gr * pir) / rr;
  T upsl = tl ? T(0) : gl - T(1), upsr = tr ? T(0) : gr - T(1);
  T sl = sqrt(rl), sr = sqrt(rr);
  T den = sl + sr;
  T psit = (sl * psil + sr * psir) / den;
  T upst = (sl * upsl + sr * upsr) / den;
  T du = (ur - ul) / den;
  T prt = (sl * (pl / rl) + sr * (pr / rr)) / den + T(0.5) * (sl * sr) * (du * du);
  T ct2 = psit + upst * prt;
  T ct = sqrt(ct2 > T(0) ? ct2 : T(0));
  T ut = (sl * ul + sr * ur) / den;
  T SL = fmin(ul - cl, ut - ct);
  T SR = fmax(ut + ct, ur + cr);
  T ml = (ul - SL) * rl, mr = (SR - ur) * rr;
  T SM = (mr * ur + ml * ul + pl - pr) / (mr + ml);
  T psl = pl + rl * (SL - ul) * (SM - ul);
  T psr = pr + rr * (SR - ur) * (SM - ur);
  *ustar = SM;
  *pstar = T(0.5) * (psl + psr);
}

// ------------------------------------------- positive-part simplex fractions
__device__ inline double frac_seg(double a, double b) {
  int np = (a > 0.0) + (b > 0.0), nn = (a < 0.0) + (b < 0.0);
  if (nn == 0) return np == 0 ? 0.5 : 1.0;
  if (np == 0) return 0.0;
  double pos = a > 0.0 ? a : b, neg = a > 0.0 ? b : a;
  return pos / (pos - neg);
}
__device__ inline void sort3_desc(double& a, double& b, double& c) {
  // insertion order identical to a stable descending insertion sort
  double t;
  if (b > a) { t = a; a = b; b = t; }
  if (c > b) {
    t = b; b = c; c = t;
    if (b > a) { t = a; a = b; b = t; }
  }
}
__device__ inline double frac_tri(double a, double b, double c) {
  sort3_desc(a, b, c);
  int np = (a > 0.0) + (b > 0.0) + (c > 0.0);
  int nn = (a < 0.0) + (b < 0.0) + (c < 0.0);
  if (nn == 0) return np == 0 ? 0.5 : 1.0;
  if (np == 0) return 0.0;
  if (np == 1) return (a * a) / ((a - b) * (a - c));
  return 1.0 - (c * c) / ((a - c) * (b - c));
}
__device__ inline double frac_tet(double a, double b, double c, double d) {
  double v[4] = {a, b, c, d};
  for (int i = 1; i < 4; i++)
    for (int j = i; j > 0 && v[j] > v[j - 1]; j--) {
      double t = v[j]; v[j] = v[j - 1]; v[j - 1] = t;
    }
  int np = (v[0] > 0.0) + (v[1] > 0.0) + (v[2] > 0.0) + (v[3] > 0.0);
  int nn = (v[0] < 0.0) + (v[1] < 0.0) + (v[2] < 0.0) + (v[3] < 0.0);
  if (nn == 0) return np == 0 ? 0.5 : 1.0;
  if (np == 0) return 0.0;
  if (np == 1) return (v[0] * v[0] * v[0]) / (((v[0] - v[1]) * (v[0] - v[2])) * (v[0] - v[3]));
  if (np == 3) {
    double m3 = -v[3];
    return 1.0 - (m3 * m3 * m3) / (((v[0] - v[3]) * (v[1] - v[3])) * (v[2] - v[3]));
  }
  double A = v[0], B = v[1], C = v[2], E = v[3];
  double num = A * A * (B * B) - A * B * (A + B) * (C + E) + C * E * (A * A + A * B + B * B);
  double den = ((A - C) * (A - E)) * ((B - C) * (B - E));
  return num / den;
}

// strict sign tests on the bit pattern (integer compares, so that they leave
// the FP64 pipes free): 0 < x <= +inf, and -inf <= x < 0; a zero of either
// sign and a NaN fail both
__device__ __forceinline__ bool pos_bits(double x) {
  const long long u = __double_as_longlong(x);
  return u > 0 && u <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool neg_bits(double x) {
  const long long u = __double_as_longlong(x);
  return u > (long long)0x8000000000000000ULL && u <= (long long)0xfff0000000000000ULL;
}

// order key of a double: signed integers that compare as the values do (the
// magnitude bits of a negative value reversed), except that -0 sorts below +0
__device__ __forceinline__ long long okey(double x) {
  const long long u = __double_as_longlong(x);
  return u >= 0 ? u : (u ^ 0x7fffffffffffffffLL);
}

// a < b on the bit patterns (integer compares): the order keys, with a +0 and
// a -0 equal and a NaN unordered, as the IEEE comparison has them
__device__ __forceinline__ bool lt_bits(double a, double b) {
  const long long ma = __double_as_longlong(a) & 0x7fffffffffffffffLL;
  const long long mb = __double_as_longlong(b) & 0x7fffffffffffffffLL;
  const bool nan = ma > 0x7ff0000000000000LL || mb > 0x7ff0000000000000LL;
  return !nan && (ma | mb) != 0 && okey(a) < okey(b);
}

// The same fractions without divergent branches and without FP64 compares,
// for warps whose lanes take different cases: the values are sorted by a
// network of compare and exchange steps on their order keys, the signs are
// counted with the bit tests, every case's numerator and denominator is
// formed with the expressions above, and one division follows the selection.
// For values that are not NaN the results are those of frac_tri and frac_tet
// bit for bit: equal keys are equal values, and the only equal values that
// the keys order differently are a +0 and a -0, which no formula
// distinguishes (they enter only as differences a - 0 and as the one zero of
// a case with a single zero).
__device__ __forceinline__ void cx_desc(double& a, long long& ka, double& b, long long& kb) {
  const bool sw = kb > ka;
  const double hi = sw ? b : a, lo = sw ? a : b;
  const long long khi = sw ? kb : ka, klo = sw ? ka : kb;
  a = hi;
  b = lo;
  ka = khi;
  kb = klo;
}
__device__ __forceinline__ double frac_tri_nb(double a, double b, double c) {
  long long ka = okey(a), kb = okey(b), kc = okey(c);
  cx_desc(a, ka, b, kb);
  cx_desc(b, kb, c, kc);
  cx_desc(a, ka, b, kb);
  const int np = pos_bits(a) + pos_bits(b) + pos_bits(c);
  const int nn = neg_bits(a) + neg_bits(b) + neg_bits(c);
  const double n1 = a * a, d1 = (a - b) * (a - c);  // np == 1
  const double n2 = c * c, d2 = (a - c) * (b - c);  // np == 2
  const double q = (np == 1 ? n1 : n2) / (np == 1 ? d1 : d2);
  if (nn == 0) return np == 0 ? 0.5 : 1.0;
  if (np == 0) return 0.0;
  return np == 1 ? q : 1.0 - q;
}
__device__ __forceinline__ double frac_tet_nb(double a, double b, double c, double d) {
  long long ka = okey(a), kb = okey(b), kc = okey(c), kd = okey(d);
  cx_desc(a, ka, b, kb);
  cx_desc(c, kc, d, kd);
  cx_desc(a, ka, c, kc);
  cx_desc(b, kb, d, kd);
  cx_desc(b, kb, c, kc);
  const int np = pos_bits(a) + pos_bits(b) + pos_bits(c) + pos_bits(d);
  const int nn = neg_bits(a) + neg_bits(b) + neg_bits(c) + neg_bits(d);
  const double n1 = a * a * a, d1 = ((a - b) * (a - c)) * (a - d);  // np == 1
  const double m3 = -d;
  const double n3 = m3 * m3 * m3, d3 = ((a - d) * (b - d)) * (c - d);  // np == 3
  const double n2 = a * a * (b * b) - a * b * (a + b) * (c + d) + c * d * (a * a + a * b + b * b);
  const double d2 = ((a - c) * (a - d)) * ((b - c) * (b - d));  // np == 2
  const double q = (np == 1 ? n1 : (np == 3 ? n3 : n2)) / (np == 1 ? d1 : (np == 3 ? d3 : d2));
  if (nn == 0) return np == 0 ? 0.5 : 1.0;
  if (np == 0) return 0.0;
  return np == 3 ? 1.0 - q : q;
}

// ---------------------------------- local level sets (Sec. 2.2, operator C_m)
__device__ inline double phi_m(const double* phi, const uint8_t* chi, long long c, int m) {
  return chi[c] == m ? phi[c] : -phi[c];
}
// value at grid vertex (I, J, K): mean of the 2^D cells around it, summed in memory order
__device__ inline double vertex_val(const Grid& g, const double* phi, const uint8_t* chi, int I, int J, int K, int m) {
  const int D = g.D;
  double s = 0.0;
  const int k0 = D >= 3 ? K - 1 : K, j0 = D >= 2 ? J - 1 : J;
  for (int kk = k0; kk <= K; kk++)
    for (int jj = j0; jj <= J; jj++)
      for (int ii = I - 1; ii <= I; ii++) s += phi_m(phi, chi, cell_at(g, ii, jj, kk), m);
  return s * (D == 1 ? 0.5 : (D == 2 ? 0.25 : 0.125));
}
__device__ inline double facec_val(const Grid& g, const double* phi, const uint8_t* chi, long long c, int d, int side,
                                   int m) {
  long long a = side ? c : c - g.st[d], b = side ? c + g.st[d] : c;
  return (phi_m(phi, chi, a, m) + phi_m(phi, chi, b, m)) * 0.5;
}

// volume fraction and raw face apertures of material m in cell c
template <int D>
__device__ inline void cell_geom(const Grid& g, const double* phi, const uint8_t* chi, long long c, int m,
                                 double* alpha, double* alo, double* ahi) {
  int q[3];
  coords(g, c, q);
  const int i = q[0], j = q[1], k = q[2];
  double vc = phi_m(phi, chi, c, m);
  if constexpr (D == 1) {
    double c0 = vertex_val(g, phi, chi, i, j, k, m), c1 = vertex_val(g, phi, chi, i + 1, j, k, m);
    *alpha = (frac_seg(c0, vc) + frac_seg(vc, c1)) * 0.5;
    alo[0] = c0 > 0.0 ? 1.0 : (c0 < 0.0 ? 0.0 : 0.5);
    ahi[0] = c1 > 0.0 ? 1.0 : (c1 < 0.0 ? 0.0 : 0.5);
  } else if constexpr (D == 2) {
    double c00 = vertex_val(g, phi, chi, i, j, k, m), c10 = vertex_val(g, phi, chi, i + 1, j, k, m);
    double c01 = vertex_val(g, phi, chi, i, j + 1, k, m), c11 = vertex_val(g, phi, chi, i + 1, j + 1, k, m);
    alo[0] = frac_seg(c00, c01);
    ahi[0] = frac_seg(c10, c11);
    alo[1] = frac_seg(c00, c10);
    ahi[1] = frac_seg(c01, c11);
    *alpha = (frac_tri(vc, c00, c01) + frac_tri(vc, c10, c11) + frac_tri(vc, c00, c10) + frac_tri(vc, c01, c11)) * 0.25;
  } else {
    double cv[2][2][2];
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int e = 0; e < 2; e++) cv[a][b][e] = vertex_val(g, phi, chi, i + e, j + b, k + a, m);
    double vol = 0.0;
    for (int f = 0; f < 6; f++) {
      const int d = f >> 1, side = f & 1;
      double fc = facec_val(g, phi, chi, c, d, side, m);
      double p[4];
      // corners of face f in cyclic order
      if (d == 0) {
        p[0] = cv[0][0][side]; p[1] = cv[0][1][side]; p[2] = cv[1][1][side]; p[3] = cv[1][0][side];
      } else if (d == 1) {
        p[0] = cv[0][side][0]; p[1] = cv[0][side][1]; p[2] = cv[1][side][1]; p[3] = cv[1][side][0];
      } else {
        p[0] = cv[side][0][0]; p[1] = cv[side][0][1]; p[2] = cv[side][1][1]; p[3] = cv[side][1][0];
      }
      double ap = 0.0;
      for (int e = 0; e < 4; e++) {
        double p0 = p[e], p1 = p[(e + 1) & 3];
        ap += frac_tri(fc, p0, p1);
        vol += frac_tet(vc, fc, p0, p1);
      }
      ap = ap * 0.25;
      if (side) ahi[d] = ap; else alo[d] = ap;
    }
    *alpha = vol * (1.0 / 24.0);
  }
}

// one face f (axis f >> 1, side f & 1) of a 3D cell for material m: the raw
// aperture of the face and the four tetrahedron fractions between the face and
// the cell centre, each evaluated exactly as cell_geom<3> evaluates them (so
// that a caller summing them in cell_geom<3>'s order gets the same bits)
__device__ __forceinline__ void face_geom3(const Grid& g, const double* phi, const uint8_t* chi, long long c, int m, int f,
                                  double& ap, double (&t)[4]) {
  int q[3];
  coords(g, c, q);
  const int i = q[0], j = q[1], k = q[2];
  const double vc = phi_m(phi, chi, c, m);
  const int d = f >> 1, side = f & 1;
  const double fc = facec_val(g, phi, chi, c, d, side, m);
  // corner (e, b, a) of the cell is grid vertex (i + e, j + b, k + a)
  double p[4];
  if (d == 0) {
    p[0] = vertex_val(g, phi, chi, i + side, j, k, m);
    p[1] = vertex_val(g, phi, chi, i + side, j + 1, k, m);
    p[2] = vertex_val(g, phi, chi, i + side, j + 1, k + 1, m);
    p[3] = vertex_val(g, phi, chi, i + side, j, k + 1, m);
  } else if (d == 1) {
    p[0] = vertex_val(g, phi, chi, i, j + side, k, m);
    p[1] = vertex_val(g, phi, chi, i + 1, j + side, k, m);
    p[2] = vertex_val(g, phi, chi, i + 1, j + side, k + 1, m);
    p[3] = vertex_val(g, phi, chi, i, j + side, k + 1, m);
  } else {
    p[0] = vertex_val(g, phi, chi, i, j, k + side, m);
    p[1] = vertex_val(g, phi, chi, i + 1, j, k + side, m);
    p[2] = vertex_val(g, phi, chi, i + 1, j + 1, k + side, m);
    p[3] = vertex_val(g, phi, chi, i, j + 1, k + side, m);
  }
  ap = 0.0;
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const double p0 = p[e], p1 = p[(e + 1) & 3];
    ap += frac_tri_nb(fc, p0, p1);
    t[e] = frac_tet_nb(vc, fc, p0, p1);
  }
  ap = ap * 0.25;
}

// Conversions between binary32 and binary64 on the integer pipes, from the
// IEEE-754 layouts (sign, biased exponent, fraction); bit for bit the
// hardware conversions, which run on the FP64 pipes. Values outside the range
// handled here (subnormals, infinities, NaNs, and for the narrowing the
// binary32 subnormal and overflow range) take the hardware conversion.
//
// float -> double, exact: the exponent is rebiased (127 -> 1023) and the 23
// fraction bits become the leading 23 of 52.
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned u = __float_as_uint(x), mag = u & 0x7fffffffu;
  const unsigned e = mag >> 23;
  if (mag == 0u) return __hiloint2double((int)u, 0);  // +-0
  if (e == 0u || e == 0xffu) return (double)x;
  const unsigned hi = (u & 0x80000000u) | ((mag >> 3) + ((1023u - 127u) << 20));
  return __hiloint2double((int)hi, (int)(u << 29));
}
// double -> float, rounded to nearest even: the leading 23 of the 52 fraction
// bits are kept and the 29 dropped bits decide the rounding (a carry out of
// the fraction raises the exponent; out of the largest binade it gives
// infinity, as the rounding rule does).
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned mag = hi & 0x7fffffffu, E = mag >> 20;
  if ((mag | lo) == 0u) return __uint_as_float(hi);  // +-0
  if (E < 1023u - 126u || E > 1023u + 127u) return (float)x;
  unsigned r = (hi & 0x80000000u) | ((mag - ((1023u - 127u) << 20)) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu, half = 0x10000000u;
  r += (rem > half || (rem == half && (r & 1u))) ? 1u : 0u;
  return __uint_as_float(r);
}
// finite (neither infinite nor NaN): the exponent field is not all ones
__device__ __forceinline__ bool finite_bits(double x) {
  return (((unsigned)__double2hiint(x) >> 20) & 0x7ffu) != 0x7ffu;
}

// Uncut cell: the sign that phi^m takes at every simplex vertex of cell c
// (centre, corners and, in 3D, face centres; the values cell_geom computes,
// from the same functions): +1 when all are > 0, -1 when all are < 0, 0
// otherwise. For +1 every segment, triangle and tetrahedron fraction of the
// cell is exactly 1, for -1 exactly 0, so cell_geom's sums are constants.
template <int D>
__device__ __forceinline__ int uncut_sign(const Grid& g, const double* phi, const uint8_t* chi, long long c, int m) {
  int q[3];
  coords(g, c, q);
  const double vc = phi_m(phi, chi, c, m);
  bool pos = pos_bits(vc), neg = neg_bits(vc);
  if constexpr (D == 3) {
#pragma unroll
    for (int f = 0; f < 6; f++) {
      const double v = facec_val(g, phi, chi, c, f >> 1, f & 1, m);
      pos = pos && pos_bits(v);
      neg = neg && neg_bits(v);
    }
  }
  const int nz = D >= 3 ? 2 : 1;
#pragma unroll
  for (int a = 0; a < nz; a++)
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const double v = vertex_val(g, phi, chi, q[0] + e, q[1] + b, q[2] + a, m);
        pos = pos && pos_bits(v);
        neg = neg && neg_bits(v);
      }
  return pos ? 1 : (neg ? -1 : 0);
}

// min / max of phi^m over the simplex vertices of cell c (centre, corners, 3D face centres)
__device__ inline void vertex_minmax(const Grid& g, const double* phi, const uint8_t* chi, long long c, int m,
                                     double* mn, double* mx) {
  int q[3];
  coords(g, c, q);
  double lo = phi_m(phi, chi, c, m), hi = lo;
  const int nz = g.D >= 3 ? 2 : 1, ny = g.D >= 2 ? 2 : 1;
  for (int a = 0; a < nz; a++)
    for (int b = 0; b < ny; b++)
      for (int e = 0; e < 2; e++) {
        double v = vertex_val(g, phi, chi, q[0] + e, q[1] + b, q[2] + a, m);
        lo = fmin(lo, v);
        hi = fmax(hi, v);
      }
  if (g.D == 3)
    for (int d = 0; d < 3; d++)
      for (int s = 0; s < 2; s++) {
        double v = facec_val(g, phi, chi, c, d, s, m);
        lo = fmin(lo, v);
        hi = fmax(hi, v);
      }
  *mn = lo;
  *mx = hi;
}

// unit normal of phi^m by central differences (zero where the gradient vanishes)
__device__ inline void normal_m(const Grid& g, const double* phi, const uint8_t* chi, long long c, int m, double* n) {
  double gr[3] = {0.0, 0.0, 0.0}, q = 0.0;
  for (int d = 0; d < g.D; d++)
    gr[d] = (phi_m(phi, chi, c + g.st[d], m) - phi_m(phi, chi, c - g.st[d], m)) * g.rh2[d];
  for (int d = 0; d < g.D; d++) q += gr[d] * gr[d];
  double len = sqrt(q);
  n[0] = n[1] = n[2] = 0.0;
  if (len > 0.0)
    for (int d = 0; d < g.D; d++) n[d] = gr[d] / len;
}

// boundary source along axis d of halo coordinate idx: transmissive / inflow
// take the nearest interior cell; reflective mirrors about the boundary,
// repeatedly when the halo is deeper than the interior (flip: odd count)
__host__ __device__ inline int bc_source(const Grid& g, int d, int idx, int* side, int* flip) {
  const int n = g.n[d], off = g.off[d], r = idx - off;
  *side = r < 0 ? 0 : 1;
  *flip = 0;
  if (g.bc[d][*side] != 1) return r < 0 ? off : off + n - 1;
  const int P = 2 * n, k = ((r % P) + P) % P;
  const int count = r < 0 ? (-r - 1) / n + 1 : (r - n) / n + 1;
  *flip = count & 1;
  return off + (k >= n ? P - 1 - k : k);
}

__device__ inline void atomic_max_pos_double(unsigned long long* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace msf
