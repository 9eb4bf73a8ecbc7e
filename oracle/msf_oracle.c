/*
 * msf_oracle.c -- plain, slow, FP64 CPU oracle of the per-stage update of the
 * conservative sharp-interface method for compressible multi-material flows
 * (Pan, Han, Hu & Adams, arXiv:1704.00519).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py load this library. It shares no
 * source with the CUDA path and never calls it.
 *
 * Everything here is written as plain loops over cells in the order the
 * method states its steps. Where the paper is silent the fixed readings
 * below are used (the CUDA path makes the same choices independently):
 *
 *   EOS        stiffened gas p = (g-1) rho e - g pinf, c^2 = g (p+pinf)/rho;
 *              or Tait's p = B (rho/rho0)^g - B + p0 with the energy and the
 *              sound speed of the stiffened gas with pinf = B - p0 (Sec. 2.1)
 *              (Sec. 2.1; pinf = 0 gives the ideal gas of Sec. 2.1).
 *   geometry   per-material local field phi^m = C_m(phi, chi) (Sec. 2.2,
 *              construction operator); piecewise-linear interpolant on a
 *              simplex split of each cell (centre + corners [+ face centres]);
 *              volume fraction = positive-part measure, aperture = positive
 *              part of the face (Sec. 2.3, Eq. discretized_equ).
 *   correction alpha^{chi*} += 1 - sum(alpha), chi* = argmin alpha rho
 *              (Sec. 2.3.1, Eq. vol_corr2) in cells with >= 3 materials.
 *   ghosts     constant extrapolation by Jacobi sweeps from the real cells
 *              of each material, upwind along its normal (used in Sec. 2.3.2).
 *   exchange   reduced model: heaviest two materials, HLLC interface state
 *              with the general-EOS wave speeds (Sec. 2.3.2).
 *   fluxes     component-wise WENO5-JS of Lax-Friedrichs split fluxes, scaled
 *              by the apertures (Sec. 3 numerics, Eq. discretized_equ).
 *   time       three-stage TVD Runge-Kutta in the beta_s form of Eq.
 *              local-advection (beta = 0, 3/4, 1/3); CFL time step.
 *   level set  local advection of each phi^r, HJ-WENO5 derivatives, then the
 *              reconstruction operator R (Sec. 2.2).
 *   mixing     conservative exchange of small-volume-fraction cells with
 *              neighbours along the normal after each sub-step (Sec. 2.3.2);
 *              non-physical states mix like small cells and every pair is
 *              scaled so that the weights of a cell sum to at most one.
 *   scale sep. oddball cells, indicator swap and distance re-assignment
 *              (Sec. 2.3.3).
 *   Case II    axisymmetric grid of one dimension (face areas r_f, volumes
 *              r_i h, source p alpha / r of the radial momentum) and a held
 *              free-surface ambient driven by p(t), u* from the two-shock wave
 *              curve of the solved side, |u*| in the CFL bound (Sec. 3.2).
 * The paper prints no values for the ghost-extension and interface-velocity
 * sweeps, the mixing weights and band maintenance (reinitialisation of the
 * non-cut band); the tests pin them through special cases with exact answers
 * (a planar interface: ghost states of their own row; a moving contact: the
 * velocity u in the band, the interface at x0 + u t, phi its distance; a
 * crowded mixing target kept in range) and invariants (conservation,
 * equilibrium, symmetry, convexity), not through general values.
 * Compile with -ffp-contract=off: no fused multiply-add anywhere.
 *
 * Built twice: single-threaded (the tests' oracle), and with -fopenmp for
 * the timed CPU baseline on all host cores. The OpenMP pragmas only split
 * loops whose iterations each write their own cell; shared error flags and
 * counters are updated atomically, maxima are order-free and every sum keeps
 * its serial order, so both builds give the same bits.
 */
#include "msf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define G 4 /* halo layers */

struct orc {
  orc_params p;
  int D, N, NV;
  int S; /* Runge-Kutta stages */
  int n[3], pn[3], off[3];
  long st[3], ncell;
  double h[3], rh[3], rh2[3], ih2[3], farea[3], V, rV, hmin, eps_ss, cap;
  double gm1[ORC_MAXM], gpi[ORC_MAXM];
  /* state */
  double *Q, *Q1, *Q2; /* [N][NV][ncell] */
  double *phi, *phin, *phit;
  uint8_t *chi, *chin, *chit;
  double t, dt;
  /* per step */
  uint8_t *smask, *inB;
  /* per stage geometry */
  uint8_t *xs, *mixed, *cut;
  double *alpha;       /* [N][ncell] */
  double *Alo, *Ahi;   /* [3][N][ncell] */
  /* stage work */
  double *W, *Wt;      /* [N][NV][ncell] primitive */
  uint8_t *fill, *fillt, *isreal; /* [N][ncell] */
  double *Uh;          /* [N][NV][ncell] stencil state, conservative */
  double *X;           /* [N][NV][ncell] exchange flux */
  double *vel, *velt;  /* [3][ncell] */
  uint8_t *vf, *vft;
  double *F;           /* [3][N][NV][ncell], flux through the lower face of a cell */
  double ledger[ORC_MAXM][5];
  long long cnt[ORC_NCOUNT];
  int err;
};

/* ------------------------------------------------------------------ */
/* indexing                                                            */
/* ------------------------------------------------------------------ */
static inline long QI(const orc* o, int m, int v, long c) { return ((long)m * o->NV + v) * o->ncell + c; }
static inline long MI(const orc* o, int m, long c) { return (long)m * o->ncell + c; }
static inline long AI(const orc* o, int d, int m, long c) { return ((long)d * o->N + m) * o->ncell + c; }

static void coords(const orc* o, long c, int* ijk) {
  ijk[0] = (int)(c % o->pn[0]);
  ijk[1] = (int)((c / o->pn[0]) % o->pn[1]);
  ijk[2] = (int)(c / ((long)o->pn[0] * o->pn[1]));
}
static long cell_at(const orc* o, const int* ijk) {
  return ijk[0] + o->st[1] * ijk[1] + o->st[2] * ijk[2];
}
static int in_array(const orc* o, const int* ijk) {
  for (int d = 0; d < 3; d++)
    if (ijk[d] < 0 || ijk[d] >= o->pn[d]) return 0;
  return 1;
}
static int interior(const orc* o, const int* ijk) {
  for (int d = 0; d < o->D; d++)
    if (ijk[d] < o->off[d] || ijk[d] >= o->off[d] + o->n[d]) return 0;
  return 1;
}
static int interior_c(const orc* o, long c) {
  int ijk[3];
  coords(o, c, ijk);
  return interior(o, ijk);
}
static double centre(const orc* o, int d, int idx) {
  return o->p.lo[d] + ((double)(idx - o->off[d]) + 0.5) * o->h[d];
}
static int popc(unsigned x) {
  int k = 0;
  while (x) { k += (int)(x & 1u); x >>= 1; }
  return k;
}
/* sticky error flag and event counters, shared by the cells of a loop */
static void set_err(orc* o, int f) {
#pragma omp atomic
  o->err |= f;
}
static void count(orc* o, int k) {
#pragma omp atomic
  o->cnt[k]++;
}

/* ------------------------------------------------------------------ */
/* EOS (Sec. 2.1, 2.3.2): stiffened gas, or Tait's equation             */
/* ------------------------------------------------------------------ */
/* Tait's equation (Sec. 2.1): p = B (rho / rho0)^gamma - B + p0. Its
 * pressure does not depend on the internal energy; the energy carried with
 * it is that of the stiffened gas with pinf = B - p0 (the gas whose isentrope
 * through (rho0, p0) is Tait's curve), which is what prim_to_cons uses. */
static double tait_pressure(const orc* o, int m, double rho) {
  double B = o->p.tait_B[m];
  return B * pow(rho / o->p.tait_rho0[m], o->p.gamma[m]) - B + o->p.tait_p0[m];
}
/* conservative (rho, rho u_d, rho E) -> primitive (rho, u_d, p) */
static void cons_to_prim(const orc* o, int m, const double* u, double* w) {
  int D = o->D;
  double rho = u[0];
  double vel[3] = {0, 0, 0};
  double q = 0.0;
  for (int d = 0; d < D; d++) vel[d] = u[1 + d] / rho;
  for (int d = 0; d < D; d++) q += vel[d] * vel[d];
  double ke = 0.5 * rho * q;
  w[0] = rho;
  for (int d = 0; d < D; d++) w[1 + d] = vel[d];
  w[D + 1] = o->p.eos_kind[m] == 1 ? tait_pressure(o, m, rho) : o->gm1[m] * (u[D + 1] - ke) - o->gpi[m];
}
static void prim_to_cons(const orc* o, int m, const double* w, double* u) {
  int D = o->D;
  double rho = w[0];
  double q = 0.0;
  for (int d = 0; d < D; d++) q += w[1 + d] * w[1 + d];
  u[0] = rho;
  for (int d = 0; d < D; d++) u[1 + d] = rho * w[1 + d];
  u[D + 1] = (w[D + 1] + o->gpi[m]) / o->gm1[m] + 0.5 * rho * q;
}
/* c^2 = Psi + Upsilon p / rho = gamma (p + pinf) / rho (Sec. 2.3.2) */
static double sound2(const orc* o, int m, double rho, double p) {
  return (o->p.gamma[m] * (p + o->p.pinf[m])) / rho;
}
static double sound(orc* o, int m, double rho, double p) {
  double c2 = sound2(o, m, rho, p);
  if (!(rho > 0.0) || !(c2 > 0.0)) {
    set_err(o, ORC_ENEGATIVE);
    c2 = c2 > 0.0 ? c2 : 0.0;
  }
  return sqrt(c2);
}

/* ------------------------------------------------------------------ */
/* axisymmetric grid and free-surface ambient (Sec. 3, Case II)         */
/* ------------------------------------------------------------------ */
/* A cylindrical grid of one dimension takes x as the radius: the volume of
 * cell i is r_i h and the area of a face r_f (per radian and unit length),
 * so the update of a cell reads L = (A_lo F_lo r_lo - A_hi F_hi r_hi + X) /
 * (r_i h) plus the source p alpha / r_i of the radial momentum (the pressure
 * on the sides of the wedge). Volume fractions stay those of the segment. */
static int cyl(const orc* o) { return o->p.geom == 1; }
static double face_r(const orc* o, int i) { return o->p.lo[0] + (double)(i - o->off[0]) * o->h[0]; }
static double cell_r(const orc* o, int i) { return o->p.lo[0] + ((double)(i - o->off[0]) + 0.5) * o->h[0]; }
/* volume of cell c over the Cartesian cell volume (1 on Cartesian grids) */
static double vfac(const orc* o, long c) { return cyl(o) ? cell_r(o, (int)(c % o->pn[0])) : 1.0; }

/* pressure the ambient exerts at time t: p0 up to t0, linear to p1 at t1, p1 after */
static double fs_pressure(const orc* o, double t) {
  const orc_params* p = &o->p;
  if (t <= p->fs_t0) return p->fs_p0;
  if (t >= p->fs_t1) return p->fs_p1;
  return p->fs_p0 - (p->fs_p0 - p->fs_p1) * (t - p->fs_t0) / (p->fs_t1 - p->fs_t0);
}
/* velocity jump across the wave of a material at (rho, pK) that takes its
 * pressure to p, on the two-shock approximation of the Riemann problem
 * (Toro, Riemann Solvers, Sec. 9.4.2): (p - pK) sqrt(A / (p + pinf + B)),
 * A = 2 / ((g + 1) rho), B = (g - 1) / (g + 1) (pK + pinf) */
static double fs_wave(const orc* o, int m, double rho, double pK, double p) {
  double g = o->p.gamma[m], pi = o->p.pinf[m];
  double A = 2.0 / ((g + 1.0) * rho), B = (g - 1.0) / (g + 1.0) * (pK + pi);
  return (p - pK) * sqrt(A / (p + pi + B));
}
/* the ambient is not solved: its conserved state is alpha (fs_rho, 0, p(t)) */
static void hold_ambient(orc* o, double* Qc, double t) {
  int F = o->p.fs_mat;
  if (F < 0) return;
  double w[5] = {0, 0, 0, 0, 0}, u[5];
  w[0] = o->p.fs_rho;
  w[o->D + 1] = fs_pressure(o, t);
  prim_to_cons(o, F, w, u);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    if (!interior_c(o, c)) continue;
    double a = o->alpha[MI(o, F, c)];
    for (int v = 0; v < o->NV; v++) Qc[QI(o, F, v, c)] = a * u[v];
  }
}

/* ------------------------------------------------------------------ */
/* WENO5-JS (Jiang & Shu), value at i+1/2 from cells i-2..i+2           */
/* ------------------------------------------------------------------ */
double orc_weno5(double a, double b, double c, double d, double e, double eps) {
  double q0 = (2.0 * a - 7.0 * b + 11.0 * c) * (1.0 / 6.0);
  double q1 = (-b + 5.0 * c + 2.0 * d) * (1.0 / 6.0);
  double q2 = (2.0 * c + 5.0 * d - e) * (1.0 / 6.0);
  double t, s0, s1, s2;
  t = a - 2.0 * b + c;
  s0 = 13.0 / 12.0 * t * t;
  t = a - 4.0 * b + 3.0 * c;
  s0 = s0 + 0.25 * t * t;
  t = b - 2.0 * c + d;
  s1 = 13.0 / 12.0 * t * t;
  t = b - d;
  s1 = s1 + 0.25 * t * t;
  t = c - 2.0 * d + e;
  s2 = 13.0 / 12.0 * t * t;
  t = 3.0 * c - 4.0 * d + e;
  s2 = s2 + 0.25 * t * t;
  /* Jiang & Shu's unnormalised weights a_k = d_k / (eps + beta_k)^2 with the
     ideal weights d = (1/10, 6/10, 3/10); the value is sum_k w_k q_k with the
     normalised weights w_k = a_k / sum_j a_j */
  double b0 = eps + s0, b1 = eps + s1, b2 = eps + s2;
  double a0 = 0.1 / (b0 * b0);
  double a1 = 0.6 / (b1 * b1);
  double a2 = 0.3 / (b2 * b2);
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* ------------------------------------------------------------------ */
/* HLLC interface state for two general-EOS states (Sec. 2.3.2)        */
/* w = (rho, u_n, p), eos = (gamma, pinf, kind); c^2 = Psi + Upsilon p/rho:
 * stiffened gas Psi = (p + gamma pinf)/rho, Upsilon = gamma - 1; Tait
 * (pinf = B - p0) Psi = gamma (p + pinf)/rho, Upsilon = 0                 */
/* ------------------------------------------------------------------ */
void orc_hllc(const double* wl, const double* wr, const double* eosl, const double* eosr,
              double* ustar, double* pstar) {
  double rl = wl[0], ul = wl[1], pl = wl[2], gl = eosl[0], pil = eosl[1];
  double rr = wr[0], ur = wr[1], pr = wr[2], gr = eosr[0], pir = eosr[1];
  double c2l = (gl * (pl + pil)) / rl, c2r = (gr * (pr + pir)) / rr;
  double cl = sqrt(c2l > 0.0 ? c2l : 0.0), cr = sqrt(c2r > 0.0 ? c2r : 0.0);
  /* Psi = dp/drho|_e, Upsilon = (1/rho) dp/de|_rho */
  int tl = eosl[2] == 1.0, tr = eosr[2] == 1.0;
  double psil = tl ? (gl * (pl + pil)) / rl : (pl + gl * pil) / rl;
  double psir = tr ? (gr * (pr + pir)) / rr : (pr + gr * pir) / rr;
  double upsl = tl ? 0.0 : gl - 1.0, upsr = tr ? 0.0 : gr - 1.0;
  double sl = sqrt(rl), sr = sqrt(rr);
  double den = sl + sr;
  double psit = (sl * psil + sr * psir) / den;
  double upst = (sl * upsl + sr * upsr) / den;
  double du = (ur - ul) / den;
  double prt = (sl * (pl / rl) + sr * (pr / rr)) / den + 0.5 * (sl * sr) * (du * du);
  double ct2 = psit + upst * prt;
  double ct = sqrt(ct2 > 0.0 ? ct2 : 0.0);
  double ut = (sl * ul + sr * ur) / den;
  double SL = fmin(ul - cl, ut - ct);
  double SR = fmax(ut + ct, ur + cr);
  double ml = (ul - SL) * rl, mr = (SR - ur) * rr;
  double SM = (mr * ur + ml * ul + pl - pr) / (mr + ml);
  double psl = pl + rl * (SL - ul) * (SM - ul);
  double psr = pr + rr * (SR - ur) * (SM - ur);
  *ustar = SM;
  *pstar = 0.5 * (psl + psr);
}

/* ------------------------------------------------------------------ */
/* positive-part fractions of a linear function on a simplex           */
/* ------------------------------------------------------------------ */
static void sort_desc(double* v, int k) {
  for (int i = 1; i < k; i++)
    for (int j = i; j > 0 && v[j] > v[j - 1]; j--) {
      double t = v[j]; v[j] = v[j - 1]; v[j - 1] = t;
    }
}
double orc_seg_frac(double a, double b) {
  int np = (a > 0) + (b > 0), nn = (a < 0) + (b < 0);
  if (nn == 0) return np == 0 ? 0.5 : 1.0;
  if (np == 0) return 0.0;
  double pos = a > 0 ? a : b, neg = a > 0 ? b : a;
  return pos / (pos - neg);
}
double orc_tri_frac(double a, double b, double c) {
  double v[3] = {a, b, c};
  sort_desc(v, 3);
  int np = (v[0] > 0) + (v[1] > 0) + (v[2] > 0);
  int nn = (v[0] < 0) + (v[1] < 0) + (v[2] < 0);
  if (nn == 0) return np == 0 ? 0.5 : 1.0;
  if (np == 0) return 0.0;
  if (np == 1) return (v[0] * v[0]) / ((v[0] - v[1]) * (v[0] - v[2]));
  return 1.0 - (v[2] * v[2]) / ((v[0] - v[2]) * (v[1] - v[2]));
}
double orc_tet_frac(double a, double b, double c, double d) {
  double v[4] = {a, b, c, d};
  sort_desc(v, 4);
  int np = (v[0] > 0) + (v[1] > 0) + (v[2] > 0) + (v[3] > 0);
  int nn = (v[0] < 0) + (v[1] < 0) + (v[2] < 0) + (v[3] < 0);
  if (nn == 0) return np == 0 ? 0.5 : 1.0;
  if (np == 0) return 0.0;
  if (np == 1) return (v[0] * v[0] * v[0]) / (((v[0] - v[1]) * (v[0] - v[2])) * (v[0] - v[3]));
  if (np == 3) {
    double m3 = -v[3];
    return 1.0 - (m3 * m3 * m3) / (((v[0] - v[3]) * (v[1] - v[3])) * (v[2] - v[3]));
  }
  {
    double A = v[0], B = v[1], C = v[2], E = v[3];
    double num = A * A * (B * B) - A * B * (A + B) * (C + E) + C * E * (A * A + A * B + B * B);
    double den = ((A - C) * (A - E)) * ((B - C) * (B - E));
    return num / den;
  }
}

/* ------------------------------------------------------------------ */
/* construction operator C_m (Sec. 2.2) and vertex values              */
/* ------------------------------------------------------------------ */
static double phim(const orc* o, long c, int m) { return o->chi[c] == m ? o->phi[c] : -o->phi[c]; }
static double phim_n(const orc* o, long c, int m) { return o->chin[c] == m ? o->phin[c] : -o->phin[c]; }

/* value at the grid vertex with index (I,J,K): mean of the 2^D cells around it,
   summed in memory order */
static double corner_val(const orc* o, int I, int J, int K, int m) {
  int D = o->D;
  double s = 0.0;
  int kz0 = D >= 3 ? K - 1 : K, kz1 = K;
  int jy0 = D >= 2 ? J - 1 : J, jy1 = J;
  for (int kk = kz0; kk <= kz1; kk++)
    for (int jj = jy0; jj <= jy1; jj++)
      for (int ii = I - 1; ii <= I; ii++) {
        int ijk[3] = {ii, jj, kk};
        s += phim(o, cell_at(o, ijk), m);
      }
  return s * (D == 1 ? 0.5 : (D == 2 ? 0.25 : 0.125));
}
/* 3D face centre between the cell and its neighbour along +e_d or -e_d */
static double facec_val(const orc* o, long c, int d, int side, int m) {
  long a = side ? c : c - o->st[d], b = side ? c + o->st[d] : c;
  return (phim(o, a, m) + phim(o, b, m)) * 0.5;
}

/* volume fraction and apertures of material m in cell c (Sec. 2.3, Fig. 2) */
static void cell_geometry(const orc* o, long c, int m, double* alpha, double* Alo, double* Ahi) {
  int D = o->D, ijk[3];
  coords(o, c, ijk);
  int i = ijk[0], j = ijk[1], k = ijk[2];
  double vc = phim(o, c, m);
  if (D == 1) {
    double c0 = corner_val(o, i, j, k, m), c1 = corner_val(o, i + 1, j, k, m);
    *alpha = (orc_seg_frac(c0, vc) + orc_seg_frac(vc, c1)) * 0.5;
    Alo[0] = c0 > 0 ? 1.0 : (c0 < 0 ? 0.0 : 0.5);
    Ahi[0] = c1 > 0 ? 1.0 : (c1 < 0 ? 0.0 : 0.5);
  } else if (D == 2) {
    double c00 = corner_val(o, i, j, k, m), c10 = corner_val(o, i + 1, j, k, m);
    double c01 = corner_val(o, i, j + 1, k, m), c11 = corner_val(o, i + 1, j + 1, k, m);
    Alo[0] = orc_seg_frac(c00, c01);
    Ahi[0] = orc_seg_frac(c10, c11);
    Alo[1] = orc_seg_frac(c00, c10);
    Ahi[1] = orc_seg_frac(c01, c11);
    *alpha = (orc_tri_frac(vc, c00, c01) + orc_tri_frac(vc, c10, c11) + orc_tri_frac(vc, c00, c10) +
              orc_tri_frac(vc, c01, c11)) * 0.25;
  } else {
    double cv[2][2][2]; /* [z][y][x] */
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int e = 0; e < 2; e++) cv[a][b][e] = corner_val(o, i + e, j + b, k + a, m);
    /* each face: centre value and its 4 corners in cyclic order */
    double fc[6], q[6][4];
    fc[0] = facec_val(o, c, 0, 0, m);
    q[0][0] = cv[0][0][0]; q[0][1] = cv[0][1][0]; q[0][2] = cv[1][1][0]; q[0][3] = cv[1][0][0];
    fc[1] = facec_val(o, c, 0, 1, m);
    q[1][0] = cv[0][0][1]; q[1][1] = cv[0][1][1]; q[1][2] = cv[1][1][1]; q[1][3] = cv[1][0][1];
    fc[2] = facec_val(o, c, 1, 0, m);
    q[2][0] = cv[0][0][0]; q[2][1] = cv[0][0][1]; q[2][2] = cv[1][0][1]; q[2][3] = cv[1][0][0];
    fc[3] = facec_val(o, c, 1, 1, m);
    q[3][0] = cv[0][1][0]; q[3][1] = cv[0][1][1]; q[3][2] = cv[1][1][1]; q[3][3] = cv[1][1][0];
    fc[4] = facec_val(o, c, 2, 0, m);
    q[4][0] = cv[0][0][0]; q[4][1] = cv[0][0][1]; q[4][2] = cv[0][1][1]; q[4][3] = cv[0][1][0];
    fc[5] = facec_val(o, c, 2, 1, m);
    q[5][0] = cv[1][0][0]; q[5][1] = cv[1][0][1]; q[5][2] = cv[1][1][1]; q[5][3] = cv[1][1][0];
    double vol = 0.0;
    for (int f = 0; f < 6; f++) {
      double ap = 0.0;
      for (int e = 0; e < 4; e++) {
        double p0 = q[f][e], p1 = q[f][(e + 1) & 3];
        ap += orc_tri_frac(fc[f], p0, p1);
        vol += orc_tet_frac(vc, fc[f], p0, p1);
      }
      ap = ap * 0.25;
      if (f & 1) Ahi[f >> 1] = ap; else Alo[f >> 1] = ap;
    }
    *alpha = vol * (1.0 / 24.0);
  }
}

/* min and max of phi^m over the simplex vertices of cell c */
static void vertex_minmax(const orc* o, long c, int m, double* mn, double* mx) {
  int D = o->D, ijk[3];
  coords(o, c, ijk);
  double lo = phim(o, c, m), hi = lo;
  int nz = D >= 3 ? 2 : 1, ny = D >= 2 ? 2 : 1;
  for (int a = 0; a < nz; a++)
    for (int b = 0; b < ny; b++)
      for (int e = 0; e < 2; e++) {
        double v = corner_val(o, ijk[0] + e, ijk[1] + b, ijk[2] + a, m);
        lo = fmin(lo, v); hi = fmax(hi, v);
      }
  if (D == 3)
    for (int d = 0; d < 3; d++)
      for (int s = 0; s < 2; s++) {
        double v = facec_val(o, c, d, s, m);
        lo = fmin(lo, v); hi = fmax(hi, v);
      }
  *mn = lo; *mx = hi;
}

/* unit normal n^m = grad phi^m / |grad phi^m|, central differences (Sec. 2.3.2) */
static void normal_m(const orc* o, long c, int m, double* n) {
  double g[3] = {0, 0, 0}, q = 0.0;
  for (int d = 0; d < o->D; d++) g[d] = (phim(o, c + o->st[d], m) - phim(o, c - o->st[d], m)) * o->rh2[d];
  for (int d = 0; d < o->D; d++) q += g[d] * g[d];
  double len = sqrt(q);
  for (int d = 0; d < 3; d++) n[d] = 0.0;
  if (len > 0.0)
    for (int d = 0; d < o->D; d++) n[d] = g[d] / len;
}

/* ------------------------------------------------------------------ */
/* boundary fill of phi, chi (a1)                                        */
/* ------------------------------------------------------------------ */
/* source cell of a halo coordinate along axis d: transmissive and inflow copy
   the nearest interior cell; reflective mirrors about the boundary, repeatedly
   when the halo is deeper than the interior (flip = odd number of mirrors) */
static int bc_src(const orc* o, int d, int idx, int* side, int* flip) {
  int n = o->n[d], off = o->off[d], r = idx - off;
  *side = r < 0 ? 0 : 1;
  *flip = 0;
  if (o->p.bc[d][*side] != 1) return r < 0 ? off : off + n - 1;
  int P = 2 * n, k = ((r % P) + P) % P;
  int count = r < 0 ? (-r - 1) / n + 1 : (r - n) / n + 1;
  *flip = count & 1;
  return off + (k >= n ? P - 1 - k : k);
}
static void bc_phichi(orc* o) {
  for (int d = 0; d < o->D; d++) {
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) {
      int ijk[3], side;
      coords(o, c, ijk);
      int r = ijk[d] - o->off[d];
      if (r >= 0 && r < o->n[d]) continue;
      int ok = 1;
      for (int e = d + 1; e < o->D; e++) /* later axes: interior only, filled by their own pass */
        if (ijk[e] < o->off[e] || ijk[e] >= o->off[e] + o->n[e]) ok = 0;
      if (!ok) continue;
      int src[3] = {ijk[0], ijk[1], ijk[2]}, flip;
      src[d] = bc_src(o, d, ijk[d], &side, &flip);
      long s = cell_at(o, src);
      o->phi[c] = o->phi[s];
      o->chi[c] = o->chi[s];
    }
  }
}

/* ------------------------------------------------------------------ */
/* narrow band of the step (Sec. 2.4: interface operations run only in */
/* the band) and the geometry of one stage                             */
/* ------------------------------------------------------------------ */
static void compute_xs(orc* o) {
  int D = o->D;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    int ijk[3];
    coords(o, c, ijk);
    unsigned bits = 0;
    for (int dz = (D >= 3 ? -1 : 0); dz <= (D >= 3 ? 1 : 0); dz++)
      for (int dy = (D >= 2 ? -1 : 0); dy <= (D >= 2 ? 1 : 0); dy++)
        for (int dx = -1; dx <= 1; dx++) {
          int q[3] = {ijk[0] + dx, ijk[1] + dy, ijk[2] + dz};
          if (!in_array(o, q)) continue;
          bits |= 1u << o->chi[cell_at(o, q)];
        }
    o->xs[c] = (uint8_t)bits;
  }
}
static void step_band(orc* o) {
  int D = o->D;
  const int R = 4;
  compute_xs(o);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    o->smask[c] = 0;
    o->inB[c] = 0;
    if (!interior_c(o, c)) continue;
    int ijk[3];
    coords(o, c, ijk);
    unsigned bits = 0;
    for (int dz = (D >= 3 ? -R : 0); dz <= (D >= 3 ? R : 0); dz++)
      for (int dy = (D >= 2 ? -R : 0); dy <= (D >= 2 ? R : 0); dy++)
        for (int dx = -R; dx <= R; dx++) {
          int q[3] = {ijk[0] + dx, ijk[1] + dy, ijk[2] + dz};
          if (!in_array(o, q)) continue;
          bits |= o->xs[cell_at(o, q)];
        }
    o->smask[c] = (uint8_t)bits;
    o->inB[c] = popc(bits) >= 2;
  }
}

/* geometry + conservation correction of the current (phi, chi), Q = Qs */
static void geometry(orc* o, const double* Qs) {
  /* Qs == NULL: raw volume fractions, no correction */
  int N = o->N, D = o->D;
  compute_xs(o);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    o->mixed[c] = 0;
    if (!interior_c(o, c)) continue;
    for (int m = 0; m < N; m++) {
      o->alpha[MI(o, m, c)] = 0.0;
      for (int d = 0; d < 3; d++) o->Alo[AI(o, d, m, c)] = o->Ahi[AI(o, d, m, c)] = 0.0;
    }
    int mixed = o->inB[c] && popc(o->xs[c]) >= 2;
    if (!mixed) {
      int m = o->chi[c];
      o->alpha[MI(o, m, c)] = 1.0;
      for (int d = 0; d < D; d++) o->Alo[AI(o, d, m, c)] = o->Ahi[AI(o, d, m, c)] = 1.0;
      continue;
    }
    o->mixed[c] = 1;
    for (int m = 0; m < N; m++) {
      if (!((o->xs[c] >> m) & 1u)) continue;
      double a, alo[3] = {0, 0, 0}, ahi[3] = {0, 0, 0};
      cell_geometry(o, c, m, &a, alo, ahi);
      o->alpha[MI(o, m, c)] = a;
      for (int d = 0; d < D; d++) {
        o->Alo[AI(o, d, m, c)] = alo[d];
        o->Ahi[AI(o, d, m, c)] = ahi[d];
      }
    }
    /* the materials partition every face: apertures divided by their sum over
       the local materials (two-material faces already sum to one). Next to a
       junction the averaged vertex values can leave a face on which every
       local field is <= 0; such a face goes to the indicators of the two cells
       that share it (whole when they agree, half each otherwise), so that
       every face is closed and both cells see the same apertures */
    for (int d = 0; d < D; d++)
      for (int side = 0; side < 2; side++) {
        double* A = side ? o->Ahi : o->Alo;
        double s = 0.0;
        for (int m = 0; m < N; m++)
          if ((o->xs[c] >> m) & 1u) s += A[AI(o, d, m, c)];
        if (s > 0.0) {
          for (int m = 0; m < N; m++)
            if ((o->xs[c] >> m) & 1u) A[AI(o, d, m, c)] = A[AI(o, d, m, c)] / s;
        } else {
          int ca = o->chi[side ? c : c - o->st[d]], cb = o->chi[side ? c + o->st[d] : c];
          if (ca == cb) {
            A[AI(o, d, ca, c)] = 1.0;
          } else {
            A[AI(o, d, ca, c)] = 0.5;
            A[AI(o, d, cb, c)] = 0.5;
          }
        }
      }
    /* conservation correction (Sec. 2.3.1, Eq. vol_corr2) */
    int np = 0;
    double sum = 0.0;
    for (int m = 0; m < N; m++)
      if (o->alpha[MI(o, m, c)] > 0.0) { np++; sum += o->alpha[MI(o, m, c)]; }
    if (np >= 3 && Qs) {
      count(o, ORC_C_MULTI);
      double rem = 1.0 - sum;
      if (rem != 0.0) count(o, ORC_C_CORRECTED);
      /* apply to the lightest material (alpha rho = Q_rho); overflow below zero
         moves on to the next lightest */
      uint8_t used = 0;
      while (rem != 0.0) {
        int best = -1;
        for (int m = 0; m < N; m++) {
          if (o->alpha[MI(o, m, c)] > 0.0 && !((used >> m) & 1u)) {
            if (best < 0 || Qs[QI(o, m, 0, c)] < Qs[QI(o, best, 0, c)]) best = m;
          }
        }
        if (best < 0) break;
        used |= (uint8_t)(1u << best);
        double na = o->alpha[MI(o, best, c)] + rem;
        if (na >= 0.0) {
          o->alpha[MI(o, best, c)] = na;
          rem = 0.0;
        } else {
          o->alpha[MI(o, best, c)] = 0.0;
          rem = na;
        }
      }
    }
  }
}


/* material m is present in cell c when its sub-cell is non-empty: positive
   volume fraction or a positive aperture on one of the cell's faces (so a cell
   whose face lies on the interface counts, as in the definition of S_0,
   Sec. 2.3.3) */
static int present(const orc* o, long c, int m) {
  if (o->alpha[MI(o, m, c)] > 0.0) return 1;
  if (!o->mixed[c] || !((o->xs[c] >> m) & 1u)) return 0;
  for (int d = 0; d < o->D; d++)
    if (o->Alo[AI(o, d, m, c)] > 0.0 || o->Ahi[AI(o, d, m, c)] > 0.0) return 1;
  return 0;
}

/* aperture of material m on the face between cL and cR = cL + e_d */
static double face_aperture(const orc* o, long cL, long cR, int d, int m) {
  if (o->mixed[cL]) {
    if ((o->xs[cL] >> m) & 1u) return o->Ahi[AI(o, d, m, cL)];
    return 0.0;
  }
  if (o->mixed[cR]) {
    if ((o->xs[cR] >> m) & 1u) return o->Alo[AI(o, d, m, cR)];
    return 0.0;
  }
  return (o->chi[cL] == m && o->chi[cR] == m) ? 1.0 : 0.0;
}

/* ------------------------------------------------------------------ */
/* primitive recovery + ghost states (a5, a6), stencil state Uhat      */
/* ------------------------------------------------------------------ */
static void prim_extend(orc* o, const double* Qs) {
  int N = o->N, NV = o->NV, D = o->D;
  double nanv = nan("");
  for (int m = 0; m < N; m++) {
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) {
      o->fill[MI(o, m, c)] = 0;
      o->isreal[MI(o, m, c)] = 0;
      if (!o->inB[c] || !((o->smask[c] >> m) & 1u)) continue;
      double a = o->alpha[MI(o, m, c)];
      if (o->chi[c] == m && a > 0.0) {
        double u[5], w[5];
        for (int v = 0; v < NV; v++) u[v] = Qs[QI(o, m, v, c)] / a;
        cons_to_prim(o, m, u, w);
        for (int v = 0; v < NV; v++) o->W[QI(o, m, v, c)] = w[v];
        o->fill[MI(o, m, c)] = 1;
        o->isreal[MI(o, m, c)] = 1;
      }
    }
    for (int sw = 0; sw < o->p.ext_sweeps; sw++) {
#pragma omp parallel for schedule(static)
      for (long c = 0; c < o->ncell; c++) {
        o->fillt[MI(o, m, c)] = o->fill[MI(o, m, c)];
        for (int v = 0; v < NV; v++) o->Wt[QI(o, m, v, c)] = o->W[QI(o, m, v, c)];
      }
#pragma omp parallel for schedule(static)
      for (long c = 0; c < o->ncell; c++) {
        if (!o->inB[c] || !((o->smask[c] >> m) & 1u) || o->isreal[MI(o, m, c)]) continue;
        double n[3];
        normal_m(o, c, m, n);
        double acc[5] = {0, 0, 0, 0, 0}, acc2[5] = {0, 0, 0, 0, 0}, sw_ = 0.0;
        int cnt = 0;
        for (int d = 0; d < D; d++)
          for (int s = 0; s < 2; s++) {
            long j = s ? c + o->st[d] : c - o->st[d];
            if (!interior_c(o, j) || !o->inB[j] || !((o->smask[j] >> m) & 1u) || !o->fillt[MI(o, m, j)]) continue;
            double w = s ? n[d] : -n[d];
            w = w > 0.0 ? w : 0.0;
            for (int v = 0; v < NV; v++) {
              acc[v] += w * o->Wt[QI(o, m, v, j)];
              acc2[v] += o->Wt[QI(o, m, v, j)];
            }
            sw_ += w;
            cnt++;
          }
        if (sw_ > 0.0) {
          for (int v = 0; v < NV; v++) o->W[QI(o, m, v, c)] = acc[v] / sw_;
          o->fill[MI(o, m, c)] = 1;
        } else if (cnt > 0) {
          for (int v = 0; v < NV; v++) o->W[QI(o, m, v, c)] = acc2[v] / (double)cnt;
          o->fill[MI(o, m, c)] = 1;
        }
      }
    }
  }
  /* stencil state of every interior cell */
  for (int m = 0; m < N; m++)
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) {
      if (!interior_c(o, c)) continue;
      double u[5];
      if (!o->inB[c]) {
        if (o->chi[c] == m)
          for (int v = 0; v < NV; v++) u[v] = Qs[QI(o, m, v, c)];
        else
          for (int v = 0; v < NV; v++) u[v] = nanv;
      } else if (!((o->smask[c] >> m) & 1u)) {
        for (int v = 0; v < NV; v++) u[v] = nanv;
      } else if (o->isreal[MI(o, m, c)]) {
        double a = o->alpha[MI(o, m, c)];
        for (int v = 0; v < NV; v++) u[v] = Qs[QI(o, m, v, c)] / a;
      } else if (o->fill[MI(o, m, c)]) {
        double w[5];
        for (int v = 0; v < NV; v++) w[v] = o->W[QI(o, m, v, c)];
        prim_to_cons(o, m, w, u);
      } else {
        for (int v = 0; v < NV; v++) u[v] = nanv;
      }
      for (int v = 0; v < NV; v++) o->Uh[QI(o, m, v, c)] = u[v];
    }
  (void)D;
}

/* boundary fill of the stencil state (a1); halo cells along one axis only */
static void bc_uhat(orc* o) {
  int N = o->N, NV = o->NV, D = o->D;
  for (int d = 0; d < D; d++)
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) {
      int ijk[3], side;
      coords(o, c, ijk);
      int r = ijk[d] - o->off[d];
      if (r >= 0 && r < o->n[d]) continue;
      if (r < -G || r >= o->n[d] + G) continue;
      int ok = 1;
      for (int e = 0; e < D; e++)
        if (e != d && (ijk[e] < o->off[e] || ijk[e] >= o->off[e] + o->n[e])) ok = 0;
      if (!ok) continue;
      int src[3] = {ijk[0], ijk[1], ijk[2]}, flip;
      src[d] = bc_src(o, d, ijk[d], &side, &flip);
      long s = cell_at(o, src);
      int type = o->p.bc[d][side];
      for (int m = 0; m < N; m++) {
        double u[5];
        if (type == 2 && m == o->p.inflow_mat[d][side]) {
          prim_to_cons(o, m, o->p.inflow_prim[d][side], u);
        } else {
          for (int v = 0; v < NV; v++) u[v] = o->Uh[QI(o, m, v, s)];
          if (flip) u[1 + d] = -u[1 + d];
        }
        for (int v = 0; v < NV; v++) o->Uh[QI(o, m, v, c)] = u[v];
      }
    }
}

/* ------------------------------------------------------------------ */
/* CFL time step (a2)                                                   */
/* ------------------------------------------------------------------ */
static void compute_dt(orc* o, double t_end) {
  int N = o->N, D = o->D;
  double lam = 0.0;
#pragma omp parallel for schedule(static) reduction(max : lam)
  for (long c = 0; c < o->ncell; c++) {
    if (!interior_c(o, c)) continue;
    for (int m = 0; m < N; m++) {
      if (!(o->alpha[MI(o, m, c)] > 0.0) || m == o->p.fs_mat) continue;
      double u[5], w[5];
      for (int v = 0; v < o->NV; v++) u[v] = o->Uh[QI(o, m, v, c)];
      cons_to_prim(o, m, u, w);
      double cs = sound(o, m, w[0], w[D + 1]);
      double s = 0.0;
      for (int d = 0; d < D; d++) s += (fabs(w[1 + d]) + cs) * o->rh[d];
      if (s > lam) lam = s;
    }
  }
  /* a free surface moves at the u* of its wave curve, which the material
     states do not bound: its cut cells enter the bound with |u*| */
  if (o->p.fs_mat >= 0)
#pragma omp parallel for schedule(static) reduction(max : lam)
    for (long c = 0; c < o->ncell; c++) {
      if (!o->cut[c] || !(o->alpha[MI(o, o->p.fs_mat, c)] > 0.0)) continue;
      double s = 0.0;
      for (int d = 0; d < D; d++) s += fabs(o->vel[d * o->ncell + c]) * o->rh[d];
      if (s > lam) lam = s;
    }
  double dt = o->p.cfl / lam;
  if (o->t + dt >= t_end) dt = t_end - o->t;
  o->dt = dt;
}

/* ------------------------------------------------------------------ */
/* reduced interface interaction (a7, Sec. 2.3.2)                       */
/* ------------------------------------------------------------------ */
static void interface_exchange(orc* o, const double* Qs, double ts) {
  int N = o->N, NV = o->NV, D = o->D;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < (long)N * NV * o->ncell; i++) o->X[i] = 0.0;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    o->cut[c] = 0;
    for (int d = 0; d < 3; d++) o->vel[d * o->ncell + c] = 0.0;
    if (!o->mixed[c]) continue;
    int np = 0;
    for (int m = 0; m < N; m++)
      if (present(o, c, m)) np++;
    if (np < 2) continue;
    o->cut[c] = 1;
    count(o, ORC_C_CUT);
    /* the heaviest two present materials by alpha rho */
    int eta = -1, xi = -1;
    for (int m = 0; m < N; m++)
      if (present(o, c, m) && (eta < 0 || Qs[QI(o, m, 0, c)] > Qs[QI(o, eta, 0, c)])) eta = m;
    for (int m = 0; m < N; m++)
      if (m != eta && present(o, c, m) && (xi < 0 || Qs[QI(o, m, 0, c)] > Qs[QI(o, xi, 0, c)])) xi = m;
    int L, R;
    if (Qs[QI(o, xi, 0, c)] < Qs[QI(o, eta, 0, c)]) { L = xi; R = eta; }
    else { L = eta; R = xi; }
    double n[3];
    normal_m(o, c, R, n); /* normal of the heavier material, pointing into it */
    double uL[5], uR[5], wL[5], wR[5];
    for (int v = 0; v < NV; v++) { uL[v] = o->Uh[QI(o, L, v, c)]; uR[v] = o->Uh[QI(o, R, v, c)]; }
    if (isnan(uL[0]) || isnan(uR[0])) { set_err(o, ORC_EBAND); continue; }
    cons_to_prim(o, L, uL, wL);
    cons_to_prim(o, R, uR, wR);
    double unl = 0.0, unr = 0.0;
    for (int d = 0; d < D; d++) { unl += wL[1 + d] * n[d]; unr += wR[1 + d] * n[d]; }
    double rl[3] = {wL[0], unl, wL[D + 1]}, rr[3] = {wR[0], unr, wR[D + 1]};
    double el[3] = {o->p.gamma[L], o->p.pinf[L], (double)o->p.eos_kind[L]};
    double er[3] = {o->p.gamma[R], o->p.pinf[R], (double)o->p.eos_kind[R]};
    double us, ps;
    const int F = o->p.fs_mat;
    if (F >= 0 && (L == F || R == F)) {
      /* free surface: the ambient imposes p* = p(t); the solved side's
         two-shock wave curve gives u* */
      ps = fs_pressure(o, ts);
      if (R == F) {
        (void)sound(o, L, wL[0], wL[D + 1]);
        us = unl - fs_wave(o, L, wL[0], wL[D + 1], ps);
      } else {
        (void)sound(o, R, wR[0], wR[D + 1]);
        us = unr + fs_wave(o, R, wR[0], wR[D + 1], ps);
      }
    } else {
      orc_hllc(rl, rr, el, er, &us, &ps);
    }
    /* the pair's interface state acts on the boundary segment of every other
       present material, S^m = sum_f A^m_f |f| n_f^out (pointing into m);
       material R takes minus their sum, so sum_m X^m = 0 exactly and with
       two materials X^R = -X^L as in the reduced model. For comparison,
       literal_reduced lets only the pair exchange (X^R from S^R, X^L = -X^R,
       the other materials nothing), and literal_normal uses |S^m| n^m. */
    double XR[5] = {0, 0, 0, 0, 0};
    const int lit = o->p.literal_reduced;
    for (int m = 0; m < N; m++) {
      if (lit ? m != R : (m == R || !present(o, c, m))) continue;
      double S[3] = {0, 0, 0}, nS = 0.0;
      if (cyl(o)) {
        /* interface area r_I n: the faces' r_f A_f less the wedge side alpha h */
        int ic = (int)(c % o->pn[0]);
        S[0] = o->Ahi[AI(o, 0, m, c)] * face_r(o, ic + 1) - o->Alo[AI(o, 0, m, c)] * face_r(o, ic) -
               o->alpha[MI(o, m, c)] * o->h[0];
      } else {
        for (int d = 0; d < D; d++) S[d] = (o->Ahi[AI(o, d, m, c)] - o->Alo[AI(o, d, m, c)]) * o->farea[d];
      }
      if (o->p.literal_normal) {
        double nm[3], len = 0.0;
        normal_m(o, c, m, nm);
        for (int d = 0; d < D; d++) len += S[d] * S[d];
        len = sqrt(len);
        for (int d = 0; d < D; d++) S[d] = len * nm[d];
      }
      for (int d = 0; d < D; d++) nS += n[d] * S[d];
      for (int d = 0; d < D; d++) {
        o->X[QI(o, m, 1 + d, c)] = ps * S[d];
        XR[1 + d] -= ps * S[d];
      }
      o->X[QI(o, m, D + 1, c)] = ps * us * nS;
      XR[D + 1] -= ps * us * nS;
    }
    if (lit)
      for (int v = 1; v < NV; v++) o->X[QI(o, L, v, c)] = XR[v];
    else
      for (int v = 1; v < NV; v++) o->X[QI(o, R, v, c)] = XR[v];
    for (int d = 0; d < D; d++) o->vel[d * o->ncell + c] = us * n[d];
  }
}

/* interface velocity extended into the band (used by Eq. local-advection) */
static void extend_velocity(orc* o) {
  int D = o->D;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) o->vf[c] = o->cut[c];
  for (int sw = 0; sw < o->p.vel_sweeps; sw++) {
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) {
      o->vft[c] = o->vf[c];
      for (int d = 0; d < 3; d++) o->velt[d * o->ncell + c] = o->vel[d * o->ncell + c];
    }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) {
      if (!o->inB[c] || o->cut[c]) continue;
      double acc[3] = {0, 0, 0}, acc2[3] = {0, 0, 0};
      int cnt = 0, cnt2 = 0;
      for (int d = 0; d < D; d++)
        for (int s = 0; s < 2; s++) {
          long j = s ? c + o->st[d] : c - o->st[d];
          if (!interior_c(o, j) || !o->inB[j] || !o->vft[j]) continue;
          for (int e = 0; e < D; e++) acc2[e] += o->velt[e * o->ncell + j];
          cnt2++;
          if (o->phi[j] < o->phi[c]) {
            for (int e = 0; e < D; e++) acc[e] += o->velt[e * o->ncell + j];
            cnt++;
          }
        }
      if (cnt > 0) {
        for (int e = 0; e < D; e++) o->vel[e * o->ncell + c] = acc[e] / (double)cnt;
        o->vf[c] = 1;
      } else if (cnt2 > 0) {
        for (int e = 0; e < D; e++) o->vel[e * o->ncell + c] = acc2[e] / (double)cnt2;
        o->vf[c] = 1;
      }
    }
  }
}

/* ------------------------------------------------------------------ */
/* fluxes and the RK stage update (a8, Eq. discretized_equ)            */
/* ------------------------------------------------------------------ */
/* Shu-Osher TVD Runge-Kutta in the beta form of Eq. local-advection:
 * Q^(s+1) = beta_s Q^n + (1 - beta_s) (Q^(s) + dt L(Q^(s))). The ledger weight
 * of stage s is the coefficient of dt L(Q^(s)) in Q^{n+1}. Three stages
 * (beta = 0, 3/4, 1/3) or the paper's two (beta = 0, 1/2). */
static const double BETA3[3] = {0.0, 0.75, 1.0 / 3.0};
static const double LEDGER_W3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
static const double BETA2[2] = {0.0, 0.5};
static const double LEDGER_W2[2] = {0.5, 0.5};
static double rk_beta(const orc* o, int s) { return o->S == 2 ? BETA2[s] : BETA3[s]; }
static double rk_ledger_w(const orc* o, int s) { return o->S == 2 ? LEDGER_W2[s] : LEDGER_W3[s]; }
/* time of stage s as a fraction of the step (s = S: the step's end) */
static const double RKC3[4] = {0.0, 1.0, 0.5, 1.0};
static const double RKC2[3] = {0.0, 1.0, 1.0};
static double rk_c(const orc* o, int s) { return o->S == 2 ? RKC2[s] : RKC3[s]; }

/* Positivity-preserving limiting of one face flux (Hu, Adams & Shu, J.
 * Comput. Phys. 242, 2013), a reading added for long runs (the paper has no
 * positivity treatment). The update of the two cells sharing the face is a
 * convex combination of half states u_L - lam F and u_R + lam F with
 * lam = 2 D dt / h_d; the first-order Lax-Friedrichs flux
 * F_LF = (F(u_L) + F(u_R) - a (u_R - u_L)) / 2 (a the stencil's wave-speed
 * maximum) keeps them physical under the CFL bound. The high-order flux F is
 * replaced by F_LF + theta (F - F_LF) with the largest theta in [0, 1] for
 * which the half states keep rho and p + pinf at or above
 * eps = min(1e-13, the values of the Lax-Friedrichs half states): first the
 * density (linear in theta), then p + pinf along the segment from the
 * Lax-Friedrichs half state to the density-limited one (p is concave in the
 * conserved variables, so the linear bound is safe). Tait materials take
 * the density step only (their p + pinf is positive with rho). A flux whose
 * half states need no limiting is kept bit for bit. */
static void pp_limit(const orc* o, int m, int d, const double* uL, const double* uR, const double* FL,
                     const double* FR, double a, double* Fh) {
  const int D = o->D, NV = o->NV;
  const double lam = ((2.0 * D) * o->dt) * o->rh[d];
  double Flf[5], hl[2][5], hh[2][5];
  for (int v = 0; v < NV; v++) Flf[v] = 0.5 * ((FL[v] + FR[v]) - a * (uR[v] - uL[v]));
  for (int v = 0; v < NV; v++) {
    hl[0][v] = uL[v] - lam * Flf[v];
    hl[1][v] = uR[v] + lam * Flf[v];
    hh[0][v] = uL[v] - lam * Fh[v];
    hh[1][v] = uR[v] + lam * Fh[v];
  }
  /* density */
  double eps = fmin(1e-13, fmin(hl[0][0], hl[1][0]));
  double th = 1.0;
  for (int s = 0; s < 2; s++)
    if (hh[s][0] < eps) th = fmin(th, (hl[s][0] - eps) / (hl[s][0] - hh[s][0]));
  /* a flux that needs no limiting is kept as it is */
  double F1[5];
  for (int v = 0; v < NV; v++) F1[v] = th < 1.0 ? Flf[v] + th * (Fh[v] - Flf[v]) : Fh[v];
  if (o->p.eos_kind[m] != 1) {
    /* p + pinf = (gamma - 1)(E - |rho u|^2 / (2 rho)) - gamma pinf + pinf */
    double ql[2], q1[2];
    for (int s = 0; s < 2; s++) {
      const double* u = s ? uR : uL;
      const double sg = s ? 1.0 : -1.0;
      double h1[5];
      for (int v = 0; v < NV; v++) h1[v] = u[v] + sg * (lam * F1[v]);
      double kl = 0.0, k1 = 0.0;
      for (int e = 0; e < D; e++) {
        kl += hl[s][1 + e] * hl[s][1 + e];
        k1 += h1[1 + e] * h1[1 + e];
      }
      ql[s] = (o->gm1[m] * (hl[s][D + 1] - 0.5 * kl / hl[s][0]) - o->gpi[m]) + o->p.pinf[m];
      q1[s] = (o->gm1[m] * (h1[D + 1] - 0.5 * k1 / h1[0]) - o->gpi[m]) + o->p.pinf[m];
    }
    double epq = fmin(1e-13, fmin(ql[0], ql[1]));
    double tp = 1.0;
    for (int s = 0; s < 2; s++)
      if (q1[s] < epq) tp = fmin(tp, (ql[s] - epq) / (ql[s] - q1[s]));
    if (tp < 1.0)
      for (int v = 0; v < NV; v++) F1[v] = Flf[v] + tp * (F1[v] - Flf[v]);
  }
  for (int v = 0; v < NV; v++) Fh[v] = F1[v];
}

static void face_flux(orc* o, long cL, int d, int m, double* Fh) {
  int NV = o->NV, D = o->D;
  long s = o->st[d];
  double U[6][5], Fd[6][5], a = 0.0;
  for (int q = 0; q < 6; q++) {
    long k = cL + (q - 2) * s;
    double w[5];
    for (int v = 0; v < NV; v++) U[q][v] = o->Uh[QI(o, m, v, k)];
    if (isnan(U[q][0])) {
      set_err(o, ORC_EBAND);
      for (int v = 0; v < NV; v++) Fh[v] = 0.0;
      return;
    }
    cons_to_prim(o, m, U[q], w);
    double cs = sound(o, m, w[0], w[D + 1]);
    double p = w[D + 1], un = w[1 + d];
    Fd[q][0] = U[q][1 + d];
    for (int e = 0; e < D; e++) Fd[q][1 + e] = e == d ? U[q][1 + e] * un + p : U[q][1 + e] * un;
    Fd[q][D + 1] = un * (U[q][D + 1] + p);
    double sp = fabs(un) + cs;
    if (sp > a) a = sp;
  }
  double eps = o->p.weno_eps;
  for (int v = 0; v < NV; v++) {
    double fp[6], fm[6];
    for (int q = 0; q < 6; q++) {
      fp[q] = 0.5 * (Fd[q][v] + a * U[q][v]);
      fm[q] = 0.5 * (Fd[q][v] - a * U[q][v]);
    }
    Fh[v] = orc_weno5(fp[0], fp[1], fp[2], fp[3], fp[4], eps) + orc_weno5(fm[5], fm[4], fm[3], fm[2], fm[1], eps);
  }
  if (o->p.positivity) pp_limit(o, m, d, U[2], U[3], Fd[2], Fd[3], a, Fh);
}

static void flux_update(orc* o, int s, const double* Qs, double* Qout) {
  int N = o->N, NV = o->NV, D = o->D;
  double Fb[ORC_MAXM][5];
  memset(Fb, 0, sizeof(Fb));
  /* face fluxes: lower face of every cell with interior index 0..n_d along d */
  for (int d = 0; d < D; d++) {
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) {
      int ijk[3];
      coords(o, c, ijk);
      int r = ijk[d] - o->off[d];
      if (r < 0 || r > o->n[d]) continue;
      int ok = 1;
      for (int e = 0; e < D; e++)
        if (e != d && (ijk[e] < o->off[e] || ijk[e] >= o->off[e] + o->n[e])) ok = 0;
      if (!ok) continue;
      long cL = c - o->st[d];
      for (int m = 0; m < N; m++) {
        double Fh[5] = {0, 0, 0, 0, 0};
        double A = face_aperture(o, cL, c, d, m);
        if (A > 0.0 && m != o->p.fs_mat) {
          int lin = interior_c(o, cL), rin = interior_c(o, c);
          if ((lin && !((o->smask[cL] >> m) & 1u)) || (rin && !((o->smask[c] >> m) & 1u))) set_err(o, ORC_EBAND);
          face_flux(o, cL, d, m, Fh);
        }
        for (int v = 0; v < NV; v++) o->F[((long)(d * N + m) * NV + v) * o->ncell + c] = Fh[v];
      }
    }
  }
  /* boundary ledger: net inflow through the domain boundary faces, summed in
     face order */
  for (int d = 0; d < D; d++)
    for (long c = 0; c < o->ncell; c++) {
      int ijk[3];
      coords(o, c, ijk);
      int r = ijk[d] - o->off[d];
      if (r != 0 && r != o->n[d]) continue;
      int ok = 1;
      for (int e = 0; e < D; e++)
        if (e != d && (ijk[e] < o->off[e] || ijk[e] >= o->off[e] + o->n[e])) ok = 0;
      if (!ok) continue;
      long cL = c - o->st[d];
      for (int m = 0; m < N; m++) {
        double A = face_aperture(o, cL, c, d, m);
        double fa = cyl(o) ? face_r(o, ijk[0]) : o->farea[d];
        for (int v = 0; v < NV; v++) {
          double Fh = o->F[((long)(d * N + m) * NV + v) * o->ncell + c];
          if (r == 0) Fb[m][v] += A * Fh * fa;
          if (r == o->n[d]) Fb[m][v] -= A * Fh * fa;
        }
      }
    }
  double beta = rk_beta(o, s), omb = 1.0 - rk_beta(o, s), dt = o->dt;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    if (!interior_c(o, c)) continue;
    for (int m = 0; m < N; m++) {
      if (!((o->smask[c] >> m) & 1u)) continue;
      double Alo[3], Ahi[3];
      for (int d = 0; d < D; d++) {
        Alo[d] = face_aperture(o, c - o->st[d], c, d, m);
        Ahi[d] = face_aperture(o, c, c + o->st[d], d, m);
      }
      double rlo = 0.0, rhi = 0.0, rvc = 0.0, psrc = 0.0;
      if (cyl(o)) {
        int ic = (int)(c % o->pn[0]);
        double rc = cell_r(o, ic), a = o->alpha[MI(o, m, c)];
        rlo = face_r(o, ic);
        rhi = face_r(o, ic + 1);
        rvc = 1.0 / (rc * o->h[0]);
        if (a > 0.0) {
          double u[5], w[5];
          for (int v = 0; v < NV; v++) u[v] = o->Uh[QI(o, m, v, c)];
          cons_to_prim(o, m, u, w);
          psrc = w[D + 1] * a / rc;
        }
      }
      for (int v = 0; v < NV; v++) {
        double L = 0.0;
        if (cyl(o)) {
          double flo = o->F[((long)m * NV + v) * o->ncell + c];
          double fhi = o->F[((long)m * NV + v) * o->ncell + c + 1];
          L = (Alo[0] * flo * rlo - Ahi[0] * fhi * rhi) * rvc + o->X[QI(o, m, v, c)] * rvc;
          if (v == 1) L = L + psrc;
        } else {
          for (int d = 0; d < D; d++) {
            double flo = o->F[((long)(d * N + m) * NV + v) * o->ncell + c];
            double fhi = o->F[((long)(d * N + m) * NV + v) * o->ncell + c + o->st[d]];
            L = L + (Alo[d] * flo - Ahi[d] * fhi) * o->rh[d];
          }
          L = L + o->X[QI(o, m, v, c)] * o->rV;
        }
        if (m == o->p.fs_mat) L = 0.0;
        double qn = o->Q[QI(o, m, v, c)], qs = Qs[QI(o, m, v, c)];
        double q = beta * qn + omb * (qs + dt * L);
        if (!isfinite(q)) set_err(o, ORC_ENONFINITE);
        Qout[QI(o, m, v, c)] = q;
      }
    }
  }
  for (int m = 0; m < N; m++)
    for (int v = 0; v < NV; v++) o->ledger[m][v] += rk_ledger_w(o, s) * dt * Fb[m][v];
}

/* ------------------------------------------------------------------ */
/* level-set stage and reconstruction (a9, Eqs. construction,          */
/* local-advection, reconstruction)                                    */
/* ------------------------------------------------------------------ */
static double phir_at(const orc* o, long c, int r) { return phim(o, c, r); }

static void levelset_stage(orc* o, int s) {
  int N = o->N, D = o->D;
  double beta = rk_beta(o, s), omb = 1.0 - rk_beta(o, s), dt = o->dt, eps = o->p.weno_eps;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    o->phit[c] = o->phi[c];
    o->chit[c] = o->chi[c];
  }
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    if (!o->inB[c]) continue;
    double best = 0.0;
    int arg = -1;
    for (int r = 0; r < N; r++) {
      if (!((o->xs[c] >> r) & 1u)) continue;
      double adv = 0.0;
      for (int d = 0; d < D; d++) {
        double vd = o->vel[d * o->ncell + c];
        if (vd == 0.0) continue;
        long st = o->st[d];
        double g;
        double rh = o->rh[d];
        if (vd > 0.0) {
          double v1 = (phir_at(o, c - 2 * st, r) - phir_at(o, c - 3 * st, r)) * rh;
          double v2 = (phir_at(o, c - st, r) - phir_at(o, c - 2 * st, r)) * rh;
          double v3 = (phir_at(o, c, r) - phir_at(o, c - st, r)) * rh;
          double v4 = (phir_at(o, c + st, r) - phir_at(o, c, r)) * rh;
          double v5 = (phir_at(o, c + 2 * st, r) - phir_at(o, c + st, r)) * rh;
          g = orc_weno5(v1, v2, v3, v4, v5, eps);
        } else {
          double v1 = (phir_at(o, c + 3 * st, r) - phir_at(o, c + 2 * st, r)) * rh;
          double v2 = (phir_at(o, c + 2 * st, r) - phir_at(o, c + st, r)) * rh;
          double v3 = (phir_at(o, c + st, r) - phir_at(o, c, r)) * rh;
          double v4 = (phir_at(o, c, r) - phir_at(o, c - st, r)) * rh;
          double v5 = (phir_at(o, c - st, r) - phir_at(o, c - 2 * st, r)) * rh;
          g = orc_weno5(v1, v2, v3, v4, v5, eps);
        }
        adv = adv + vd * g;
      }
      double val = beta * phim_n(o, c, r) + omb * (phir_at(o, c, r) - dt * adv);
      if (arg < 0 || val > best) { best = val; arg = r; }
    }
    double ph = fabs(best);
    if (ph > o->cap) ph = o->cap;
    o->phit[c] = ph;
    o->chit[c] = (uint8_t)arg;
  }
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    o->phi[c] = o->phit[c];
    o->chi[c] = o->chit[c];
  }
}

/* ------------------------------------------------------------------ */
/* mixing of small cells (a11, Sec. 2.3.2)                              */
/* ------------------------------------------------------------------ */
/* mixing targets, as sets of axes (bit d = axis d): 1D x; 2D x, y, xy;
   3D x, y, z, xy, xz, yz, xyz */
static const int MIX_NK[4] = {0, 1, 3, 7};
static const int MIX_AX2[3] = {1, 2, 3};
static const int MIX_AX3[7] = {1, 2, 4, 3, 5, 6, 7};

#define MIX_MAXT 26
typedef struct {
  int small, ntarget;
  long tgt[MIX_MAXT];
  double M[MIX_MAXT][5];
  double ws[MIX_MAXT], wt[MIX_MAXT]; /* weight of the partner in the small cell's / the target's mixed state */
} mixrec;

static int mix_axes(int D, int kidx) { return D <= 2 ? MIX_AX2[kidx] : MIX_AX3[kidx]; }

static void mix_source(const orc* o, const double* Qc, long c, int m, mixrec* r, int* fail, int* merge) {
  int D = o->D, NV = o->NV;
  r->small = 0;
  r->ntarget = 0;
  *fail = 0;
  *merge = 0;
  double as = o->alpha[MI(o, m, c)];
  int small = 0;
  if (as > 0.0 && as < o->p.mix_alpha) small = 1;
  if (as == 0.0)
    for (int v = 0; v < NV; v++)
      if (Qc[QI(o, m, v, c)] != 0.0) small = 1;
  /* a non-physical state (rho <= 0 or p + pinf <= 0) mixes like a small cell */
  if (as > 0.0 && !small) {
    double u[5], w[5];
    for (int v = 0; v < NV; v++) u[v] = Qc[QI(o, m, v, c)] / as;
    cons_to_prim(o, m, u, w);
    if (!(w[0] > 0.0) || !(w[NV - 1] + o->p.pinf[m] > 0.0)) small = 1;
  }
  if (!small) return;
  r->small = 1;
  double n[3];
  normal_m(o, c, m, n);
  int sg[3];
  for (int d = 0; d < 3; d++) sg[d] = n[d] > 0.0 ? 1 : (n[d] < 0.0 ? -1 : 0);
  double w[7];
  long t[7];
  int ok[7];
  double sw = 0.0;
  int nk = MIX_NK[D];
  for (int k = 0; k < nk; k++) {
    int ax = mix_axes(D, k);
    ok[k] = 1;
    double wk = 1.0;
    int na = 0;
    long tc = c;
    for (int d = 0; d < D; d++)
      if ((ax >> d) & 1) {
        if (sg[d] == 0) ok[k] = 0;
        tc += sg[d] * o->st[d];
        wk = na == 0 ? fabs(n[d]) : wk * fabs(n[d]);
        na++;
      }
    if (na == 1) wk = wk * wk;
    w[k] = wk;
    t[k] = tc;
    if (!ok[k]) continue;
    if (!interior_c(o, tc) || !o->inB[tc] || !((o->smask[tc] >> m) & 1u) ||
        !(o->alpha[MI(o, m, tc)] > as))
      ok[k] = 0;
    if (ok[k]) sw += w[k];
  }
  long tlist[MIX_MAXT];
  double wlist[MIX_MAXT];
  int nt = 0;
  for (int k = 0; k < nk; k++)
    if (ok[k]) { tlist[nt] = t[k]; wlist[nt] = w[k]; nt++; }
  if (!(sw > 0.0)) {
    /* no neighbour along the normal: any neighbour of the 3^d block with a
       larger volume fraction, weighted by its volume fraction */
    int ijk[3];
    coords(o, c, ijk);
    nt = 0;
    sw = 0.0;
    for (int dz = (D >= 3 ? -1 : 0); dz <= (D >= 3 ? 1 : 0); dz++)
      for (int dy = (D >= 2 ? -1 : 0); dy <= (D >= 2 ? 1 : 0); dy++)
        for (int dx = -1; dx <= 1; dx++) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          int q[3] = {ijk[0] + dx, ijk[1] + dy, ijk[2] + dz};
          if (!interior(o, q)) continue;
          long tc = cell_at(o, q);
          if (!o->inB[tc] || !((o->smask[tc] >> m) & 1u) || !(o->alpha[MI(o, m, tc)] > as)) continue;
          tlist[nt] = tc;
          wlist[nt] = o->alpha[MI(o, m, tc)];
          sw += wlist[nt];
          nt++;
        }
  }
  if (!(sw > 0.0)) {
    *fail = 1;
    if (as == 0.0) *merge = 1;
    return;
  }
  /* with cell volumes V (r h on a cylindrical grid) the pair moves the content
     C = beta V_s V_t (a_s Q_t - a_t Q_s) / (a_s V_s + a_t V_t): M below is
     C / (V_s V_t); the small cell gains M V_t, the target loses M V_s */
  const double vs = vfac(o, c);
  for (int k = 0; k < nt; k++) {
    double beta = wlist[k] / sw;
    double at = o->alpha[MI(o, m, tlist[k])], vt = vfac(o, tlist[k]);
    int q = r->ntarget++;
    r->tgt[q] = tlist[k];
    for (int v = 0; v < NV; v++)
      r->M[q][v] = beta * (as * Qc[QI(o, m, v, tlist[k])] - at * Qc[QI(o, m, v, c)]) / (as * vs + at * vt);
    r->ws[q] = beta * (at * vt) / (as * vs + at * vt);
    r->wt[q] = beta * (as * vs) / (as * vs + at * vt);
  }
}

/* scale of a pair exchange from the weight sums of its two cells */
static double mix_limit(double Ts, double Tt) {
  double f = 1.0;
  if (Ts > 1.0) f = fmin(f, 1.0 / Ts);
  if (Tt > 1.0) f = fmin(f, 1.0 / Tt);
  return f;
}

static void mixing(orc* o, double* Qc) {
  int N = o->N, NV = o->NV, D = o->D;
  long nc = o->ncell;
  mixrec* rec = (mixrec*)calloc((size_t)N * nc, sizeof(mixrec));
  uint8_t* mergef = (uint8_t*)calloc((size_t)N * nc, 1);
  for (int m = 0; m < N; m++)
#pragma omp parallel for schedule(static)
    for (long c = 0; c < nc; c++) {
      if (!o->inB[c] || !((o->smask[c] >> m) & 1u)) continue;
      int fail, merge;
      mix_source(o, Qc, c, m, &rec[MI(o, m, c)], &fail, &merge);
      if (rec[MI(o, m, c)].small) count(o, ORC_C_SMALL);
      if (fail) count(o, ORC_C_MIXFAIL);
      if (merge && m != o->chi[c]) mergef[MI(o, m, c)] = 1;
    }
  /* Weight limit (a reading of the mixing of Sec. 2.3.2): a pair exchange
   * M = beta (a_s Q_t - a_t Q_s) / (a_s + a_t) moves the per-volume state of
   * each side towards the other's with weight w (w_s = beta a_t / (a_s + a_t)
   * for the small cell, w_t = beta a_s / (a_s + a_t) for the target). A cell
   * in several pairs takes the sum T of its weights; when T > 1 its mixed state
   * would extrapolate, so each pair's exchange is scaled by
   * min(1, 1/T_s, 1/T_t): every mixed state is then a convex combination of
   * the pre-mixing states around it, and the exchanges stay antisymmetric
   * (conservative). T sums the cell's own pairs in target order, then the
   * pairs of the neighbours that target it in (z, y, x) offset order. A small
   * cell without volume (a_s = 0) has no per-volume state to keep convex and
   * adds nothing to its target's T (w_t = 0): its exchanges stay whole, so
   * its content always leaves. */
  double* Tw = (double*)calloc((size_t)N * nc, sizeof(double));
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; c++) {
    if (!o->inB[c]) continue;
    int ijk[3];
    coords(o, c, ijk);
    for (int m = 0; m < N; m++) {
      if (!((o->smask[c] >> m) & 1u)) continue;
      double T = 0.0;
      const mixrec* own = &rec[MI(o, m, c)];
      for (int q = 0; q < own->ntarget; q++) T += own->ws[q];
      for (int dz = (D >= 3 ? -1 : 0); dz <= (D >= 3 ? 1 : 0); dz++)
        for (int dy = (D >= 2 ? -1 : 0); dy <= (D >= 2 ? 1 : 0); dy++)
          for (int dx = -1; dx <= 1; dx++) {
            if (dx == 0 && dy == 0 && dz == 0) continue;
            int sq[3] = {ijk[0] - dx, ijk[1] - dy, ijk[2] - dz};
            if (!in_array(o, sq)) continue;
            const mixrec* rs = &rec[MI(o, m, cell_at(o, sq))];
            for (int q = 0; q < rs->ntarget; q++)
              if (rs->tgt[q] == c) T += rs->wt[q];
          }
      Tw[MI(o, m, c)] = T;
    }
  }
  double* Qnew = (double*)malloc(sizeof(double) * (size_t)N * NV * nc);
  memcpy(Qnew, Qc, sizeof(double) * (size_t)N * NV * nc);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; c++) {
    if (!o->inB[c]) continue;
    int ijk[3];
    coords(o, c, ijk);
    for (int m = 0; m < N; m++) {
      if (!((o->smask[c] >> m) & 1u)) continue;
      double acc[5] = {0, 0, 0, 0, 0};
      const mixrec* own = &rec[MI(o, m, c)];
      for (int q = 0; q < own->ntarget; q++) {
        const double f = o->alpha[MI(o, m, c)] == 0.0 ? 1.0 : mix_limit(Tw[MI(o, m, c)], Tw[MI(o, m, own->tgt[q])]);
        const double vt = vfac(o, own->tgt[q]);
        for (int v = 0; v < NV; v++) acc[v] += f * (own->M[q][v] * vt);
      }
      /* exchanges that neighbours send to this cell, neighbour offsets in
         lexicographic (z, y, x) order */
      for (int dz = (D >= 3 ? -1 : 0); dz <= (D >= 3 ? 1 : 0); dz++)
        for (int dy = (D >= 2 ? -1 : 0); dy <= (D >= 2 ? 1 : 0); dy++)
          for (int dx = -1; dx <= 1; dx++) {
            if (dx == 0 && dy == 0 && dz == 0) continue;
            int sq[3] = {ijk[0] - dx, ijk[1] - dy, ijk[2] - dz};
            if (!in_array(o, sq)) continue;
            long sc = cell_at(o, sq);
            const mixrec* rs = &rec[MI(o, m, sc)];
            for (int q = 0; q < rs->ntarget; q++)
              if (rs->tgt[q] == c) {
                const double f = o->alpha[MI(o, m, sc)] == 0.0 ? 1.0 : mix_limit(Tw[MI(o, m, sc)], Tw[MI(o, m, c)]);
                const double vs = vfac(o, sc);
                for (int v = 0; v < NV; v++) acc[v] -= f * (rs->M[q][v] * vs);
              }
          }
      for (int v = 0; v < NV; v++) Qnew[QI(o, m, v, c)] = Qc[QI(o, m, v, c)] + acc[v];
    }
    /* material that lost all volume and has no same-material neighbour: merged
       into the cell's primary material */
    for (int m = 0; m < N; m++) {
      if (!mergef[MI(o, m, c)]) continue;
      int pm = o->chi[c];
      for (int v = 0; v < NV; v++) {
        Qnew[QI(o, pm, v, c)] = Qnew[QI(o, pm, v, c)] + Qnew[QI(o, m, v, c)];
        Qnew[QI(o, m, v, c)] = 0.0;
      }
      count(o, ORC_C_MERGE);
    }
  }
  memcpy(Qc, Qnew, sizeof(double) * (size_t)N * NV * nc);
  free(Qnew);
  free(rec);
  free(mergef);
  free(Tw);
}

/* ------------------------------------------------------------------ */
/* scale separation (a12, Sec. 2.3.3)                                   */
/* ------------------------------------------------------------------ */
static void scale_separation(orc* o) {
  int N = o->N, D = o->D;
  double eps = o->eps_ss;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    o->phit[c] = o->phi[c];
    o->chit[c] = o->chi[c];
  }
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    if (!o->inB[c] || !o->mixed[c]) continue;
    int np = 0;
    for (int m = 0; m < N; m++)
      if (present(o, c, m)) np++;
    if (np < 2) continue; /* not in S_0 */
    int chi1 = o->chi[c], ijk[3];
    coords(o, c, ijk);
    int near_minus = 0;
    for (int dz = (D >= 3 ? -1 : 0); dz <= (D >= 3 ? 1 : 0) && !near_minus; dz++)
      for (int dy = (D >= 2 ? -1 : 0); dy <= (D >= 2 ? 1 : 0) && !near_minus; dy++)
        for (int dx = -1; dx <= 1 && !near_minus; dx++) {
          int q[3] = {ijk[0] + dx, ijk[1] + dy, ijk[2] + dz};
          double mn, mx;
          vertex_minmax(o, cell_at(o, q), chi1, &mn, &mx);
          if (mn - eps <= 0.0 && mx - eps >= 0.0) near_minus = 1;
        }
    if (near_minus) continue;
    /* oddball: new indicator = the other material of largest volume fraction */
    count(o, ORC_C_ODDBALL);
    int chs = -1;
    for (int m = 0; m < N; m++) {
      if (m == chi1 || !((o->xs[c] >> m) & 1u)) continue;
      if (chs < 0 || o->alpha[MI(o, m, c)] > o->alpha[MI(o, chs, c)]) chs = m;
    }
    double dmin = 0.0;
    int found = 0;
    for (int dz = (D >= 3 ? -3 : 0); dz <= (D >= 3 ? 3 : 0); dz++)
      for (int dy = (D >= 2 ? -3 : 0); dy <= (D >= 2 ? 3 : 0); dy++)
        for (int dx = -3; dx <= 3; dx++) {
          int q[3] = {ijk[0] + dx, ijk[1] + dy, ijk[2] + dz};
          if (!interior(o, q)) continue;
          long i0 = cell_at(o, q);
          double mn, mx;
          vertex_minmax(o, i0, chs, &mn, &mx);
          if (!(mn + eps <= 0.0 && mx + eps >= 0.0)) continue; /* not in S_+ */
          double n[3];
          normal_m(o, i0, chs, n);
          double ps = phim(o, i0, chs);
          double dd = 0.0;
          for (int d = 0; d < D; d++) {
            double pd = centre(o, d, q[d]) - (ps + eps) * n[d];
            double df = centre(o, d, ijk[d]) - pd;
            dd += df * df;
          }
          dd = sqrt(dd);
          if (!found || dd < dmin) { dmin = dd; found = 1; }
        }
    if (found) o->phit[c] = fabs(dmin - eps);
    o->chit[c] = (uint8_t)chs;
    /* the cell now belongs to chi_1*; when chi_1* holds no content in it
       (its volume appeared with the new topology, as in the droplet demo's
       neck), the content of chi_1 becomes chi_1*'s: the totals are kept,
       per-material mass knowingly not (counted with the merges), and chi_1,
       left with a small volume and no content, is a small cell for mixing */
    if (o->Q[QI(o, chs, 0, c)] == 0.0 && o->Q[QI(o, chi1, 0, c)] > 0.0) {
      for (int v = 0; v < o->NV; v++) {
        o->Q[QI(o, chs, v, c)] = o->Q[QI(o, chi1, v, c)];
        o->Q[QI(o, chi1, v, c)] = 0.0;
      }
      count(o, ORC_C_MERGE);
    }
  }
#pragma omp parallel for schedule(static)
  for (long c = 0; c < o->ncell; c++) {
    o->phi[c] = o->phit[c];
    o->chi[c] = o->chit[c];
  }
}

/* ------------------------------------------------------------------ */
/* band maintenance: Godunov eikonal Jacobi iterations on band cells   */
/* away from the interface                                             */
/* ------------------------------------------------------------------ */
static double godunov(const orc* o, long c) {
  int D = o->D;
  double a[3] = {0, 0, 0}, hh[3] = {1, 1, 1}, w[3] = {1, 1, 1};
  for (int d = 0; d < D; d++) {
    long jm = c - o->st[d], jp = c + o->st[d];
    double vm = interior_c(o, jm) ? o->phi[jm] : o->phi[c];
    double vp = interior_c(o, jp) ? o->phi[jp] : o->phi[c];
    a[d] = fmin(vm, vp);
    hh[d] = o->h[d];
    w[d] = o->ih2[d];
  }
  /* sort ascending by a, stable */
  for (int i = 1; i < D; i++)
    for (int j = i; j > 0 && a[j] < a[j - 1]; j--) {
      double t = a[j]; a[j] = a[j - 1]; a[j - 1] = t;
      t = hh[j]; hh[j] = hh[j - 1]; hh[j - 1] = t;
      t = w[j]; w[j] = w[j - 1]; w[j - 1] = t;
    }
  /* smallest k with a solution of sum_{j<=k} ((phi - a_j)/h_j)^2 = 1, phi > a_k */
  double ph = a[0] + hh[0];
  for (int k = 1; k < D; k++) {
    if (ph <= a[k]) break;
    double A = 0.0, B = 0.0, C = -1.0;
    for (int j = 0; j <= k; j++) {
      A += w[j];
      B += w[j] * a[j];
      C += w[j] * a[j] * a[j];
    }
    double disc = B * B - A * C;
    ph = (B + sqrt(disc > 0.0 ? disc : 0.0)) / A;
  }
  return ph;
}
static void reinit(orc* o) {
  compute_xs(o);
  for (int it = 0; it < o->p.reinit_iters; it++) {
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) o->phit[c] = o->phi[c];
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) {
      if (!o->inB[c] || popc(o->xs[c]) >= 2) continue;
      double ph = godunov(o, c);
      if (ph > o->cap) ph = o->cap;
      o->phit[c] = ph;
    }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; c++) o->phi[c] = o->phit[c];
  }
}

/* ------------------------------------------------------------------ */
/* driver                                                               */
/* ------------------------------------------------------------------ */
/* One full step. Record mode (tphi != NULL, replay == 0): the level set after
 * the boundary fill at the start of every stage and after the level-set stage
 * of the last stage is copied to tape slots 0..3 and the time step to *tdt.
 * Replay mode (replay == 1): the interface evolution is frozen to a recorded
 * tape. Slot s replaces the level set at the start of stage s, slot s+1 the
 * level-set stage of stage s, and the time step is *tdt; band maintenance
 * and scale separation are skipped (the next step's tape brings their result).
 * What remains a function of the conserved state is the flow part of the
 * step: primitive recovery, ghost extension, interface exchange, fluxes,
 * RK combination and mixing, with every volume fraction, aperture and normal
 * taken from the recorded interface. */
static int step_once(orc* o, double t_end, double* tphi, uint8_t* tchi, double* tdt, int replay) {
  const long nc = o->ncell;
  if (replay) {
    memcpy(o->phi, tphi, sizeof(double) * nc);
    memcpy(o->chi, tchi, nc);
  } else {
    bc_phichi(o);
    if (tphi) {
      memcpy(tphi, o->phi, sizeof(double) * nc);
      memcpy(tchi, o->chi, nc);
    }
  }
  step_band(o);
  geometry(o, o->Q);
  hold_ambient(o, o->Q, o->t);
  memcpy(o->phin, o->phi, sizeof(double) * nc);
  memcpy(o->chin, o->chi, nc);
  int last = 0;
  for (int s = 0; s < o->S; s++) {
    double* Qs = s == 0 ? o->Q : (s == 1 ? o->Q1 : o->Q2);
    double* Qo = s == o->S - 1 ? o->Q : (s == 0 ? o->Q1 : o->Q2);
    prim_extend(o, Qs);
    bc_uhat(o);
    /* the exchange of stage 0 comes first: the bound of the step reads the
       free-surface velocities it sets */
    interface_exchange(o, Qs, s == 0 ? o->t : o->t + rk_c(o, s) * o->dt);
    if (s == 0) {
      if (replay) {
        o->dt = *tdt;
      } else {
        compute_dt(o, t_end);
        last = o->t + o->dt >= t_end;
        if (tdt) *tdt = o->dt;
      }
    }
    if (!replay) extend_velocity(o);
    flux_update(o, s, Qs, Qo);
    if (replay) {
      memcpy(o->phi, tphi + (long)(s + 1) * nc, sizeof(double) * nc);
      memcpy(o->chi, tchi + (long)(s + 1) * nc, nc);
    } else {
      levelset_stage(o, s);
      bc_phichi(o);
      if (tphi) {
        memcpy(tphi + (long)(s + 1) * nc, o->phi, sizeof(double) * nc);
        memcpy(tchi + (long)(s + 1) * nc, o->chi, nc);
      }
    }
    geometry(o, Qo);
    hold_ambient(o, Qo, o->t + rk_c(o, s + 1) * o->dt);
    mixing(o, Qo);
  }
  o->t = last ? t_end : o->t + o->dt;
  o->cnt[ORC_C_STEPS]++;
  if (replay) return o->err;
  if (o->p.scale_sep) {
    scale_separation(o);
    bc_phichi(o);
  }
  if (o->p.reinit) {
    reinit(o);
    bc_phichi(o);
  }
  return o->err;
}

int orc_step(orc* o, int32_t nsteps, double t_end) {
  for (int it = 0; it < nsteps; it++) {
    if (o->err) return o->err;
    if (!(o->t < t_end)) break;
    step_once(o, t_end, NULL, NULL, NULL, 0);
  }
  return o->err;
}

long orc_ncell(const orc* o) { return o->ncell; }

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int orc_step_taped(orc* o, double t_end, double* tphi, uint8_t* tchi, double* tdt) {
  if (o->err) return o->err;
  if (!(o->t < t_end)) return -1;
  return step_once(o, t_end, tphi, tchi, tdt, 0);
}

int orc_replay_step(orc* o, const double* tphi, const uint8_t* tchi, double dt) {
  if (o->err) return o->err;
  return step_once(o, 0.0, (double*)tphi, (uint8_t*)tchi, &dt, 1);
}

orc* orc_create(const orc_params* p) {
  if (p->dim < 1 || p->dim > 3 || p->nmat < 1 || p->nmat > ORC_MAXM) return NULL;
  if (p->rk_stages != 0 && p->rk_stages != 2 && p->rk_stages != 3) return NULL;
  for (int m = 0; m < p->nmat; m++)
    if (p->eos_kind[m] == 1 && !(p->tait_B[m] > 0.0 && p->tait_rho0[m] > 0.0)) return NULL;
  if (p->geom != 0 && !(p->geom == 1 && p->dim == 1 && p->lo[0] >= 0.0)) return NULL;
  if (p->fs_mat < -1 || p->fs_mat >= p->nmat) return NULL;
  if (p->fs_mat >= 0 && !(p->fs_rho > 0.0 && p->fs_t1 > p->fs_t0)) return NULL;
  orc* o = (orc*)calloc(1, sizeof(orc));
  o->p = *p;
  /* Tait materials: the effective pinf of the sound speed and of the energy */
  for (int m = 0; m < p->nmat; m++)
    if (p->eos_kind[m] == 1) o->p.pinf[m] = p->tait_B[m] - p->tait_p0[m];
  o->S = p->rk_stages == 2 ? 2 : 3;
  o->D = p->dim;
  o->N = p->nmat;
  o->NV = p->dim + 2;
  for (int d = 0; d < 3; d++) {
    int act = d < o->D;
    o->n[d] = act ? p->n[d] : 1;
    o->pn[d] = act ? p->n[d] + 2 * G : 1;
    o->off[d] = act ? G : 0;
    o->h[d] = act ? (p->hi[d] - p->lo[d]) / (double)p->n[d] : 1.0;
    o->rh[d] = 1.0 / o->h[d];
    o->rh2[d] = 0.5 * o->rh[d];
    o->ih2[d] = o->rh[d] * o->rh[d];
  }
  o->st[0] = 1;
  o->st[1] = o->pn[0];
  o->st[2] = (long)o->pn[0] * o->pn[1];
  o->ncell = (long)o->pn[0] * o->pn[1] * o->pn[2];
  o->V = 1.0;
  for (int d = 0; d < o->D; d++) o->V = o->V * o->h[d];
  o->rV = 1.0 / o->V;
  for (int d = 0; d < o->D; d++) o->farea[d] = o->V / o->h[d];
  o->hmin = o->h[0];
  for (int d = 1; d < o->D; d++) o->hmin = fmin(o->hmin, o->h[d]);
  double ce = p->scale_eps_h > 0 ? p->scale_eps_h : (o->D == 1 ? 0.5 : (o->D == 2 ? 0.75 : 0.9));
  o->eps_ss = ce * o->hmin;
  o->cap = p->phi_cap_h * o->hmin;
  for (int m = 0; m < o->N; m++) {
    o->gm1[m] = o->p.gamma[m] - 1.0;
    o->gpi[m] = o->p.gamma[m] * o->p.pinf[m];
  }
  long nc = o->ncell, N = o->N, NV = o->NV;
  o->Q = (double*)calloc((size_t)(N * NV * nc), 8);
  o->Q1 = (double*)calloc((size_t)(N * NV * nc), 8);
  o->Q2 = (double*)calloc((size_t)(N * NV * nc), 8);
  o->phi = (double*)calloc((size_t)nc, 8);
  o->phin = (double*)calloc((size_t)nc, 8);
  o->phit = (double*)calloc((size_t)nc, 8);
  o->chi = (uint8_t*)calloc((size_t)nc, 1);
  o->chin = (uint8_t*)calloc((size_t)nc, 1);
  o->chit = (uint8_t*)calloc((size_t)nc, 1);
  o->smask = (uint8_t*)calloc((size_t)nc, 1);
  o->inB = (uint8_t*)calloc((size_t)nc, 1);
  o->xs = (uint8_t*)calloc((size_t)nc, 1);
  o->mixed = (uint8_t*)calloc((size_t)nc, 1);
  o->cut = (uint8_t*)calloc((size_t)nc, 1);
  o->alpha = (double*)calloc((size_t)(N * nc), 8);
  o->Alo = (double*)calloc((size_t)(3 * N * nc), 8);
  o->Ahi = (double*)calloc((size_t)(3 * N * nc), 8);
  o->W = (double*)calloc((size_t)(N * NV * nc), 8);
  o->Wt = (double*)calloc((size_t)(N * NV * nc), 8);
  o->fill = (uint8_t*)calloc((size_t)(N * nc), 1);
  o->fillt = (uint8_t*)calloc((size_t)(N * nc), 1);
  o->isreal = (uint8_t*)calloc((size_t)(N * nc), 1);
  o->Uh = (double*)calloc((size_t)(N * NV * nc), 8);
  o->X = (double*)calloc((size_t)(N * NV * nc), 8);
  o->vel = (double*)calloc((size_t)(3 * nc), 8);
  o->velt = (double*)calloc((size_t)(3 * nc), 8);
  o->vf = (uint8_t*)calloc((size_t)nc, 1);
  o->vft = (uint8_t*)calloc((size_t)nc, 1);
  o->F = (double*)calloc((size_t)(3 * N * NV * nc), 8);
  return o;
}

void orc_destroy(orc* o) {
  if (!o) return;
  void* ptrs[] = {o->Q, o->Q1, o->Q2, o->phi, o->phin, o->phit, o->chi, o->chin, o->chit, o->smask,
                  o->inB, o->xs, o->mixed, o->cut, o->alpha, o->Alo, o->Ahi, o->W, o->Wt, o->fill,
                  o->fillt, o->isreal, o->Uh, o->X, o->vel, o->velt, o->vf, o->vft, o->F};
  for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); i++) free(ptrs[i]);
  free(o);
}

/* interior linear index of padded cell c */
static long interior_index(const orc* o, const int* ijk) {
  long i = ijk[0] - o->off[0], j = ijk[1] - o->off[1], k = ijk[2] - o->off[2];
  return (k * o->n[1] + j) * o->n[0] + i;
}
static long n_interior(const orc* o) { return (long)o->n[0] * o->n[1] * o->n[2]; }

/* initial data: unsigned distance phi, indicator chi, primitive state of each
   material in each cell ([N][NV][interior cells]) */
int orc_set_levelset(orc* o, const double* phi, const int32_t* chi, const double* prim) {
  int N = o->N, NV = o->NV;
  long ni = n_interior(o);
  for (long c = 0; c < o->ncell; c++) {
    int ijk[3];
    coords(o, c, ijk);
    if (!interior(o, ijk)) continue;
    long q = interior_index(o, ijk);
    double ph = phi[q];
    if (ph > o->cap) ph = o->cap;
    o->phi[c] = ph;
    o->chi[c] = (uint8_t)chi[q];
  }
  bc_phichi(o);
  step_band(o);
  /* the correction at start-up needs the masses alpha rho: raw volume
     fractions first, then the corrected ones with those masses */
  geometry(o, NULL);
  double* mass = (double*)calloc((size_t)N * NV * o->ncell, 8);
  for (long c = 0; c < o->ncell; c++) {
    int ijk[3];
    coords(o, c, ijk);
    if (!interior(o, ijk)) continue;
    long q = interior_index(o, ijk);
    for (int m = 0; m < N; m++) mass[QI(o, m, 0, c)] = o->alpha[MI(o, m, c)] * prim[((long)m * NV) * ni + q];
  }
  geometry(o, mass);
  free(mass);
  memset(o->Q, 0, sizeof(double) * (size_t)N * NV * o->ncell);
  for (long c = 0; c < o->ncell; c++) {
    int ijk[3];
    coords(o, c, ijk);
    if (!interior(o, ijk)) continue;
    long q = interior_index(o, ijk);
    for (int m = 0; m < N; m++) {
      double a = o->alpha[MI(o, m, c)];
      if (!(a > 0.0)) continue;
      double w[5], u[5];
      for (int v = 0; v < NV; v++) w[v] = prim[((long)m * NV + v) * ni + q];
      prim_to_cons(o, m, w, u);
      for (int v = 0; v < NV; v++) o->Q[QI(o, m, v, c)] = a * u[v];
    }
  }
  o->t = 0.0;
  o->dt = 0.0;
  o->err = 0;
  hold_ambient(o, o->Q, 0.0);
  memset(o->ledger, 0, sizeof(o->ledger));
  memset(o->cnt, 0, sizeof(o->cnt));
  return 0;
}

void orc_get_state(const orc* o, double* Q, double* alpha, double* phi, int32_t* chi, double* t) {
  int N = o->N, NV = o->NV;
  long ni = n_interior(o);
  for (long c = 0; c < o->ncell; c++) {
    int ijk[3];
    coords(o, c, ijk);
    if (!interior(o, ijk)) continue;
    long q = interior_index(o, ijk);
    if (Q)
      for (int m = 0; m < N; m++)
        for (int v = 0; v < NV; v++) Q[((long)m * NV + v) * ni + q] = o->Q[QI(o, m, v, c)];
    if (alpha)
      for (int m = 0; m < N; m++) alpha[(long)m * ni + q] = o->alpha[MI(o, m, c)];
    if (phi) phi[q] = o->phi[c];
    if (chi) chi[q] = o->chi[c];
  }
  if (t) *t = o->t;
}

void orc_set_state(orc* o, const double* Q, const double* phi, const int32_t* chi, double t) {
  int N = o->N, NV = o->NV;
  long ni = n_interior(o);
  for (long c = 0; c < o->ncell; c++) {
    int ijk[3];
    coords(o, c, ijk);
    if (!interior(o, ijk)) continue;
    long q = interior_index(o, ijk);
    for (int m = 0; m < N; m++)
      for (int v = 0; v < NV; v++) o->Q[QI(o, m, v, c)] = Q[((long)m * NV + v) * ni + q];
    o->phi[c] = phi[q];
    o->chi[c] = (uint8_t)chi[q];
  }
  o->t = t;
  o->err = 0;
  bc_phichi(o);
  step_band(o);
  geometry(o, o->Q);
}

/* overwrite the conserved state of the interior cells (SoA [N][NV][cells]),
 * keeping the level set, the time and the counters */
/* the mixing pass alone on the current state and geometry (a test hook: its
   conservation, convexity and weight limit are pinned on it) */
void orc_mix_only(orc* o) { mixing(o, o->Q); }

/* the scale-separation pass alone on the current level set and geometry (a
   test hook: the oddball choice and the distance re-assignment of Sec. 2.3.3
   are pinned on it) */
void orc_scale_sep_only(orc* o) {
  scale_separation(o);
  bc_phichi(o);
}

void orc_set_conserved(orc* o, const double* Q) {
  int N = o->N, NV = o->NV;
  long ni = n_interior(o);
  for (long c = 0; c < o->ncell; c++) {
    int ijk[3];
    coords(o, c, ijk);
    if (!interior(o, ijk)) continue;
    long q = interior_index(o, ijk);
    for (int m = 0; m < N; m++)
      for (int v = 0; v < NV; v++) o->Q[QI(o, m, v, c)] = Q[((long)m * NV + v) * ni + q];
  }
  o->err = 0;
}

void orc_totals(const orc* o, double* totals, double* ledger) {
  int N = o->N, NV = o->NV;
  for (int m = 0; m < N; m++)
    for (int v = 0; v < NV; v++) {
      double s = 0.0;
      for (long c = 0; c < o->ncell; c++)
        if (interior_c(o, c)) s += cyl(o) ? o->Q[QI(o, m, v, c)] * vfac(o, c) : o->Q[QI(o, m, v, c)];
      if (totals) totals[m * NV + v] = s * o->V;
      if (ledger) ledger[m * NV + v] = o->ledger[m][v];
    }
}
void orc_counters(const orc* o, int64_t* c) {
  for (int i = 0; i < ORC_NCOUNT; i++) c[i] = o->cnt[i];
}
double orc_last_dt(const orc* o) { return o->dt; }
int orc_error(const orc* o) { return o->err; }

void orc_debug_field(const orc* o, int32_t which, double* out) {
  int N = o->N, NV = o->NV;
  long ni = n_interior(o);
  for (long c = 0; c < o->ncell; c++) {
    int ijk[3];
    coords(o, c, ijk);
    if (!interior(o, ijk)) continue;
    long q = interior_index(o, ijk);
    switch (which) {
      case 0:
        for (int m = 0; m < N; m++) out[(long)m * ni + q] = o->alpha[MI(o, m, c)];
        break;
      case 1:
        for (int m = 0; m < N; m++)
          for (int v = 0; v < NV; v++) out[((long)m * NV + v) * ni + q] = o->Uh[QI(o, m, v, c)];
        break;
      case 2:
        for (int m = 0; m < N; m++)
          for (int v = 0; v < NV; v++) out[((long)m * NV + v) * ni + q] = o->X[QI(o, m, v, c)];
        break;
      case 3:
        for (int d = 0; d < 3; d++) out[(long)d * ni + q] = o->vel[d * o->ncell + c];
        break;
      case 4: out[q] = o->mixed[c]; break;
      case 5: out[q] = o->smask[c]; break;
      case 6:
      case 7:
        for (int d = 0; d < 3; d++)
          for (int m = 0; m < N; m++)
            out[((long)d * N + m) * ni + q] = (which == 6 ? o->Alo : o->Ahi)[AI(o, d, m, c)];
        break;
      default: break;
    }
  }
}
