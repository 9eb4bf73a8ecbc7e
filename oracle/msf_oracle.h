/*
 * msf_oracle.h -- plain FP64 CPU oracle of the conservative sharp-interface
 * multi-material method of Pan, Han, Hu & Adams (arXiv:1704.00519).
 *
 * TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py are the only users. The product (the CUDA
 * library) neither includes nor links this file; the two share no code.
 */
#ifndef MSF_ORACLE_H
#define MSF_ORACLE_H
#include <stdint.h>

#define ORC_MAXM 8

typedef struct {
  int32_t dim;               /* 1, 2 or 3 */
  int32_t n[3];              /* interior cells per axis (1 for unused axes) */
  double lo[3], hi[3];       /* domain box */
  int32_t bc[3][2];          /* 0 transmissive, 1 reflective, 2 inflow */
  double inflow_prim[3][2][5];
  int32_t inflow_mat[3][2];
  int32_t nmat;
  double gamma[ORC_MAXM], pinf[ORC_MAXM]; /* stiffened gas p=(g-1)rho e - g pinf */
  double cfl, weno_eps, mix_alpha;
  int32_t ext_sweeps, vel_sweeps, reinit_iters;
  int32_t scale_sep, reinit;
  double scale_eps_h;        /* epsilon / h_min of the scale separation */
  double phi_cap_h;          /* level-set clamp, in units of h_min */
  int32_t rk_stages;         /* 3: TVD-RK3 (0 means 3); 2: the TVD-RK2 of Sec. 3 */
  /* equation of state per material: 0 stiffened gas (gamma, pinf); 1 Tait's
   * equation p = B (rho/rho0)^gamma - B + p0 (Sec. 2.1; gamma, tait_*) */
  int32_t eos_kind[ORC_MAXM];
  double tait_B[ORC_MAXM], tait_rho0[ORC_MAXM], tait_p0[ORC_MAXM];
  /* 0 Cartesian; 1 axisymmetric cylindrical grid of one dimension, x = radius
   * (Sec. 3, Case II): cell volume r_i h, face areas r_f, momentum source p/r */
  int32_t geom;
  /* free-surface ambient (Sec. 3, Case II): material fs_mat (-1: none) is not
   * solved; its state is held at (fs_rho, 0, p(t)) and the interfaces of the
   * other materials with it carry the pressure p(t) = fs_p0 for t <= fs_t0,
   * falling linearly to fs_p1 at fs_t1, fs_p1 after */
  int32_t fs_mat;
  double fs_rho, fs_p0, fs_t0, fs_t1, fs_p1;
  /* reduced interaction model of Sec. 2.3.2, for comparison with the reading
   * the method runs by default (0: the heavier material R of the pair takes
   * minus the exchange of every other present material, whose area vector
   * S^m carries the pair's interface state): literal_reduced = 1 lets only the
   * pair exchange, X^R = [0, p* S^R, p* u* n.S^R], X^L = -X^R, other
   * materials 0; literal_normal = 1 replaces each area vector S^m by
   * |S^m| n^m (the material's own level-set normal) */
  int32_t literal_reduced, literal_normal;
  /* positivity = 1: every face flux is limited towards the first-order
   * Lax-Friedrichs flux so that the density and p + pinf of the two half
   * states it feeds stay positive (Hu, Adams & Shu 2013); the paper describes
   * no positivity treatment, so this is off by default */
  int32_t positivity;
} orc_params;

typedef struct orc orc;

/* error bits (sticky) */
#define ORC_ENONFINITE 1
#define ORC_ENEGATIVE 2
#define ORC_EBAND 4

/* counters */
enum { ORC_C_CUT = 0, ORC_C_MULTI, ORC_C_CORRECTED, ORC_C_SMALL, ORC_C_MIXFAIL,
       ORC_C_MERGE, ORC_C_ODDBALL, ORC_C_STEPS, ORC_NCOUNT };

orc* orc_create(const orc_params* p);
void orc_destroy(orc* o);
int orc_set_levelset(orc* o, const double* phi, const int32_t* chi, const double* prim);
int orc_step(orc* o, int32_t nsteps, double t_end);
/* replay tape of one step: level set (phi [4][ncell], chi [4][ncell], padded
 * layout) at the start of each stage and after the last level-set stage, and
 * the time step. orc_step_taped takes one step and records it (-1: t >= t_end);
 * orc_replay_step takes one step from the current conserved state with the
 * interface evolution frozen to the tape (the flow part of the step only). */
long orc_ncell(const orc* o);
/* threads the loops over cells use: 1 in the plain build, the OpenMP
   maximum in the -fopenmp build (same results either way) */
int orc_threads(void);
int orc_step_taped(orc* o, double t_end, double* tphi, uint8_t* tchi, double* tdt);
int orc_replay_step(orc* o, const double* tphi, const uint8_t* tchi, double dt);
void orc_set_conserved(orc* o, const double* Q);
/* the mixing pass (Sec. 2.3.2) alone on the current state and geometry */
void orc_mix_only(orc* o);
/* the scale-separation pass (Sec. 2.3.3) alone on the current level set and
   geometry, then the boundary fill of (phi, chi) */
void orc_scale_sep_only(orc* o);
void orc_get_state(const orc* o, double* Q, double* alpha, double* phi, int32_t* chi, double* t);
void orc_set_state(orc* o, const double* Q, const double* phi, const int32_t* chi, double t);
void orc_totals(const orc* o, double* totals, double* ledger);
void orc_counters(const orc* o, int64_t* c);
double orc_last_dt(const orc* o);
int orc_error(const orc* o);
/* intermediate fields of the last stage, interior cells: 0 alpha [N], 1 Uhat [N][nv],
   2 exchange X [N][nv], 3 interface velocity [3], 4 mixed flag, 5 step mask,
   6 lower-face apertures [3][N], 7 upper-face apertures [3][N] */
void orc_debug_field(const orc* o, int32_t which, double* out);

/* building blocks, exported for pins */
double orc_weno5(double a, double b, double c, double d, double e, double eps);
/* eosl, eosr = (gamma, pinf, kind); kind 1 = Tait (pinf = B - p0) */
void orc_hllc(const double* wl, const double* wr, const double* eosl, const double* eosr,
              double* ustar, double* pstar);
double orc_seg_frac(double a, double b);
double orc_tri_frac(double a, double b, double c);
double orc_tet_frac(double a, double b, double c, double d);
#endif
