// msf_types.cuh -- device buffers of one instance and launch constants,
// shared by the kernels and the host runtime.
#pragma once

#include "msf_device.cuh"

namespace msf {

struct Bufs {
  double* Q[3];             // Q^n, Q^(1), Q^(2): [N][NV][ncell]
  float* Qf[3];             // FP32-bulk form: FP32 copies of Q^(1), Q^(2) written by the flux
                            // update of the stage before (index 0 unused; null in FP64 contexts)
  double *phi, *phin;       // current and step-start distance
  uint8_t *chi, *chin;      // current and step-start indicator
  uint8_t* xs;              // 3^d material bits of chi (all cells)
  uint8_t* mtmp;            // dilation scratch
  uint8_t* smask;           // step mask: materials carried by an interior cell this step
  uint8_t* xsS;             // 3^d material bits of the stage indicator (band cells)
  uint8_t* gflag;           // GF_MIXED | GF_CUT (band cells; 0 elsewhere)
  double* nrm;              // [N][3][ncell] unit normals of the local level sets (band cells)
  double* alpha;            // [N][ncell]
  double *Alo, *Ahi;        // [D][N][ncell] face apertures (mixed cells)
  void *W0, *W1;            // T [N][NV][ncell] primitive states, ping-pong
  uint8_t *f0, *f1, *isreal;  // [N][ncell]
  void* Uh;                 // T [N][NV][ncell] stencil state (band and halo cells)
  double* X;                // [N][NV][ncell] exchange flux (cut cells)
  double *vel0, *vel1;      // [3][ncell] interface velocity, ping-pong
  uint8_t *vf0, *vf1;
  int* band;                // narrow-band cell list
  int* bandidx;             // cell -> band index or -1
  double* phit;             // [nbandmax] scratch
  uint8_t* chit;            // [nbandmax] scratch
  double* mixq;             // [nbandmax][N][NV] mixed state scratch
  unsigned* mixmerge;       // [nbandmax] materials to merge into the primary
  uint8_t* mixn;            // [nbandmax][N] 0xff: not small, else mixing target count
  uint8_t* mixoff;          // [nbandmax][N][MIX_MAXT] target offset codes
  double* mixbeta;          // [nbandmax][N][MIX_MAXT] normalised mixing weights
  unsigned* mixin;          // [nbandmax][N] bit (offset code) of every neighbour that mixes into the cell
  double* mixT;             // [nbandmax][N] weight sum of the mixing pairs of the cell
  int* mixlist;             // [nbandmax * N] items (k * N + m) of the running mixing pass that mix
  int* geomlist;            // [nbandmax * N] 3D cut items (m * nband + k) of the running geometry pass
  int* lslist;              // [nbandmax * N] level-set items (r * nband + k) of the next level-set stage
  uint8_t* mixtouch;        // [nbandmax] 1: a material of band cell k mixes in this pass
  double* phir;             // [nbandmax][N] new local level-set values
  double* bflux;            // [nbnd][N][NV] boundary-face fluxes of the stage
  double* lpart;            // [ceil(nbnd / NTHREADS)][N][NV] per-block partial sums of bflux
  Ctl* ctl;
};

constexpr int NTHREADS = 256;
// narrow-band kernels: small blocks so that a few thousand band items spread
// over every SM instead of filling the first few hundred wide blocks
constexpr int BAND_THREADS = 64;

// first boundary-face id of each (axis, side): faces are numbered per side in
// interior order of the other coordinates
struct BndBase {
  long long base[6];
};

// one instance of a batch of 1D problems run by the persistent kernel
struct BatchEntry {
  Grid g;
  Bufs b;
  BndBase bb;
  void* Fface;    // T [N][NV][n + 1] face fluxes of the stage
  double* Aface;  // [N][n + 1] face apertures of the stage
  int nbnd;
};

}  // namespace msf
