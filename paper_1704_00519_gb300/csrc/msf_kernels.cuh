// msf_kernels.cuh -- kernels of one TVD-RK3 step of the conservative
// sharp-interface multi-material method (arXiv:1704.00519), templated on the
// bulk arithmetic type T (double, or float for the FP32-bulk form).
//
// Data layout in HBM (one instance): structure of arrays over the padded grid
// (G = 4 halo layers per side, x fastest): Q[m][v][cell] in FP64 for every
// material (three copies: Q^n and two RK stages), phi / chi of the regional
// level set, per-cell u8 masks, and FP64 geometry arrays that are written and
// read only inside the narrow band. Bulk cells (one material within +-5 cells)
// never touch the geometry arrays: their stencil state is Q itself.
#pragma once

#include "msf_types.cuh"

namespace msf {
// kernels have internal linkage: each precision unit compiles its own copy
namespace {

__device__ inline bool ctl_active(const Bufs& b) { return b.ctl->active != 0; }

// --------------------------------------------------------------- halo cells
__device__ inline long long halo_count(const Grid& g) { return g.ncell - g.n_interior; }
__device__ inline void halo_coords(const Grid& g, long long idx_, int* q) {
  // z slabs, then y rows of interior z, then x columns of interior (y, z)
  unsigned idx = (unsigned)idx_;
  const unsigned p0 = g.pn[0], p1 = g.pn[1], TG = 2u * G;
  if (g.D == 3) {
    const unsigned slab = TG * p0 * p1;
    if (idx < slab) {
      const unsigned l = idx / (p0 * p1), r = idx - l * (p0 * p1);
      q[2] = l < (unsigned)G ? (int)l : g.off[2] + g.n[2] + (int)(l - G);
      q[1] = (int)(r / p0);
      q[0] = (int)(r - (r / p0) * p0);
      return;
    }
    idx -= slab;
    const unsigned rows = TG * p0 * g.n[2];
    if (idx < rows) {
      const unsigned kk = idx / (TG * p0), r = idx - kk * (TG * p0), l = r / p0;
      q[2] = g.off[2] + (int)kk;
      q[1] = l < (unsigned)G ? (int)l : g.off[1] + g.n[1] + (int)(l - G);
      q[0] = (int)(r - l * p0);
      return;
    }
    idx -= rows;
    const unsigned kk = idx / (TG * g.n[1]), r = idx - kk * (TG * g.n[1]), jj = r / TG, l = r - jj * TG;
    q[2] = g.off[2] + (int)kk;
    q[1] = g.off[1] + (int)jj;
    q[0] = l < (unsigned)G ? (int)l : g.off[0] + g.n[0] + (int)(l - G);
    return;
  }
  if (g.D == 2) {
    q[2] = 0;
    const unsigned rows = TG * p0;
    if (idx < rows) {
      const unsigned l = idx / p0;
      q[1] = l < (unsigned)G ? (int)l : g.off[1] + g.n[1] + (int)(l - G);
      q[0] = (int)(idx - l * p0);
      return;
    }
    idx -= rows;
    const unsigned jj = idx / TG, l = idx - jj * TG;
    q[1] = g.off[1] + (int)jj;
    q[0] = l < (unsigned)G ? (int)l : g.off[0] + g.n[0] + (int)(l - G);
    return;
  }
  q[1] = q[2] = 0;
  q[0] = idx < (unsigned)G ? (int)idx : g.off[0] + g.n[0] + (int)(idx - G);
}

// halo cells of phi, chi: every out-of-range axis mapped to its boundary source
__device__ __forceinline__ void phase_bc_phichi(const Grid& g, const Bufs& b, int first_, int stride_) {
  long long nh = halo_count(g);
  for (long long idx = (long long)first_; idx < nh;
       idx += (long long)stride_) {
    int q[3], s[3], side, flip;
    halo_coords(g, idx, q);
    for (int d = 0; d < 3; d++) s[d] = q[d];
    for (int d = 0; d < g.D; d++)
      if (q[d] < g.off[d] || q[d] >= g.off[d] + g.n[d]) s[d] = bc_source(g, d, q[d], &side, &flip);
    long long c = cell_at(g, q[0], q[1], q[2]), sc = cell_at(g, s[0], s[1], s[2]);
    b.phi[c] = b.phi[sc];
    b.chi[c] = b.chi[sc];
  }
}
__global__ void k_bc_phichi(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  phase_bc_phichi(g, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// -------------------------------------------------- step masks and the band
// xs = material bits of the 3^d block (clamped to the array)
__device__ __forceinline__ void phase_xs(const Grid& g, const Bufs& b, int first_, int stride_) {
    for (long long c = (long long)first_; c < g.ncell;
       c += (long long)stride_) {
    int q[3];
    coords(g, c, q);
    unsigned bits = 0;
    const int rz = g.D >= 3 ? 1 : 0, ry = g.D >= 2 ? 1 : 0;
    for (int dz = -rz; dz <= rz; dz++)
      for (int dy = -ry; dy <= ry; dy++)
        for (int dx = -1; dx <= 1; dx++)
          if (in_array(g, q[0] + dx, q[1] + dy, q[2] + dz))
            bits |= 1u << b.chi[cell_at(g, q[0] + dx, q[1] + dy, q[2] + dz)];
    b.xs[c] = (uint8_t)bits;
  }
}
__global__ void k_xs(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  if (!ctl_active(b)) return;
  phase_xs(g, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
// OR-dilation by +-4 along axis d (separable box of the step mask)
__device__ __forceinline__ void phase_dilate(const Grid& g, const Bufs& b, const uint8_t* src, uint8_t* dst, int d, int first_, int stride_) {
    const int R = 4;
  for (long long c = (long long)first_; c < g.ncell;
       c += (long long)stride_) {
    int q[3];
    coords(g, c, q);
    unsigned bits = 0;
    for (int o = -R; o <= R; o++) {
      int p = q[d] + o;
      if (p < 0 || p >= g.pn[d]) continue;
      bits |= src[c + (long long)o * g.st[d]];
    }
    dst[c] = (uint8_t)bits;
  }
}
__global__ void k_dilate(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const uint8_t* src, uint8_t* dst, int d) {
  if (!ctl_active(b)) return;
  phase_dilate(g, b, src, dst, d, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
// final step mask on interior cells, band compaction, per-step resets
__device__ __forceinline__ void phase_band(const Grid& g, const Bufs& b, const uint8_t* dil, int first_, int stride_) {
    for (long long c = (long long)first_; c < g.ncell;
       c += (long long)stride_) {
    uint8_t m = 0;
    bool inner = interior_c(g, c);
    if (inner) m = dil[c];
    b.smask[c] = m;
    b.gflag[c] = 0;
    int bi = -1;
    if (inner && popcount8(m) >= 2) {
      bi = atomicAdd(&b.ctl->nband, 1);
      b.band[bi] = (int)c;
    }
    b.bandidx[c] = bi;
  }
}
__global__ void k_band(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const uint8_t* dil) {
  if (!ctl_active(b)) return;
  phase_band(g, b, dil, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// step start: activity flag, band counter reset
__global__ void k_step_begin(const __grid_constant__ Bufs b) {
  Ctl* t = b.ctl;
  t->active = (t->t < t->t_end && t->err == 0) ? 1 : 0;
  t->nband = 0;
  t->lam_bits = 0ull;
}

// save phi^n, chi^n of band cells (used pointwise by the level-set RK stages)
__device__ __forceinline__ void phase_band_save(const Grid& g, const Bufs& b, int first_, int stride_) {
    const int nb = b.ctl->nband;
  for (int k = first_; k < nb; k += stride_) {
    long long c = b.band[k];
    b.phin[c] = b.phi[c];
    b.chin[c] = b.chi[c];
  }
}
__global__ void k_band_save(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  if (!ctl_active(b)) return;
  phase_band_save(g, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// --------------------------------------------- geometry + correction (a3, a4)
__device__ inline unsigned block_bits(const Grid& g, const uint8_t* chi, const int* q) {
  unsigned bits = 0;
  const int rz = g.D >= 3 ? 1 : 0, ry = g.D >= 2 ? 1 : 0;
  for (int dz = -rz; dz <= rz; dz++)
    for (int dy = -ry; dy <= ry; dy++)
      for (int dx = -1; dx <= 1; dx++)
        if (in_array(g, q[0] + dx, q[1] + dy, q[2] + dz)) bits |= 1u << chi[cell_at(g, q[0] + dx, q[1] + dy, q[2] + dz)];
  return bits;
}

// per (band cell, material): unit normal of phi^m for the materials the cell
// carries this step, volume fraction and raw face apertures
template <int DD>
__device__ __forceinline__ void phase_geom_mat_d(const Grid& g, const Bufs& b, int first_, int stride_) {
    const int nb = b.ctl->nband, N = g.N, D = DD;
  const int total = nb * N;
  for (int it = first_; it < total; it += stride_) {
    const int m = it / nb, k = it - m * nb;
    const long long c = b.band[k];
    int q[3];
    coords(g, c, q);
    const unsigned bits = block_bits(g, b.chi, q);
    if ((b.smask[c] >> m) & 1u) {
      double n[3];
      normal_m(g, b.phi, b.chi, c, m, n);
      for (int d = 0; d < 3; d++) b.nrm[((long long)m * 3 + d) * g.ncell + c] = n[d];
    }
    double a = 0.0, alo[3] = {0, 0, 0}, ahi[3] = {0, 0, 0};
    if (popcount8(bits) < 2) {
      if (b.chi[c] == m) {
        a = 1.0;
        for (int d = 0; d < D; d++) alo[d] = ahi[d] = 1.0;
      }
    } else if ((bits >> m) & 1u) {
      // an uncut item: every fraction of cell_geom is 1 (all vertex values
      // > 0) or 0 (all < 0)
      int un = 0;
      if constexpr (DD >= 2) un = uncut_sign<DD>(g, b.phi, b.chi, c, m);
      if (un > 0) {
        a = 1.0;
        for (int d = 0; d < D; d++) alo[d] = ahi[d] = 1.0;
      } else if (un == 0) {
        cell_geom<DD>(g, b.phi, b.chi, c, m, &a, alo, ahi);
      }
    }
    b.alpha[midx(g, m, c)] = a;
    for (int d = 0; d < D; d++) {
      b.Alo[aidx(g, d, m, c)] = alo[d];
      b.Ahi[aidx(g, d, m, c)] = ahi[d];
    }
  }
}
// 3D, first pass: per (band cell, material) item the normal, the fractions of
// the items that need no simplex geometry (a 3^d block of one material, or an
// uncut item whose vertex values all have one sign: constant fractions, 24
// unit tetrahedra times 1/24 and faces of four unit triangles times 1/4), and
// a list of the cut items for k_geom_cut (a tenth of the band or less, each a
// long FP64 chain of 24 tetrahedra), appended warp by warp; the order of the
// list does not matter, each item's results depend on the item alone.
// first_ and stride_ must be warp-aligned (lane l of a warp starts at a
// multiple of 32 plus l, stride a multiple of 32).
__device__ __forceinline__ void phase_geom_mat3(const Grid& g, const Bufs& b, int first_, int stride_) {
  const int nb = b.ctl->nband;
  const int total = nb * g.N;
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  for (int base = first_ - lane; base < total; base += stride_) {
    const int it = base + lane;
    bool cut = false;
    if (it < total) {
      const int m = it / nb;
      const long long c = b.band[it - m * nb];
      int q[3];
      coords(g, c, q);
      const unsigned bits = block_bits(g, b.chi, q);
      if ((b.smask[c] >> m) & 1u) {
        double n[3];
        normal_m(g, b.phi, b.chi, c, m, n);
        for (int d = 0; d < 3; d++) b.nrm[((long long)m * 3 + d) * g.ncell + c] = n[d];
      }
      const bool heavy = popcount8(bits) >= 2 && ((bits >> m) & 1u);
      const int un = heavy ? uncut_sign<3>(g, b.phi, b.chi, c, m) : 0;
      cut = heavy && un == 0;
      if (!cut) {
        const double a = un != 0 ? (un > 0 ? 24.0 * (1.0 / 24.0) : 0.0)
                                 : ((popcount8(bits) < 2 && b.chi[c] == m) ? 1.0 : 0.0);
        b.alpha[midx(g, m, c)] = a;
        for (int d = 0; d < 3; d++) {
          b.Alo[aidx(g, d, m, c)] = a;
          b.Ahi[aidx(g, d, m, c)] = a;
        }
      }
    }
    const unsigned bal = __ballot_sync(FULL, cut);
    if (bal) {
      const int leader = __ffs(bal) - 1;
      int at = 0;
      if (lane == leader) at = (int)atomicAdd(&b.ctl->geom_count, (unsigned)__popc(bal));
      at = __shfl_sync(FULL, at, leader);
      if (cut) b.geomlist[at + __popc(bal & ((1u << lane) - 1u))] = it;
    }
  }
}
// 3D, second pass: the listed cut items, five per warp round, six lanes per
// item (one per face, face_geom3); the item's first lane then sums the 24
// tetrahedron fractions in cell_geom<3>'s order (faces in order, the four
// tetrahedra of each face in order), so the results are cell_geom<3>'s bits.
__global__ void k_geom_cut(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  if (!ctl_active(b)) return;
  const int total = (int)b.ctl->geom_count, nb = b.ctl->nband;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int slot = lane / 6, f = lane - 6 * slot;  // lanes 30 and 31 idle
  const unsigned FULL = 0xffffffffu;
  for (int r0 = 5 * warp; r0 < total; r0 += 5 * nwarps) {
    const bool has = slot < 5 && r0 + slot < total;
    int m = 0;
    long long c = 0;
    double ap = 0.0, t[4] = {0.0, 0.0, 0.0, 0.0};
    if (has) {
      const int it = b.geomlist[r0 + slot];
      m = it / nb;
      c = b.band[it - m * nb];
      face_geom3(g, b.phi, b.chi, c, m, f, ap, t);
    }
    const int from = (slot < 5 ? slot : 0) * 6;
    double vol = 0.0, apv[6];
#pragma unroll
    for (int ff = 0; ff < 6; ff++) {
      apv[ff] = __shfl_sync(FULL, ap, from + ff);
#pragma unroll
      for (int e = 0; e < 4; e++) vol += __shfl_sync(FULL, t[e], from + ff);
    }
    if (has && f == 0) {
      b.alpha[midx(g, m, c)] = vol * (1.0 / 24.0);
#pragma unroll
      for (int d = 0; d < 3; d++) {
        b.Alo[aidx(g, d, m, c)] = apv[2 * d];
        b.Ahi[aidx(g, d, m, c)] = apv[2 * d + 1];
      }
    }
  }
}
__device__ __forceinline__ void phase_geom_mat(const Grid& g, const Bufs& b, int first_, int stride_) {
  if (g.D == 1) phase_geom_mat_d<1>(g, b, first_, stride_);
  else if (g.D == 2) phase_geom_mat_d<2>(g, b, first_, stride_);
  else phase_geom_mat3(g, b, first_, stride_);
}
__global__ void k_geom_mat(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  if (!ctl_active(b)) return;
  phase_geom_mat(g, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// per band cell: flags, partition of each face among the local materials and
// the conservation correction (Sec. 2.3.1, Eq. vol_corr2).
// Qs == nullptr and mass == nullptr: raw volume fractions (start-up)
// With LIST the pass also lists the level-set items (region r, band cell k)
// of the next level-set stage, one per region present in the cell's 3^d block
// (k_levelset takes them from the list instead of striding over every pair);
// first_ and stride_ must then be warp-aligned.
template <bool LIST>
__device__ __forceinline__ void phase_geom_cell(const Grid& g, const Bufs& b, const double* Qs, const double* mass, int first_, int stride_) {
    const int nb = b.ctl->nband;
  const int N = g.N, D = g.D;
  unsigned long long nmulti = 0, ncorr = 0;
  const int lane = threadIdx.x & 31;
  for (int base = first_ - (LIST ? lane : 0); base < nb; base += stride_) {
    const int k = base + (LIST ? lane : 0);
    long long c = 0;
    unsigned bits = 0;
    int q[3] = {0, 0, 0};
    if (k < nb) {
      c = b.band[k];
      coords(g, c, q);
      bits = block_bits(g, b.chi, q);
      b.xsS[c] = (uint8_t)bits;
    }
    if (LIST) {
      const unsigned FULL = 0xffffffffu;
      const int cnt = popcount8(bits);
      int incl = cnt;  // inclusive prefix sum of the warp's item counts
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      const int tot = __shfl_sync(FULL, incl, 31);
      int at = 0;
      if (lane == 31 && tot > 0) at = (int)atomicAdd(&b.ctl->ls_count, (unsigned)tot);
      at = __shfl_sync(FULL, at, 31) + incl - cnt;
      for (int r = 0; r < N; r++)
        if ((bits >> r) & 1u) b.lslist[at++] = r * nb + k;
    }
    if (k >= nb) continue;
    if (popcount8(bits) < 2) {
      b.gflag[c] = 0;
      continue;
    }
    b.gflag[c] = GF_MIXED;
    // the materials partition every face; a face on which every local field
    // is <= 0 (the averaged vertex values can give one next to a junction)
    // goes to the indicators of its two cells, whole or half each
    for (int d = 0; d < D; d++)
      for (int side = 0; side < 2; side++) {
        double* A = side ? b.Ahi : b.Alo;
        double s = 0.0;
        for (int m = 0; m < N; m++)
          if ((bits >> m) & 1u) s += A[aidx(g, d, m, c)];
        if (s == 1.0) {
          // a division by 1 returns its dividend: nothing to scale (the faces
          // of uncut cells, apertures 1 and 0)
        } else if (s > 0.0) {
          for (int m = 0; m < N; m++)
            if ((bits >> m) & 1u) A[aidx(g, d, m, c)] = A[aidx(g, d, m, c)] / s;
        } else {
          const int ca = b.chi[side ? c : c - g.st[d]], cb = b.chi[side ? c + g.st[d] : c];
          if (ca == cb) {
            A[aidx(g, d, ca, c)] = 1.0;
          } else {
            A[aidx(g, d, ca, c)] = 0.5;
            A[aidx(g, d, cb, c)] = 0.5;
          }
        }
      }
    const double* Mref = Qs ? Qs : mass;
    if (!Mref) continue;
    int np = 0;
    double sum = 0.0;
    for (int m = 0; m < N; m++)
      if (b.alpha[midx(g, m, c)] > 0.0) {
        np++;
        sum += b.alpha[midx(g, m, c)];
      }
    if (np < 3) continue;
    nmulti++;
    double rem = 1.0 - sum;
    if (rem != 0.0) ncorr++;
    unsigned used = 0;
    while (rem != 0.0) {
      int best = -1;
      for (int m = 0; m < N; m++)
        if (b.alpha[midx(g, m, c)] > 0.0 && !((used >> m) & 1u))
          if (best < 0 || Mref[qidx(g, m, 0, c)] < Mref[qidx(g, best, 0, c)]) best = m;
      if (best < 0) break;
      used |= 1u << best;
      double na = b.alpha[midx(g, best, c)] + rem;
      if (na >= 0.0) {
        b.alpha[midx(g, best, c)] = na;
        rem = 0.0;
      } else {
        b.alpha[midx(g, best, c)] = 0.0;
        rem = na;
      }
    }
  }
  if (Qs) {
    if (nmulti) atomicAdd(&b.ctl->cnt[C_MULTI], nmulti);
    if (ncorr) atomicAdd(&b.ctl->cnt[C_CORRECTED], ncorr);
  }
}
__global__ void k_geom_cell(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qs, const double* mass) {
  if (!ctl_active(b)) return;
  phase_geom_cell<true>(g, b, Qs, mass, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// stored unit normal of material m at a band cell (written by k_geom_mat)
__device__ inline void stored_normal(const Grid& g, const Bufs& b, long long c, int m, double* n) {
  for (int d = 0; d < 3; d++) n[d] = b.nrm[((long long)m * 3 + d) * g.ncell + c];
}

// interior test of the face neighbour of a cell with coordinates q (side 0: -e_d)
__device__ inline bool nb_interior(const Grid& g, const int* q, int d, int side) {
  const int p = q[d] + (side ? 1 : -1);
  return p >= g.off[d] && p < g.off[d] + g.n[d];
}

// present: positive volume or a positive aperture on one of the cell's faces
__device__ inline bool present(const Grid& g, const Bufs& b, long long c, int m) {
  if (b.alpha[midx(g, m, c)] > 0.0) return true;
  if (!(b.gflag[c] & GF_MIXED) || !((b.xsS[c] >> m) & 1u)) return false;
  for (int d = 0; d < g.D; d++)
    if (b.Alo[aidx(g, d, m, c)] > 0.0 || b.Ahi[aidx(g, d, m, c)] > 0.0) return true;
  return false;
}

// aperture of material m on the face between cL and cR = cL + e_d
__device__ inline double face_aperture(const Grid& g, const Bufs& b, long long cL, long long cR, int d, int m) {
  if (b.gflag[cL] & GF_MIXED) return ((b.xsS[cL] >> m) & 1u) ? b.Ahi[aidx(g, d, m, cL)] : 0.0;
  if (b.gflag[cR] & GF_MIXED) return ((b.xsS[cR] >> m) & 1u) ? b.Alo[aidx(g, d, m, cR)] : 0.0;
  return (b.chi[cL] == m && b.chi[cR] == m) ? 1.0 : 0.0;
}

// volume fraction of m in an interior cell (band cells carry the geometry arrays)
__device__ inline double alpha_of(const Grid& g, const Bufs& b, long long c, int m) {
  if (b.bandidx[c] >= 0) return b.alpha[midx(g, m, c)];
  return b.chi[c] == m ? 1.0 : 0.0;
}

// -------------------------------------- primitive recovery + ghosts (a5, a6)
template <typename T>
__device__ __forceinline__ void phase_prim(const Grid& g, const Bufs& b, const double* Qs, int first_, int stride_) {
    const int nb = b.ctl->nband, N = g.N, NV = g.NV;
  T* W0 = (T*)b.W0;
  T* W1 = (T*)b.W1;
  const int total = nb * N;
  for (int it = first_; it < total; it += stride_) {
    const int m = it / nb, k = it - m * nb;
    const long long c = b.band[k];
    b.f0[midx(g, m, c)] = 0;
    b.isreal[midx(g, m, c)] = 0;
    if (!((b.smask[c] >> m) & 1u)) continue;
    const double a = b.alpha[midx(g, m, c)];
    if (b.chi[c] == m && a > 0.0) {
      T u[5], w[5];
      for (int v = 0; v < NV; v++) u[v] = (T)Qs[qidx(g, m, v, c)] / (T)a;
      cons_to_prim<T>(g, m, g.D, u, w);
      for (int v = 0; v < NV; v++) W0[qidx(g, m, v, c)] = W1[qidx(g, m, v, c)] = w[v];
      b.f0[midx(g, m, c)] = 1;
      b.isreal[midx(g, m, c)] = 1;
    }
  }
}
template <typename T>
__global__ void k_prim(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qs) {
  if (!ctl_active(b)) return;
  phase_prim<T>(g, b, Qs, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// one Jacobi sweep: targets take the upwind-weighted mean of filled face
// neighbours (weights max(0, n . e)), else the plain mean of filled neighbours.
// Every neighbour value is loaded up front, unconditionally (face neighbours of
// an interior cell lie inside the padded arrays), so that a sweep costs one
// round of memory latency instead of one per neighbour.
template <typename T, int DD>
__device__ __forceinline__ void extend_items_d(const Grid& g, const Bufs& b, const void* Win, void* Wout,
                                             const uint8_t* fin, uint8_t* fout, int first, int stride) {
  const int nb = b.ctl->nband, N = g.N, NV = DD + 2, D = DD;
  const T* Wi = (const T*)Win;
  T* Wo = (T*)Wout;
  const int total = nb * N;
  for (int it = first; it < total; it += stride) {
    const int m = it / nb, k = it - m * nb;
    const long long c = b.band[k];
    if (!((b.smask[c] >> m) & 1u)) continue;
    if (b.isreal[midx(g, m, c)]) {
      fout[midx(g, m, c)] = 1;
      continue;
    }
    const uint8_t finc = fin[midx(g, m, c)];
    int q[3];
    coords(g, c, q);
    double n[3];
    stored_normal(g, b, c, m, n);
    bool use[6];
    T x[6][5];
    for (int d = 0; d < D; d++)
      for (int s = 0; s < 2; s++) {
        const int i = 2 * d + s;
        const long long j = s ? c + g.st[d] : c - g.st[d];
        const int bij = b.bandidx[j];
        const unsigned smj = b.smask[j];
        const uint8_t fj = fin[midx(g, m, j)];
        use[i] = nb_interior(g, q, d, s) & (bij >= 0) & (((smj >> m) & 1u) != 0) & (fj != 0);
        for (int v = 0; v < NV; v++) x[i][v] = Wi[qidx(g, m, v, j)];
      }
    T acc[5] = {T(0), T(0), T(0), T(0), T(0)}, acc2[5] = {T(0), T(0), T(0), T(0), T(0)};
    // the normal in T once per item (FP32: on the integer pipes, the same bits
    // as the hardware conversion; the rounding is symmetric, so -(T)x = (T)(-x))
    T nt[3];
#pragma unroll
    for (int d = 0; d < D; d++) {
      if constexpr (sizeof(T) == 4) nt[d] = d2f_bits(n[d]);
      else nt[d] = (T)n[d];
    }
    T sw = T(0);
    int cnt = 0;
    for (int d = 0; d < D; d++)
      for (int s = 0; s < 2; s++) {
        const int i = 2 * d + s;
        if (!use[i]) continue;
        T w = s ? nt[d] : -nt[d];
        w = w > T(0) ? w : T(0);
        for (int v = 0; v < NV; v++) {
          acc[v] += w * x[i][v];
          acc2[v] += x[i][v];
        }
        sw += w;
        cnt++;
      }
    if (sw > T(0)) {
      for (int v = 0; v < NV; v++) Wo[qidx(g, m, v, c)] = acc[v] / sw;
      fout[midx(g, m, c)] = 1;
    } else if (cnt > 0) {
      for (int v = 0; v < NV; v++) Wo[qidx(g, m, v, c)] = acc2[v] / (T)cnt;
      fout[midx(g, m, c)] = 1;
    } else {
      for (int v = 0; v < NV; v++) Wo[qidx(g, m, v, c)] = Wi[qidx(g, m, v, c)];
      fout[midx(g, m, c)] = finc;
    }
  }
}
template <typename T>
__device__ __forceinline__ void extend_items(const Grid& g, const Bufs& b, const void* Win, void* Wout,
                                             const uint8_t* fin, uint8_t* fout, int first, int stride) {
  if (g.D == 1) extend_items_d<T, 1>(g, b, Win, Wout, fin, fout, first, stride);
  else if (g.D == 2) extend_items_d<T, 2>(g, b, Win, Wout, fin, fout, first, stride);
  else extend_items_d<T, 3>(g, b, Win, Wout, fin, fout, first, stride);
}

// one Jacobi sweep: targets take the upwind-weighted mean of filled face
// neighbours (weights max(0, n . e)), else the plain mean of filled neighbours
template <typename T>
__global__ void k_extend(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const void* Win,
                         void* Wout, const uint8_t* fin, uint8_t* fout) {
  if (!ctl_active(b)) return;
  extend_items<T>(g, b, Win, Wout, fin, fout, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// stencil state of band cells: real Q/alpha, ghost cons(W), else NaN
template <typename T>
__device__ __forceinline__ void phase_cons(const Grid& g, const Bufs& b, const double* Qs, const void* Wfin, const uint8_t* ffin, int first_, int stride_) {
    const int nb = b.ctl->nband, N = g.N, NV = g.NV;
  const T* W = (const T*)Wfin;
  T* Uh = (T*)b.Uh;
  const T nanv = (T)__longlong_as_double(0x7ff8000000000000LL);
  const int total = nb * N;
  for (int it = first_; it < total; it += stride_) {
    const int m = it / nb, k = it - m * nb;
    const long long c = b.band[k];
    {
      T u[5];
      if (!((b.smask[c] >> m) & 1u)) {
        for (int v = 0; v < NV; v++) u[v] = nanv;
      } else if (b.isreal[midx(g, m, c)]) {
        const double a = b.alpha[midx(g, m, c)];
        for (int v = 0; v < NV; v++) u[v] = (T)Qs[qidx(g, m, v, c)] / (T)a;
      } else if (ffin[midx(g, m, c)]) {
        T w[5];
        for (int v = 0; v < NV; v++) w[v] = W[qidx(g, m, v, c)];
        prim_to_cons<T>(g, m, g.D, w, u);
      } else {
        for (int v = 0; v < NV; v++) u[v] = nanv;
      }
      for (int v = 0; v < NV; v++) Uh[qidx(g, m, v, c)] = u[v];
    }
  }
}
template <typename T>
__global__ void k_cons(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qs, const void* Wfin, const uint8_t* ffin) {
  if (!ctl_active(b)) return;
  phase_cons<T>(g, b, Qs, Wfin, ffin, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// stencil state of an interior cell (bulk: Q; band: Uh; otherwise NaN)
template <typename T>
__device__ __forceinline__ void interior_uhat(const Grid& g, const Bufs& b, const double* Qs, long long c, int m, T* u) {
  const T nanv = (T)__longlong_as_double(0x7ff8000000000000LL);
  const T* Uh = (const T*)b.Uh;
  if (b.bandidx[c] >= 0) {
    if ((b.smask[c] >> m) & 1u)
      for (int v = 0; v < g.NV; v++) u[v] = Uh[qidx(g, m, v, c)];
    else
      for (int v = 0; v < g.NV; v++) u[v] = nanv;
  } else if (b.chi[c] == m) {
    for (int v = 0; v < g.NV; v++) u[v] = (T)Qs[qidx(g, m, v, c)];
  } else {
    for (int v = 0; v < g.NV; v++) u[v] = nanv;
  }
}
// the FP32 stencil state of an interior cell from the FP32 copy of the stage
// state (the values (float)Q that interior_uhat_n<float> converts)
template <int NV>
__device__ __forceinline__ void interior_uhat_f(const Grid& g, const Bufs& b, const float* Qf, long long c, int m,
                                                float* u) {
  const float nanv = __int_as_float(0x7fc00000);
  const float* Uh = (const float*)b.Uh;
  const int bi = b.bandidx[c];
  const uint8_t ch = b.chi[c];
  float q[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) q[v] = Qf[qidx(g, m, v, c)];
  if (bi >= 0) {
    if ((b.smask[c] >> m) & 1u) {
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = Uh[qidx(g, m, v, c)];
    } else {
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = nanv;
    }
  } else if (ch == m) {
#pragma unroll
    for (int v = 0; v < NV; v++) u[v] = q[v];
  } else {
#pragma unroll
    for (int v = 0; v < NV; v++) u[v] = nanv;
  }
}
// the same with the variable count known at compile time; the band index,
// the indicator and the conserved state are loaded together (one round of
// memory latency for a bulk cell)
template <typename T, int NV>
__device__ __forceinline__ void interior_uhat_n(const Grid& g, const Bufs& b, const double* Qs, long long c, int m,
                                                T* u) {
  const T nanv = (T)__longlong_as_double(0x7ff8000000000000LL);
  const T* Uh = (const T*)b.Uh;
  const int bi = b.bandidx[c];
  const uint8_t ch = b.chi[c];
  double q[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) q[v] = Qs[qidx(g, m, v, c)];
  if (bi >= 0) {
    if ((b.smask[c] >> m) & 1u) {
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = Uh[qidx(g, m, v, c)];
    } else {
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = nanv;
    }
  } else if (ch == m) {
#pragma unroll
    for (int v = 0; v < NV; v++) u[v] = (T)q[v];
  } else {
#pragma unroll
    for (int v = 0; v < NV; v++) u[v] = nanv;
  }
}

// halo cells of the stencil state (one axis out of range at a time)
template <typename T, int DD>
__device__ __forceinline__ void phase_bc_uhat_d(const Grid& g, const Bufs& b, const double* Qs, int first_, int stride_) {
    const int N = g.N, NV = DD + 2, D = DD;
  long long per[3] = {0, 0, 0}, total = 0;
  for (int d = 0; d < D; d++) {
    per[d] = 2LL * G * (g.n_interior / g.n[d]);
    total += per[d];
  }
  T* Uh = (T*)b.Uh;
  for (long long idx = (long long)first_; idx < total;
       idx += (long long)stride_) {
    int d = 0;
    long long r0 = idx;
    while (r0 >= per[d]) { r0 -= per[d]; d++; }
    // r -> (layer l in [0, 2G), other coordinates in interior order)
    const unsigned r = (unsigned)r0;
    const unsigned rest0 = r / (2u * G);
    const unsigned l = r - rest0 * (2u * G);
    unsigned rest = rest0;
    int q[3];
    for (int e = 0; e < 3; e++) {
      if (e == d) continue;
      if (e >= D) { q[e] = 0; continue; }
      const unsigned ne = (unsigned)g.n[e], t = rest / ne;
      q[e] = g.off[e] + (int)(rest - t * ne);
      rest = t;
    }
    q[d] = l < (unsigned)G ? (int)l : g.off[d] + g.n[d] + (int)(l - G);
    int side, flip;
    int s[3] = {q[0], q[1], q[2]};
    s[d] = bc_source(g, d, q[d], &side, &flip);
    const long long c = cell_at(g, q[0], q[1], q[2]), sc = cell_at(g, s[0], s[1], s[2]);
    const int type = g.bc[d][side];
    for (int m = 0; m < N; m++) {
      T u[5];
      if (type == 2 && m == g.inflow_mat[d][side]) {
        T w[5];
        for (int v = 0; v < NV; v++) w[v] = (T)g.inflow_prim[d][side][v];
        prim_to_cons<T>(g, m, D, w, u);
      } else {
        interior_uhat<T>(g, b, Qs, sc, m, u);
        if (flip) u[1 + d] = -u[1 + d];
      }
      for (int v = 0; v < NV; v++) Uh[qidx(g, m, v, c)] = u[v];
    }
  }
}
template <typename T>
__device__ __forceinline__ void phase_bc_uhat(const Grid& g, const Bufs& b, const double* Qs, int first_, int stride_) {
  if (g.D == 1) phase_bc_uhat_d<T, 1>(g, b, Qs, first_, stride_);
  else if (g.D == 2) phase_bc_uhat_d<T, 2>(g, b, Qs, first_, stride_);
  else phase_bc_uhat_d<T, 3>(g, b, Qs, first_, stride_);
}
template <typename T>
__global__ void k_bc_uhat(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qs) {
  if (!ctl_active(b)) return;
  phase_bc_uhat<T>(g, b, Qs, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ----------------------------------------------------------- CFL step (a2)
// largest sum_d (|u_d| + c) / h_d over the items [first, n_interior) with stride
template <typename T, int DD>
__device__ __forceinline__ double dt_items_d(const Grid& g, const Bufs& b, const double* Qs, long long first,
                                           long long stride, unsigned& err, const T* tab = nullptr) {
  const int N = g.N, D = DD, NV = DD + 2;
  double lam = 0.0;
  // the largest material bound is kept in T: widening to FP64 is exact and
  // monotone, so the maximum of the widened values is the widened maximum
  T lamT = T(0);
  T rhT[3];
#pragma unroll
  for (int d = 0; d < D; d++) rhT[d] = (T)g.rh[d];
  // FP32-bulk form: the bulk states of stage 0 from the FP32 copy of Q^n
  // (the values interior_uhat<float> converts)
  const float* Qf = sizeof(T) == 4 ? b.Qf[0] : nullptr;
  for (long long idx = first; idx < g.n_interior; idx += stride) {
    const long long c = interior_cell(g, idx);
    const bool inb = b.bandidx[c] >= 0;
    for (int m = 0; m < N; m++) {
      if ((inb ? !(b.alpha[midx(g, m, c)] > 0.0) : b.chi[c] != m) || m == g.fs_mat) continue;
      T u[5], w[5];
      if (Qf && !inb) {
#pragma unroll
        for (int v = 0; v < NV; v++) u[v] = (T)Qf[qidx(g, m, v, c)];
      } else {
        interior_uhat<T>(g, b, Qs, c, m, u);
      }
      // material constants in T from the table when given (the values the
      // conversions below produce)
      T cs;
      if (tab) {
        cons_to_prim_k<T>(g, m, D, u, w, tab[m], tab[MAXM + m]);
        cs = sound_k<T>(tab[2 * MAXM + m], tab[3 * MAXM + m], w[0], w[D + 1], &err);
      } else {
        cons_to_prim<T>(g, m, D, u, w);
        cs = sound<T>(g, m, w[0], w[D + 1], &err);
      }
      T s = T(0);
#pragma unroll
      for (int d = 0; d < D; d++) s += (fabs(w[1 + d]) + cs) * rhT[d];
      if (s > lamT) lamT = s;
    }
    // a free surface moves at the u* of its wave curve, which the material
    // states do not bound: its cut cells enter the bound with |u*|
    if (g.fs_mat >= 0 && inb && (b.gflag[c] & GF_CUT) && b.alpha[midx(g, g.fs_mat, c)] > 0.0) {
      double s = 0.0;
      for (int d = 0; d < D; d++) s += fabs(b.vel0[d * g.ncell + c]) * g.rh[d];
      if (s > lam) lam = s;
    }
  }
  return (double)lamT > lam ? (double)lamT : lam;
}
template <typename T>
__device__ __forceinline__ double dt_items(const Grid& g, const Bufs& b, const double* Qs, long long first,
                                           long long stride, unsigned& err, const T* tab) {
  if (g.D == 1) return dt_items_d<T, 1>(g, b, Qs, first, stride, err, tab);
  if (g.D == 2) return dt_items_d<T, 2>(g, b, Qs, first, stride, err, tab);
  return dt_items_d<T, 3>(g, b, Qs, first, stride, err, tab);
}
// block maximum of per-thread values (blockDim.x a multiple of 32, at most
// 1024): a butterfly of exchanges in each warp, then the warps' maxima (a
// maximum does not depend on the order)
__device__ __forceinline__ double block_max(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();  // the previous call's readers are done with red
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); w++) r = fmax(r, red[w]);
  return r;
}
template <typename T>
__global__ void k_dt(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qs) {
  if (!ctl_active(b)) return;
  // per-material constants in T: gamma - 1, gamma pinf, gamma, pinf
  __shared__ T s_tab[4 * MAXM];
  if (threadIdx.x < (unsigned)g.N) {
    const int m = threadIdx.x;
    s_tab[m] = T(g.gm1[m]);
    s_tab[MAXM + m] = T(g.gpi[m]);
    s_tab[2 * MAXM + m] = T(g.gamma[m]);
    s_tab[3 * MAXM + m] = T(g.pinf[m]);
  }
  __syncthreads();
  unsigned err = 0;
  const double lam = dt_items<T>(g, b, Qs, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                                 (long long)gridDim.x * blockDim.x, err, s_tab);
  const double bm = block_max(lam);
  if (threadIdx.x == 0) atomic_max_pos_double(&b.ctl->lam_bits, bm);
  if (err) atomicOr(&b.ctl->err, err);
}
__global__ void k_dt_finalize(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  Ctl* t = b.ctl;
  if (!t->active) return;
  const double lam = __longlong_as_double((long long)t->lam_bits);
  t->lam = lam;
  double dt = g.cfl / lam;
  int last = 0;
  if (t->t + dt >= t->t_end) {
    dt = t->t_end - t->t;
    last = 1;
  }
  t->dt = dt;
  t->last = last;
}
__global__ void k_step_end(const __grid_constant__ Bufs b) {
  Ctl* t = b.ctl;
  if (!t->active) return;
  t->t = t->last ? t->t_end : t->t + t->dt;
  t->cnt[C_STEPS] += 1;
}

// ----------------------------------------- reduced interface interaction (a7)
template <typename T, int DD>
__device__ __forceinline__ void phase_interface_d(const Grid& g, const Bufs& b, const double* Qs, int stage, int first_,
                                                int stride_) {
    const int nb = b.ctl->nband, N = g.N, NV = DD + 2, D = DD;
  const double ts = stage == 0 ? b.ctl->t : b.ctl->t + g.rk_c[stage] * b.ctl->dt;  // time of the stage
  const T* Uh = (const T*)b.Uh;
  unsigned err = 0;
  unsigned long long ncut = 0;
  for (int k = first_; k < nb; k += stride_) {
    const long long c = b.band[k];
    for (int d = 0; d < 3; d++) b.vel0[d * g.ncell + c] = 0.0;
    b.vf0[c] = 0;
    if (!(b.gflag[c] & GF_MIXED)) continue;
    int np = 0;
    for (int m = 0; m < N; m++)
      if (present(g, b, c, m)) np++;
    if (np < 2) continue;
    b.gflag[c] |= GF_CUT;
    b.vf0[c] = 1;
    ncut++;
    int eta = -1, xi = -1;
    for (int m = 0; m < N; m++)
      if (present(g, b, c, m) && (eta < 0 || Qs[qidx(g, m, 0, c)] > Qs[qidx(g, eta, 0, c)])) eta = m;
    for (int m = 0; m < N; m++)
      if (m != eta && present(g, b, c, m) && (xi < 0 || Qs[qidx(g, m, 0, c)] > Qs[qidx(g, xi, 0, c)])) xi = m;
    int L, R;
    if (Qs[qidx(g, xi, 0, c)] < Qs[qidx(g, eta, 0, c)]) { L = xi; R = eta; }
    else { L = eta; R = xi; }
    double n[3];
    stored_normal(g, b, c, R, n);
    T uL[5], uR[5], wL[5], wR[5];
    for (int v = 0; v < NV; v++) {
      uL[v] = Uh[qidx(g, L, v, c)];
      uR[v] = Uh[qidx(g, R, v, c)];
    }
    for (int m = 0; m < N; m++)
      for (int v = 0; v < NV; v++) b.X[qidx(g, m, v, c)] = 0.0;
    if (isnan(uL[0]) || isnan(uR[0])) {
      err |= ERR_BAND;
      continue;
    }
    cons_to_prim<T>(g, L, D, uL, wL);
    cons_to_prim<T>(g, R, D, uR, wR);
    T unl = T(0), unr = T(0);
    for (int d = 0; d < D; d++) {
      unl += wL[1 + d] * (T)n[d];
      unr += wR[1 + d] * (T)n[d];
    }
    T us, ps;
    const int FS = g.fs_mat;
    if (FS >= 0 && (L == FS || R == FS)) {
      // free surface: the ambient imposes p* = p(t); the solved side's
      // two-shock wave curve gives u*
      ps = (T)fs_pressure(g, ts);
      if (R == FS) {
        (void)sound<T>(g, L, wL[0], wL[D + 1], &err);
        us = unl - fs_wave<T>(g, L, wL[0], wL[D + 1], ps);
      } else {
        (void)sound<T>(g, R, wR[0], wR[D + 1], &err);
        us = unr + fs_wave<T>(g, R, wR[0], wR[D + 1], ps);
      }
    } else {
      hllc_star<T>(wL[0], unl, wL[D + 1], (T)g.gamma[L], (T)g.pinf[L], wR[0], unr, wR[D + 1], (T)g.gamma[R],
                   (T)g.pinf[R], &us, &ps, g.eos_kind[L] == 1, g.eos_kind[R] == 1);
    }
    const double psd = (double)ps, usd = (double)us;
    // every other present material's boundary carries the pair's interface
    // state and R takes minus their sum; the printed reduced model
    // (literal bit 0) lets only the pair exchange, bit 1 uses |S^m| n^m
    const bool lit = (g.literal & 1) != 0;
    double XR[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m < N; m++) {
      if (lit ? m != R : (m == R || !present(g, b, c, m))) continue;
      double S[3] = {0, 0, 0}, nS = 0.0;
      if (g.geom == 1) {
        // interface area r_I n: the faces' r_f A_f less the wedge side alpha h
        const int ic = (int)(c % g.pn[0]);
        S[0] = b.Ahi[aidx(g, 0, m, c)] * face_r(g, ic + 1) - b.Alo[aidx(g, 0, m, c)] * face_r(g, ic) -
               b.alpha[midx(g, m, c)] * g.h[0];
      } else {
        for (int d = 0; d < D; d++) S[d] = (b.Ahi[aidx(g, d, m, c)] - b.Alo[aidx(g, d, m, c)]) * g.farea[d];
      }
      if (g.literal & 2) {
        double nm[3], len = 0.0;
        stored_normal(g, b, c, m, nm);
        for (int d = 0; d < D; d++) len += S[d] * S[d];
        len = sqrt(len);
        for (int d = 0; d < D; d++) S[d] = len * nm[d];
      }
      for (int d = 0; d < D; d++) nS += n[d] * S[d];
      for (int d = 0; d < D; d++) {
        b.X[qidx(g, m, 1 + d, c)] = psd * S[d];
        XR[1 + d] -= psd * S[d];
      }
      b.X[qidx(g, m, D + 1, c)] = psd * usd * nS;
      XR[D + 1] -= psd * usd * nS;
    }
    for (int v = 1; v < NV; v++) b.X[qidx(g, lit ? L : R, v, c)] = XR[v];
    for (int d = 0; d < D; d++) b.vel0[d * g.ncell + c] = usd * n[d];
  }
  if (ncut) atomicAdd(&b.ctl->cnt[C_CUT], ncut);
  if (err) atomicOr(&b.ctl->err, err);
}
template <typename T>
__device__ __forceinline__ void phase_interface(const Grid& g, const Bufs& b, const double* Qs, int stage, int first_,
                                                int stride_) {
  if (g.D == 1) phase_interface_d<T, 1>(g, b, Qs, stage, first_, stride_);
  else if (g.D == 2) phase_interface_d<T, 2>(g, b, Qs, stage, first_, stride_);
  else phase_interface_d<T, 3>(g, b, Qs, stage, first_, stride_);
}
template <typename T>
__global__ void k_interface(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qs, int stage) {
  if (!ctl_active(b)) return;
  phase_interface<T>(g, b, Qs, stage, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// x / n for a neighbour count n (1 to 6): a division by 1, 2 or 4 is the exact
// scaling x, x / 2, x / 4, which a multiplication by 1/2 or 1/4 gives with the
// same rounding; the count as a double without a conversion instruction
__device__ __forceinline__ double div_count(double x, int n) {
  if (n == 1) return x;
  if (n == 2) return x * 0.5;
  if (n == 4) return x * 0.25;
  const double dn = n == 3 ? 3.0 : (n == 5 ? 5.0 : (n == 6 ? 6.0 : (double)n));
  return x / dn;
}

// one sweep of the interface-velocity extension into the band
template <int DD>
__device__ __forceinline__ void extend_vel_items_d(const Grid& g, const Bufs& b, const double* vin, double* vout,
                                                 const uint8_t* fin, uint8_t* fout, int first, int stride) {
  const int nb = b.ctl->nband, D = DD;
  for (int k = first; k < nb; k += stride) {
    const long long c = b.band[k];
    // every value the sweep may use, loaded up front (one round of latency)
    const uint8_t gf = b.gflag[c], finc = fin[c];
    double vc[3];
    for (int e = 0; e < 3; e++) vc[e] = vin[e * g.ncell + c];
    if (gf & GF_CUT) {
      for (int e = 0; e < 3; e++) vout[e * g.ncell + c] = vc[e];
      fout[c] = 1;
      continue;
    }
    const double phc = b.phi[c];
    int q[3];
    coords(g, c, q);
    bool use[6];
    double phj[6], vj[6][3];
    for (int d = 0; d < D; d++)
      for (int s = 0; s < 2; s++) {
        const int i = 2 * d + s;
        const long long j = s ? c + g.st[d] : c - g.st[d];
        const int bij = b.bandidx[j];
        const uint8_t fj = fin[j];
        use[i] = nb_interior(g, q, d, s) & (bij >= 0) & (fj != 0);
        phj[i] = b.phi[j];
        for (int e = 0; e < D; e++) vj[i][e] = vin[e * g.ncell + j];
      }
    // upwind neighbours (phi_j < phi_c, compared on the bit patterns), and the
    // count of all filled ones; their plain mean is formed only when no
    // neighbour is upwind (the same sums in the same order)
    double acc[3] = {0, 0, 0};
    int cnt = 0, cnt2 = 0;
    for (int d = 0; d < D; d++)
      for (int s = 0; s < 2; s++) {
        const int i = 2 * d + s;
        if (!use[i]) continue;
        cnt2++;
        if (lt_bits(phj[i], phc)) {
          for (int e = 0; e < D; e++) acc[e] += vj[i][e];
          cnt++;
        }
      }
    uint8_t filled = 0;
    for (int e = 0; e < 3; e++) vout[e * g.ncell + c] = vc[e];
    if (cnt > 0) {
      for (int e = 0; e < D; e++) vout[e * g.ncell + c] = div_count(acc[e], cnt);
      filled = 1;
    } else if (cnt2 > 0) {
      double acc2[3] = {0, 0, 0};
      for (int d = 0; d < D; d++)
        for (int s = 0; s < 2; s++)
          if (use[2 * d + s])
            for (int e = 0; e < D; e++) acc2[e] += vj[2 * d + s][e];
      for (int e = 0; e < D; e++) vout[e * g.ncell + c] = div_count(acc2[e], cnt2);
      filled = 1;
    } else if (finc) {
      filled = 1;
    }
    fout[c] = filled;
  }
}
__device__ __forceinline__ void extend_vel_items(const Grid& g, const Bufs& b, const double* vin, double* vout,
                                                 const uint8_t* fin, uint8_t* fout, int first, int stride) {
  if (g.D == 1) extend_vel_items_d<1>(g, b, vin, vout, fin, fout, first, stride);
  else if (g.D == 2) extend_vel_items_d<2>(g, b, vin, vout, fin, fout, first, stride);
  else extend_vel_items_d<3>(g, b, vin, vout, fin, fout, first, stride);
}
__global__ void k_extend_vel(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* vin,
                             double* vout, const uint8_t* fin, uint8_t* fout) {
  if (!ctl_active(b)) return;
  extend_vel_items(g, b, vin, vout, fin, fout, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
// --------------------------------------- fluxes and the RK stage update (a8)
// One CTA owns a tile of interior cells. For each material of the tile it
// stages the stencil state (tile + 3-cell halo) and its primitive quantities
// in shared memory, evaluates every face flux of the tile once (WENO5 of the
// Lax-Friedrichs split fluxes, Jiang & Shu), then updates its cells with the
// aperture-weighted flux differences, the exchange flux and the RK weights.
template <int D>
struct Tile;
template <>
struct Tile<1> { static constexpr int X = 256, Y = 1, Z = 1; };
template <>
struct Tile<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <>
struct Tile<3> { static constexpr int X = 8, Y = 8, Z = 4; };

template <int D, typename T>
struct FluxSmem {
  static constexpr int TX = Tile<D>::X, TY = Tile<D>::Y, TZ = Tile<D>::Z;
  static constexpr int HY = D >= 2 ? 3 : 0, HZ = D >= 3 ? 3 : 0;
  static constexpr int SX = TX + 6, SY = TY + 2 * HY, SZ = TZ + 2 * HZ;
  static constexpr int NS = SX * SY * SZ;
  static constexpr int NV = D + 2;
  static constexpr int NP = D + 2;  // velocities, p, c
  static constexpr int NFX = (TX + 1) * TY * TZ;
  static constexpr int NFY = D >= 2 ? TX * (TY + 1) * TZ : 0;
  static constexpr int NFZ = D >= 3 ? TX * TY * (TZ + 1) : 0;
  static constexpr int NF = NFX + NFY + NFZ;
  // Staged stencil slots. The face stencils read the tile and its axis-aligned
  // halos only; in 3D those are stored compactly (interior, then the x, y and z
  // halo slabs: 1024 slots instead of the 1960 of the bounding box, so three
  // CTAs fit on an SM instead of two); in 1D and 2D the box layout is kept.
  static constexpr bool COMPACT = D == 3;
  static constexpr int B1 = TX * TY * TZ, B2 = B1 + 6 * TY * TZ, B3 = B2 + 6 * TX * TZ;
  static constexpr int NU = COMPACT ? B3 + 6 * TX * TY : NS;
  static constexpr size_t bytes =
      sizeof(T) * ((size_t)NU * (NV + NP) + (size_t)NF * NV) + sizeof(double) * NF + (size_t)NU;
  // slot of the stencil cell at tile-local (lx, ly, lz), at most one
  // coordinate outside the tile
  __device__ static __forceinline__ int slot(int lx, int ly, int lz) {
    if constexpr (!COMPACT) {
      return (lx + 3) + SX * ((ly + HY) + SY * (lz + HZ));
    } else {
      if (lx < 0) return B1 + (lx + 3) + 6 * (ly + TY * lz);
      if (lx >= TX) return B1 + (lx - TX + 3) + 6 * (ly + TY * lz);
      if (ly < 0) return B2 + lx + TX * ((ly + 3) + 6 * lz);
      if (ly >= TY) return B2 + lx + TX * ((ly - TY + 3) + 6 * lz);
      if (lz < 0) return B3 + lx + TX * (ly + TY * (lz + 3));
      if (lz >= TZ) return B3 + lx + TX * (ly + TY * (lz - TZ + 3));
      return lx + TX * (ly + TY * lz);
    }
  }
  // tile-local coordinates of slot s; false for a box-layout slot that no
  // stencil reads (two or more coordinates outside the tile)
  __device__ static __forceinline__ bool coords(int s, int& lx, int& ly, int& lz) {
    if constexpr (!COMPACT) {
      const int sx = s % SX, sy = (s / SX) % SY, sz = s / (SX * SY);
      lx = sx - 3;
      ly = sy - HY;
      lz = sz - HZ;
      int outs = (sx < 3 || sx >= 3 + TX);
      if (D >= 2) outs += (sy < HY || sy >= HY + TY);
      if (D >= 3) outs += (sz < HZ || sz >= HZ + TZ);
      return outs <= 1;
    } else {
      if (s < B1) {
        lx = s % TX; ly = (s / TX) % TY; lz = s / (TX * TY);
      } else if (s < B2) {
        const int t = s - B1, h = t % 6;
        lx = h < 3 ? h - 3 : TX + h - 3; ly = (t / 6) % TY; lz = t / (6 * TY);
      } else if (s < B3) {
        const int t = s - B2, h = (t / TX) % 6;
        lx = t % TX; ly = h < 3 ? h - 3 : TY + h - 3; lz = t / (TX * 6);
      } else {
        const int t = s - B3, h = t / (TX * TY);
        lx = t % TX; ly = (t / TX) % TY; lz = h < 3 ? h - 3 : TZ + h - 3;
      }
      return true;
    }
  }
};

// Tait's pressure of a stencil state, out of line: the stiffened-gas path of
// the staging loop keeps its registers
__device__ __noinline__ double tait_pressure_k(double rho, double B, double rho0, double p0, double gamma) {
  return B * pow(rho / rho0, gamma) - B + p0;
}
// Tait constants of a material (on = 0: stiffened gas)
struct TaitK {
  int on;
  double B, rho0, p0, gamma;
};
__device__ inline TaitK tait_of(const Grid& g, int m) {
  TaitK t;
  t.on = g.eos_kind[m] == 1;
  t.B = g.tait_B[m];
  t.rho0 = g.tait_rho0[m];
  t.p0 = g.tait_p0[m];
  t.gamma = g.gamma[m];
  return t;
}

// primitive velocity, pressure and sound speed of a stencil state (same
// arithmetic as cons_to_prim and sound); isbad: rho <= 0 or c^2 <= 0
template <int D, typename T>
__device__ __forceinline__ void stencil_prim(const T* u, T gm1, T gpi, T gam, T pinf, const TaitK& tk, T* vel,
                                             T& pres, T& cs, bool& isbad) {
  const T rho = u[0];
  T qsum = T(0);
#pragma unroll
  for (int e = 0; e < D; e++) vel[e] = u[1 + e] / rho;
#pragma unroll
  for (int e = 0; e < D; e++) qsum += vel[e] * vel[e];
  const T ke = T(0.5) * rho * qsum;
  if (tk.on)
    pres = (T)tait_pressure_k((double)rho, tk.B, tk.rho0, tk.p0, tk.gamma);
  else
    pres = gm1 * (u[D + 1] - ke) - gpi;
  T c2 = (gam * (pres + pinf)) / rho;
  isbad = !(rho > T(0)) || !(c2 > T(0));
  if (isbad) c2 = c2 > T(0) ? c2 : T(0);
  cs = sqrt(c2);
}

// WENO5 of the Lax-Friedrichs split fluxes through one face along axis d from
// its 6-cell stencil: U[q][v] states, un normal velocity, pr pressure, cs sound
// speed; returns the splitting's wave-speed bound a (the stencil maximum)
template <int D, typename T>
__device__ __forceinline__ T face_flux_regs(const T (&U)[6][D + 2], const T (&un)[6], const T (&pr)[6],
                                            const T (&cs)[6], int d, T eps, T* Fh) {
  constexpr int NV = D + 2;
  T a = T(0);
#pragma unroll
  for (int q = 0; q < 6; q++) {
    const T sp = fabs(un[q]) + cs[q];
    if (sp > a) a = sp;
  }
#pragma unroll
  for (int v = 0; v < NV; v++) {
    T fp[6], fm[6];
#pragma unroll
    for (int q = 0; q < 6; q++) {
      const T uu = U[q][v];
      T F;
      if (v == 0) F = U[q][1 + d];
      else if (v == NV - 1) F = un[q] * (uu + pr[q]);
      else F = (v - 1 == d) ? uu * un[q] + pr[q] : uu * un[q];
      fp[q] = T(0.5) * (F + a * uu);
      fm[q] = T(0.5) * (F - a * uu);
    }
    Fh[v] = weno5<T>(fp[0], fp[1], fp[2], fp[3], fp[4], eps) + weno5<T>(fm[5], fm[4], fm[3], fm[2], fm[1], eps);
  }
  return a;
}

// Positivity-preserving limiting of one face flux (Hu, Adams & Shu 2013; an
// option, the paper has no positivity treatment): Fh is blended towards the
// Lax-Friedrichs flux F_LF = (F(uL) + F(uR) - a (uR - uL)) / 2 with the largest
// theta in [0, 1] that keeps rho, then p + pinf, of the half states
// uL - lam F and uR + lam F (lam = 2 D dt / h_d) at or above
// eps = min(1e-13, their Lax-Friedrichs values); the pressure step runs along
// the segment from the Lax-Friedrichs half state (p is concave in the
// conserved variables) and is skipped for Tait materials; a flux that needs no
// limiting is kept bit for bit. Same operations, in the same order, as the
// oracle.
struct PosArgs {
  int on;
  double dt2d;  // 2 D dt of the stage
  double gm1, gpi, pinf;
  int tait;
};
template <int D, typename T>
__device__ __forceinline__ void pp_limit(const T* uL, const T* uR, T unL, T unR, T pL, T pR, T a, int d,
                                         const PosArgs& pa, T lam, T* Fh) {
  constexpr int NV = D + 2;
  T FL[NV], FR[NV], Flf[NV], F1[NV];
  FL[0] = uL[1 + d];
  FR[0] = uR[1 + d];
#pragma unroll
  for (int e = 0; e < D; e++) {
    FL[1 + e] = e == d ? uL[1 + e] * unL + pL : uL[1 + e] * unL;
    FR[1 + e] = e == d ? uR[1 + e] * unR + pR : uR[1 + e] * unR;
  }
  FL[D + 1] = unL * (uL[D + 1] + pL);
  FR[D + 1] = unR * (uR[D + 1] + pR);
#pragma unroll
  for (int v = 0; v < NV; v++) Flf[v] = T(0.5) * ((FL[v] + FR[v]) - a * (uR[v] - uL[v]));
  const T hl0 = uL[0] - lam * Flf[0], hl1 = uR[0] + lam * Flf[0];
  const T hh0 = uL[0] - lam * Fh[0], hh1 = uR[0] + lam * Fh[0];
  const T eps = fmin(T(1e-13), fmin(hl0, hl1));
  T th = T(1);
  if (hh0 < eps) th = fmin(th, (hl0 - eps) / (hl0 - hh0));
  if (hh1 < eps) th = fmin(th, (hl1 - eps) / (hl1 - hh1));
#pragma unroll
  for (int v = 0; v < NV; v++) F1[v] = th < T(1) ? Flf[v] + th * (Fh[v] - Flf[v]) : Fh[v];
  if (!pa.tait) {
    const T gm1 = (T)pa.gm1, gpi = (T)pa.gpi, pinf = (T)pa.pinf;
    T ql[2], q1[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const T* u = s ? uR : uL;
      const T sg = s ? T(1) : T(-1);
      T hl[NV], h1[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        hl[v] = s ? u[v] + lam * Flf[v] : u[v] - lam * Flf[v];
        h1[v] = u[v] + sg * (lam * F1[v]);
      }
      T kl = T(0), k1 = T(0);
#pragma unroll
      for (int e = 0; e < D; e++) {
        kl += hl[1 + e] * hl[1 + e];
        k1 += h1[1 + e] * h1[1 + e];
      }
      ql[s] = (gm1 * (hl[D + 1] - T(0.5) * kl / hl[0]) - gpi) + pinf;
      q1[s] = (gm1 * (h1[D + 1] - T(0.5) * k1 / h1[0]) - gpi) + pinf;
    }
    const T epq = fmin(T(1e-13), fmin(ql[0], ql[1]));
    T tp = T(1);
    if (q1[0] < epq) tp = fmin(tp, (ql[0] - epq) / (ql[0] - q1[0]));
    if (q1[1] < epq) tp = fmin(tp, (ql[1] - epq) / (ql[1] - q1[1]));
    if (tp < T(1))
#pragma unroll
      for (int v = 0; v < NV; v++) F1[v] = Flf[v] + tp * (F1[v] - Flf[v]);
  }
#pragma unroll
  for (int v = 0; v < NV; v++) Fh[v] = F1[v];
}

template <int D, typename T>
__device__ inline void face_flux_smem(const T* U, const T* P, const int (&sl)[6], int d, int NS, T eps,
                                      const PosArgs& pa, const double* rh, T* Fh) {
  // U[v*NS + s], P[e*NS + s] with e: 0..D-1 velocities, D pressure, D+1 sound speed
  constexpr int NV = D + 2;
  T u[6][NV], un[6], pr[6], cs[6];
#pragma unroll
  for (int q = 0; q < 6; q++) {
    const int s = sl[q];
#pragma unroll
    for (int v = 0; v < NV; v++) u[q][v] = U[v * NS + s];
    un[q] = P[d * NS + s];
    pr[q] = P[D * NS + s];
    cs[q] = P[(D + 1) * NS + s];
  }
  const T a = face_flux_regs<D, T>(u, un, pr, cs, d, eps, Fh);
  if (pa.on) pp_limit<D, T>(u[2], u[3], un[2], un[3], pr[2], pr[3], a, d, pa, (T)(pa.dt2d * rh[d]), Fh);
}

// one face of a flux tile: aperture, WENO5-LLF flux and the boundary ledger.
// DIR is the face normal axis; r indexes the faces of that axis in the tile.
template <int D, typename T, int DIR>
__device__ inline void flux_face(const Grid& g, const Bufs& b, const T* U, const T* P, T* F, double* A,
                                 const uint8_t* bad, const BndBase& bb, int f, int r, int x0, int y0, int z0, int m,
                                 bool anyband, T eps, const PosArgs& pa, unsigned& err) {
  using S = FluxSmem<D, T>;
  constexpr int NV = D + 2, TX = S::TX, TY = S::TY, NS = S::NU;
  int fx, fy, fz;
  if (DIR == 0) {
    fx = r % (TX + 1); fy = (r / (TX + 1)) % TY; fz = r / ((TX + 1) * TY);
  } else if (DIR == 1) {
    fx = r % TX; fy = (r / TX) % (TY + 1); fz = r / (TX * (TY + 1));
  } else {
    fx = r % TX; fy = (r / TX) % TY; fz = r / (TX * TY);
  }
  // the face is the lower face of tile cell (fx, fy, fz)
  const int gx = x0 + fx, gy = y0 + fy, gz = z0 + fz;
  const int qd = DIR == 0 ? gx : (DIR == 1 ? gy : gz);
  // the face exists when its upper cell lies in [off, off + n] along DIR and
  // the other coordinates are interior
  bool exists = gx < g.off[0] + g.n[0] + (DIR == 0 ? 1 : 0);
  if (D >= 2) exists = exists && gy < g.off[1] + g.n[1] + (DIR == 1 ? 1 : 0);
  if (D >= 3) exists = exists && gz < g.off[2] + g.n[2] + (DIR == 2 ? 1 : 0);
  double Af = 0.0;
  T Fh[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) Fh[v] = T(0);
  if (exists) {
    const long long cR = cell_at(g, gx, gy, gz), cL = cR - g.st[DIR];
    Af = anyband ? face_aperture(g, b, cL, cR, DIR, m) : 1.0;
    if (pos_bits(Af) && m != g.fs_mat) {
      if (anyband) {
        const bool lin = qd - 1 >= g.off[DIR], rin = qd < g.off[DIR] + g.n[DIR];
        if ((lin && !((b.smask[cL] >> m) & 1u)) || (rin && !((b.smask[cR] >> m) & 1u))) err |= ERR_BAND;
      }
      // the six stencil cells: tile-local coordinate along DIR from -3 to +2
      // of the face's upper cell
      int sl[6];
#pragma unroll
      for (int q = 0; q < 6; q++)
        sl[q] = DIR == 0 ? S::slot(fx - 3 + q, fy, fz) : (DIR == 1 ? S::slot(fx, fy - 3 + q, fz) : S::slot(fx, fy, fz - 3 + q));
      bool avail = true, isbad = false;
#pragma unroll
      for (int q = 0; q < 6; q++) {
        if (isnan(U[sl[q]])) avail = false;
        if (bad[sl[q]]) isbad = true;
      }
      if (!avail) {
        err |= ERR_BAND;
      } else {
        if (isbad) err |= ERR_NEGATIVE;
        face_flux_smem<D, T>(U, P, sl, DIR, NS, eps, pa, g.rh, Fh);
      }
    }
    // boundary ledger: net inflow through the domain boundary
    const int rr = qd - g.off[DIR];
    if (rr == 0 || rr == g.n[DIR]) {
      // face id: base[DIR][side] + interior index of the other coordinates
      long long lin_id = 0, mul = 1;
      const int qv[3] = {gx, gy, gz};
#pragma unroll
      for (int e = 0; e < D; e++) {
        if (e == DIR) continue;
        lin_id += (long long)(qv[e] - g.off[e]) * mul;
        mul *= g.n[e];
      }
      const long long fid = (rr == 0 ? bb.base[2 * DIR] : bb.base[2 * DIR + 1]) + lin_id;
      const double sgn = rr == 0 ? 1.0 : -1.0;
      const double fa = (D == 1 && g.geom == 1) ? face_r(g, qd) : g.farea[DIR];
#pragma unroll
      for (int v = 0; v < NV; v++) b.bflux[((fid * g.N) + m) * NV + v] = sgn * (Af * (double)Fh[v] * fa);
    }
  }
  A[f] = Af;
#pragma unroll
  for (int v = 0; v < NV; v++) F[v * S::NF + f] = Fh[v];
}

// bit-identical values (+0 and -0 differ; a NaN is never the same as anything)
__device__ inline bool same_bits(float a, float b) { return __float_as_int(a) == __float_as_int(b) && a == a; }
__device__ inline bool same_bits(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b) && a == a;
}

// does this thread's share of the staged stencil states (those the faces
// read) equal, bit for bit, the state of the tile's first cell; out of line
// so that the flux path keeps its registers
template <int D, typename T>
__device__ __noinline__ bool stencil_uniform(const T* U, const uint8_t* bad, int tid) {
  using S = FluxSmem<D, T>;
  constexpr int NV = D + 2, TX = S::TX, TY = S::TY, TZ = S::TZ, NS = S::NU;
  const int sref = S::slot(0, 0, 0);
  bool same = !bad[sref];
  for (int s = tid; s < NS && same; s += TX * TY * TZ) {
    int lx, ly, lz;
    if (!S::coords(s, lx, ly, lz)) continue;
    for (int v = 0; v < NV; v++) same = same && same_bits(U[v * NS + s], U[v * NS + sref]);
  }
  return same;
}

// a face flux widened to FP64 (exact; integer operations for FP32)
__device__ __forceinline__ double to_d(float x) { return f2d_bits(x); }
__device__ __forceinline__ double to_d(double x) { return x; }

// exact error of a float sum: s + x = t + e exactly (Knuth's two-sum; no
// multiplications, so no FMA contraction applies)
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  const float e = (s - (t - bp)) + (x - bp);
  s = t;
  c += e;
}

// one tile of the flux update (tile index over the (x, y, z) tile grid)
template <int D, typename T>
__device__ __forceinline__ void flux_tile(const Grid& g, const Bufs& b, const double* Qs, const double* Qn,
                                          double* Qout, double beta, double omb, const BndBase& bb, int tile,
                                          const float* Qsf, float* Qof) {
  using S = FluxSmem<D, T>;
  constexpr int NV = D + 2, TX = S::TX, TY = S::TY, TZ = S::TZ, NS = S::NU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* A = (double*)smem_raw;       // [NF] apertures (8-byte aligned first)
  T* U = (T*)(A + S::NF);              // [NV][NS]
  T* P = U + NV * NS;                  // [D+2][NS]
  T* F = P + (D + 2) * NS;             // [NV][NF]
  uint8_t* bad = (uint8_t*)(F + NV * S::NF);  // [NS]
  __shared__ unsigned s_union;
  __shared__ unsigned s_err;

  const int tid = threadIdx.x;
  const int nbx = (g.n[0] + TX - 1) / TX, nby = D >= 2 ? (g.n[1] + TY - 1) / TY : 1;
  const int bx = tile % nbx, by = (tile / nbx) % nby, bz = tile / (nbx * nby);
  const int x0 = g.off[0] + bx * TX, y0 = (D >= 2 ? g.off[1] : 0) + by * TY, z0 = (D >= 3 ? g.off[2] : 0) + bz * TZ;
  // the tile's faces include no domain-boundary face and its cells are all interior
  bool interior_tile = x0 > g.off[0] && x0 + TX < g.off[0] + g.n[0];
  if (D >= 2) interior_tile = interior_tile && y0 > g.off[1] && y0 + TY < g.off[1] + g.n[1];
  if (D >= 3) interior_tile = interior_tile && z0 > g.off[2] && z0 + TZ < g.off[2] + g.n[2];
  const int tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
  const int cx = x0 + tx, cy = y0 + ty, cz = z0 + tz;
  const bool inside = cx < g.off[0] + g.n[0] && (D < 2 || cy < g.off[1] + g.n[1]) && (D < 3 || cz < g.off[2] + g.n[2]);
  const long long c = inside ? cell_at(g, cx, cy, cz) : 0;
  const uint8_t mymask = inside ? b.smask[c] : 0;
  if (tid == 0) {
    s_union = 0;
    s_err = 0;
  }
  __syncthreads();
  if (mymask) atomicOr(&s_union, (unsigned)mymask);
  // a tile without band cells has one material whose faces all have aperture 1
  const bool anyband = __syncthreads_or(inside && b.bandidx[c] >= 0) != 0;
  // boundary faces of this tile: clear the slots of every material first
  if (inside) {
    for (int d = 0; d < D; d++) {
      const int qd = d == 0 ? cx : (d == 1 ? cy : cz);
      const int r = qd - g.off[d];
      for (int side = 0; side < 2; side++) {
        if (!((side == 0 && r == 0) || (side == 1 && r == g.n[d] - 1))) continue;
        int qq[3] = {cx, cy, cz};
        long long lin_id = 0, mul = 1;
        for (int e = 0; e < D; e++) {
          if (e == d) continue;
          lin_id += (long long)(qq[e] - g.off[e]) * mul;
          mul *= g.n[e];
        }
        const long long fid = (side ? bb.base[2 * d + 1] : bb.base[2 * d]) + lin_id;
        for (int mv = 0; mv < g.N * NV; mv++) b.bflux[fid * g.N * NV + mv] = 0.0;
      }
    }
  }
  __syncthreads();
  const unsigned uni = s_union;
  const T eps = (T)g.weno_eps;
  const double dt = b.ctl->dt;
  unsigned err = 0;

  // a tile that may be idle (see below); in FP64, whose divisions and square
  // roots are costly, it stages the states first and derives the primitive
  // quantities only when it is not idle
  const bool cand = !anyband && interior_tile && g.geom == 0;
  const bool fast_sum = !anyband && g.geom == 0 && (D < 2 || g.rh[1] == g.rh[0]) && (D < 3 || g.rh[2] == g.rh[0]);
  const bool defer = cand && sizeof(T) == 8;
  const int sref = S::slot(0, 0, 0);
  for (int m = 0; m < g.N; m++) {
    if (!((uni >> m) & 1u)) continue;
    const T mgm1 = T(g.gm1[m]), mgpi = T(g.gpi[m]), mgam = T(g.gamma[m]), mpinf = T(g.pinf[m]);
    const TaitK mtk = tait_of(g, m);
    PosArgs pa;
    pa.on = g.positivity;
    pa.dt2d = (2.0 * D) * dt;
    pa.gm1 = g.gm1[m];
    pa.gpi = g.gpi[m];
    pa.pinf = g.pinf[m];
    pa.tait = mtk.on;
    // stage the stencil state and its primitive quantities
#pragma unroll 1
    for (int s = tid; s < NS; s += blockDim.x) {
      int lx, ly, lz;
      // only the axis-aligned halo of the tile is read by face stencils
      const bool used = S::coords(s, lx, ly, lz);
      const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
      T u[NV];
      const bool ok = used && gx >= 0 && gx < g.pn[0] && gy >= 0 && gy < g.pn[1] && gz >= 0 && gz < g.pn[2];
      if (ok) {
        const long long gc = cell_at(g, gx, gy, gz);
        bool inner = gx >= g.off[0] && gx < g.off[0] + g.n[0];
        if (D >= 2) inner = inner && gy >= g.off[1] && gy < g.off[1] + g.n[1];
        if (D >= 3) inner = inner && gz >= g.off[2] && gz < g.off[2] + g.n[2];
        if (inner) {
          if constexpr (sizeof(T) == 4) {
            if (Qsf && m != g.fs_mat) interior_uhat_f<NV>(g, b, Qsf, gc, m, u);
            else interior_uhat_n<T, NV>(g, b, Qs, gc, m, u);
          } else {
            interior_uhat_n<T, NV>(g, b, Qs, gc, m, u);
          }
        } else {
          const T* Uh = (const T*)b.Uh;
#pragma unroll
          for (int v = 0; v < NV; v++) u[v] = Uh[qidx(g, m, v, gc)];
        }
      } else {
#pragma unroll
        for (int v = 0; v < NV; v++) u[v] = (T)__longlong_as_double(0x7ff8000000000000LL);
      }
#pragma unroll
      for (int v = 0; v < NV; v++) U[v * NS + s] = u[v];
      bad[s] = 0;
      if (!isnan(u[0]) && (!defer || s == sref)) {
        T vel[D], pres, cs;
        bool isbad;
        stencil_prim<D, T>(u, mgm1, mgpi, mgam, mpinf, mtk, vel, pres, cs, isbad);
#pragma unroll
        for (int e = 0; e < D; e++) P[e * NS + s] = vel[e];
        P[D * NS + s] = pres;
        P[(D + 1) * NS + s] = cs;
        bad[s] = isbad ? 1 : 0;  // reported only if a used face reads it
      }
    }
    __syncthreads();
    // Idle tile (block-sparse skipping): a single-material tile away from the
    // domain boundary whose used stencil states are all bit-identical has
    // bit-identical face fluxes, so every aperture-weighted difference is
    // exactly +0 and L = 0; the face evaluation is skipped and the update
    // below runs with L = 0, giving the same bits as the full evaluation.
    bool idle = false;
    if (cand) {
      idle = __syncthreads_and(stencil_uniform<D, T>(U, bad, tid)) != 0;
      if (defer && !idle) {
        // not idle after all: the primitive quantities of the other staged states
#pragma unroll 1
        for (int s = tid; s < NS; s += blockDim.x) {
          if (s == sref || isnan(U[s])) continue;
          T u[NV];
#pragma unroll
          for (int v = 0; v < NV; v++) u[v] = U[v * NS + s];
          T vel[D], pres, cs;
          bool isbad;
          stencil_prim<D, T>(u, mgm1, mgpi, mgam, mpinf, mtk, vel, pres, cs, isbad);
#pragma unroll
          for (int e = 0; e < D; e++) P[e * NS + s] = vel[e];
          P[D * NS + s] = pres;
          P[(D + 1) * NS + s] = cs;
          bad[s] = isbad ? 1 : 0;
        }
        __syncthreads();
      }
    }
    // face apertures and fluxes: x faces, then y, then z
    if (!idle)
      for (int f = tid; f < S::NF; f += blockDim.x) {
        if (f < S::NFX)
          flux_face<D, T, 0>(g, b, U, P, F, A, bad, bb, f, f, x0, y0, z0, m, anyband, eps, pa, err);
        else if (D >= 2 && f < S::NFX + S::NFY)
          flux_face<D, T, 1>(g, b, U, P, F, A, bad, bb, f, f - S::NFX, x0, y0, z0, m, anyband, eps, pa, err);
        else if (D >= 3)
          flux_face<D, T, 2>(g, b, U, P, F, A, bad, bb, f, f - S::NFX - S::NFY, x0, y0, z0, m, anyband, eps, pa, err);
      }
    __syncthreads();
    // cell update
    if (inside && ((mymask >> m) & 1u)) {
      const bool cut = (b.gflag[c] & GF_CUT) != 0;
      int flo[3], fhi[3];
      flo[0] = tx + (TX + 1) * (ty + TY * tz);
      fhi[0] = flo[0] + 1;
      if (D >= 2) {
        flo[1] = S::NFX + tx + TX * (ty + (TY + 1) * tz);
        fhi[1] = flo[1] + TX;
      }
      if (D >= 3) {
        flo[2] = S::NFX + S::NFY + tx + TX * (ty + TY * tz);
        fhi[2] = flo[2] + TX * TY;
      }
      // cylindrical grid: faces weighted by their radii, volume r_i h, and the
      // source p alpha / r_i of the radial momentum (the stage's stencil state)
      const bool cyl = D == 1 && g.geom == 1;
      double rlo = 0.0, rhi = 0.0, rvc = 0.0, psrc = 0.0;
      if (cyl) {
        const double rc = cell_r(g, cx), a = alpha_of(g, b, c, m);
        rlo = face_r(g, cx);
        rhi = face_r(g, cx + 1);
        rvc = 1.0 / (rc * g.h[0]);
        if (a > 0.0) psrc = (double)P[D * NS + S::slot(tx, ty, tz)] * a / rc;
      }
#pragma unroll
      for (int v = 0; v < NV; v++) {
        double L = 0.0;
        if (cyl) {
          const double fl = (double)F[v * S::NF + flo[0]], fh = (double)F[v * S::NF + fhi[0]];
          L = (A[flo[0]] * fl * rlo - A[fhi[0]] * fh * rhi) * rvc;
          if (cut) L = L + b.X[qidx(g, m, v, c)] * rvc;
          if (v == 1) L = L + psrc;
        } else {
          if (!idle) {
            if (sizeof(T) == 4 && fast_sum) {
              // FP32-bulk form, a tile without band cells (every aperture 1)
              // on a grid with equal spacings: the FP32 face fluxes of the
              // cell summed with their exact rounding errors, converted
              // once; each face's flux enters its two cells as the same
              // float, so the sum over cells still telescopes in FP64
              float sh = 0.0f, sc = 0.0f;
#pragma unroll
              for (int d = 0; d < D; d++) {
                two_sum_acc(sh, sc, (float)F[v * S::NF + flo[d]]);
                two_sum_acc(sh, sc, -(float)F[v * S::NF + fhi[d]]);
              }
              L = (f2d_bits(sh) + f2d_bits(sc)) * g.rh[0];
            } else {
#pragma unroll
              for (int d = 0; d < D; d++) {
                const double fl = to_d(F[v * S::NF + flo[d]]), fh = to_d(F[v * S::NF + fhi[d]]);
                L = L + (A[flo[d]] * fl - A[fhi[d]] * fh) * g.rh[d];
              }
            }
          }
          if (cut) L = L + b.X[qidx(g, m, v, c)] * g.rV;
        }
        if (m == g.fs_mat) L = 0.0;  // the ambient is not solved
        const long long qi = qidx(g, m, v, c);
        const double qs = Qs[qi];
        double qv;
        if (sizeof(T) == 4 && beta == 0.0) {
          qv = qs + dt * L;  // the first stage (beta = 0, 1 - beta = 1)
        } else {
          const double qn = Qn[qi];
          qv = beta * qn + omb * (qs + dt * L);
        }
        if (!finite_bits(qv)) err |= ERR_NONFINITE;
        Qout[qi] = qv;
        if (sizeof(T) == 4 && Qof) Qof[qi] = d2f_bits(qv);
      }
    }
    __syncthreads();
  }
  if (err) atomicOr(&s_err, err);
  __syncthreads();
  if (tid == 0 && s_err) atomicOr(&b.ctl->err, s_err);
}

// FP32 copy Qf[0] of the state Q[0], read by the FP32-bulk flux update of
// stage 0 for its bulk stencil states (the values it would otherwise convert
// there). The last flux update of a step writes it for every value it
// updates; this kernel refreshes the values of the step's band cells (all
// materials and variables) after the band kernels that follow the update
// (correction, mixing, scale separation) have changed them, and, with
// band_only = 0, converts the whole state after a host-side write of Q[0].
// So Qf[0] equals Q[0] rounded to FP32 at the start of every step.
__global__ void k_qf_copy(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, int band_only) {
  if (band_only && !ctl_active(b)) return;
  const long long per = (long long)g.N * g.NV;
  const long long nb = band_only ? (long long)b.ctl->nband : 0;
  const long long total = band_only ? nb * per : g.ncell * per;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long q = i;
    if (band_only) {
      const long long mv = i / nb, k = i - mv * nb;
      q = mv * g.ncell + b.band[k];
    }
    b.Qf[0][q] = d2f_bits(b.Q[0][q]);
  }
}

// Persistent CTAs (as many as fit on the GPU at once) take tiles from a
// counter in the control block, so that the tiles holding band cells (two or
// three materials: two to three times the work) spread over every SM instead
// of leaving a partial last wave; each tile's arithmetic does not depend on
// which CTA runs it.
template <int D, typename T>
__global__ void __launch_bounds__(Tile<D>::X* Tile<D>::Y* Tile<D>::Z, sizeof(T) == 4 ? (D == 3 ? 3 : 4) : 1)
    k_flux_update(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qs,
                  const double* Qn, double* Qout, double beta, double omb, const __grid_constant__ BndBase bb,
                  int ntiles, const float* Qsf, float* Qof) {
  if (!ctl_active(b)) return;
  __shared__ int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&b.ctl->tile_ctr, 1u);
    __syncthreads();
    const int tile = s_tile;
    __syncthreads();
    if (tile >= ntiles) break;
    flux_tile<D, T>(g, b, Qs, Qn, Qout, beta, omb, bb, tile, Qsf, Qof);
  }
}

// sum of a value over the lanes of a warp, by a butterfly of exchanges in a
// fixed order (every lane gets the same bits, on every run)
__device__ __forceinline__ double warp_sum_fixed(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// sum the boundary-face fluxes of the stage into the ledger, in two fixed-order
// passes: each block adds NTHREADS faces for every (material, variable), warp
// by warp and then over its warps in order, and one block adds the partial
// sums of all blocks the same way
__global__ void k_ledger_partial(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, int nbnd) {
  if (!ctl_active(b)) return;
  const int NMV = g.N * g.NV;
  const int f = blockIdx.x * NTHREADS + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double red[NTHREADS / 32][MAXM * 5];
  for (int mv = 0; mv < NMV; mv++) {
    const double v = warp_sum_fixed(f < nbnd ? b.bflux[(long long)f * NMV + mv] : 0.0);
    if (lane == 0) red[warp][mv] = v;
  }
  __syncthreads();
  for (int mv = threadIdx.x; mv < NMV; mv += NTHREADS) {
    double s = 0.0;
    for (int w = 0; w < NTHREADS / 32; w++) s += red[w][mv];
    b.lpart[(long long)blockIdx.x * NMV + mv] = s;
  }
}
__global__ void k_ledger(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, int nparts, double w) {
  if (!ctl_active(b)) return;
  const int NMV = g.N * g.NV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double red[NTHREADS / 32][MAXM * 5];
  for (int mv = 0; mv < NMV; mv++) {
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += NTHREADS) s += b.lpart[(long long)k * NMV + mv];
    s = warp_sum_fixed(s);
    if (lane == 0) red[warp][mv] = s;
  }
  __syncthreads();
  for (int mv = threadIdx.x; mv < NMV; mv += NTHREADS) {
    double s = 0.0;
    for (int k = 0; k < NTHREADS / 32; k++) s += red[k][mv];
    b.ctl->ledger[mv / g.NV][mv % g.NV] += w * b.ctl->dt * s;
  }
}

// --------------------------------------------- level-set stage (a9) + R
__device__ inline double phir_stage(const Bufs& b, long long c, int r) { return phi_m(b.phi, b.chi, c, r); }

// With LIST the items are the (region, band cell) pairs the geometry pass
// listed (those whose region is present in the cell's 3^d block), else every
// pair, skipping the others. The upwind side is a selection of the stencil
// differences, so lanes with opposite velocity signs share one WENO5 chain.
template <int DD, bool LIST>
__device__ __forceinline__ void phase_levelset_d(const Grid& g, const Bufs& b, const double* vel, double beta, double omb, int first_, int stride_) {
    const int nb = b.ctl->nband, N = g.N, D = DD;
  const double dt = b.ctl->dt, eps = g.weno_eps;
  const int total = LIST ? (int)b.ctl->ls_count : nb * N;
  for (int it = first_; it < total; it += stride_) {
    const int code = LIST ? b.lslist[it] : it;
    const int r = code / nb, k = code - r * nb;
    const long long c = b.band[k];
    if (!LIST && !((b.xsS[c] >> r) & 1u)) continue;
    // the 7-point line of every axis, loaded up front (one round of latency)
    double pl[3][7], vdir[3];
    for (int d = 0; d < D; d++) {
      vdir[d] = vel[d * g.ncell + c];
      for (int i = 0; i < 7; i++) pl[d][i] = phir_stage(b, c + (long long)(i - 3) * g.st[d], r);
    }
    double adv = 0.0;
    for (int d = 0; d < D; d++) {
      const double vd = vdir[d];
      if (vd == 0.0) continue;
      const double rh = g.rh[d];
      const double* p = pl[d] + 3;  // p[i] = phi^r at c + i e_d
      // vd > 0: backward differences from c - 3 e_d; vd < 0: forward
      // differences from c + 3 e_d, in reverse order
      const bool up = vd > 0.0;
      const double v1 = up ? (p[-2] - p[-3]) * rh : (p[3] - p[2]) * rh;
      const double v2 = up ? (p[-1] - p[-2]) * rh : (p[2] - p[1]) * rh;
      const double v3 = up ? (p[0] - p[-1]) * rh : (p[1] - p[0]) * rh;
      const double v4 = up ? (p[1] - p[0]) * rh : (p[0] - p[-1]) * rh;
      const double v5 = up ? (p[2] - p[1]) * rh : (p[-1] - p[-2]) * rh;
      const double gd = weno5<double>(v1, v2, v3, v4, v5, eps);
      adv = adv + vd * gd;
    }
    const double phn = b.chin[c] == r ? b.phin[c] : -b.phin[c];
    b.phir[(long long)k * N + r] = beta * phn + omb * (phir_stage(b, c, r) - dt * adv);
  }
}
template <bool LIST>
__device__ __forceinline__ void phase_levelset(const Grid& g, const Bufs& b, const double* vel, double beta, double omb, int first_, int stride_) {
  if (g.D == 1) phase_levelset_d<1, LIST>(g, b, vel, beta, omb, first_, stride_);
  else if (g.D == 2) phase_levelset_d<2, LIST>(g, b, vel, beta, omb, first_, stride_);
  else phase_levelset_d<3, LIST>(g, b, vel, beta, omb, first_, stride_);
}
__global__ void k_levelset(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* vel, double beta, double omb) {
  if (!ctl_active(b)) return;
  phase_levelset<true>(g, b, vel, beta, omb, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
// reconstruction R: |max_r phi^r| and argmax (lowest index on ties), clamped
__device__ __forceinline__ void phase_levelset_R(const Grid& g, const Bufs& b, int first_, int stride_) {
    const int nb = b.ctl->nband, N = g.N;
  for (int k = first_; k < nb; k += stride_) {
    const long long c = b.band[k];
    const unsigned bits = b.xsS[c];
    double best = 0.0;
    int arg = -1;
    for (int r = 0; r < N; r++) {
      if (!((bits >> r) & 1u)) continue;
      const double val = b.phir[(long long)k * N + r];
      if (arg < 0 || val > best) {
        best = val;
        arg = r;
      }
    }
    double ph = fabs(best);
    if (ph > g.cap) ph = g.cap;
    b.phi[c] = ph;
    b.chi[c] = (uint8_t)arg;
  }
}
__global__ void k_levelset_R(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  if (!ctl_active(b)) return;
  phase_levelset_R(g, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
// scatter band-indexed (phi, chi) back; flag selects which cells are written
__device__ __forceinline__ void phase_scatter_phichi(const Grid& g, const Bufs& b, int first_, int stride_) {
    const int nb = b.ctl->nband;
  for (int k = first_; k < nb; k += stride_) {
    const long long c = b.band[k];
    b.phi[c] = b.phit[k];
    b.chi[c] = b.chit[k];
  }
}
__global__ void k_scatter_phichi(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  if (!ctl_active(b)) return;
  phase_scatter_phichi(g, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ------------------------------------------------------------ mixing (a11)
// mixing targets as axis sets: 1D x; 2D x, y, xy; 3D x, y, z, xy, xz, yz, xyz
__device__ inline int mix_axes(int D, int k) {
  const int ax2[3] = {1, 2, 3};
  const int ax3[7] = {1, 2, 4, 3, 5, 6, 7};
  return D <= 2 ? ax2[k] : ax3[k];
}

// offset code of a 3^d neighbour (dz, dy, dx in -1..1)
__device__ inline uint8_t off_code(int dx, int dy, int dz) { return (uint8_t)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)); }

// targets (offset codes) and weights of small cell c of material m; returns
// the count (0: no target)
__device__ inline int mix_targets(const Grid& g, const Bufs& b, long long c, int m, double as, uint8_t* toff,
                                  double* tw, double* swout) {
  const int D = g.D;
  double n[3];
  stored_normal(g, b, c, m, n);
  int q[3];
  coords(g, c, q);
  int sg[3];
  for (int d = 0; d < 3; d++) sg[d] = n[d] > 0.0 ? 1 : (n[d] < 0.0 ? -1 : 0);
  const int nk = D == 1 ? 1 : (D == 2 ? 3 : 7);
  int nt = 0;
  double sw = 0.0;
  for (int kk = 0; kk < nk; kk++) {
    const int ax = mix_axes(D, kk);
    bool ok = true;
    double wk = 1.0;
    int na = 0;
    int o[3] = {0, 0, 0};
    for (int d = 0; d < D; d++)
      if ((ax >> d) & 1) {
        if (sg[d] == 0) ok = false;
        o[d] = sg[d];
        wk = na == 0 ? fabs(n[d]) : wk * fabs(n[d]);
        na++;
      }
    if (na == 1) wk = wk * wk;
    if (!ok) continue;
    int p[3] = {q[0] + o[0], q[1] + o[1], q[2] + o[2]};
    if (!interior_q(g, p)) continue;
    const long long t = cell_at(g, p[0], p[1], p[2]);
    if (b.bandidx[t] < 0 || !((b.smask[t] >> m) & 1u) || !(b.alpha[midx(g, m, t)] > as)) continue;
    toff[nt] = off_code(o[0], o[1], o[2]);
    tw[nt] = wk;
    nt++;
    sw += wk;
  }
  if (!(sw > 0.0)) {
    nt = 0;
    sw = 0.0;
    const int rz = D >= 3 ? 1 : 0, ry = D >= 2 ? 1 : 0;
    for (int dz = -rz; dz <= rz; dz++)
      for (int dy = -ry; dy <= ry; dy++)
        for (int dx = -1; dx <= 1; dx++) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          int p[3] = {q[0] + dx, q[1] + dy, q[2] + dz};
          if (!interior_q(g, p)) continue;
          const long long t = cell_at(g, p[0], p[1], p[2]);
          if (b.bandidx[t] < 0 || !((b.smask[t] >> m) & 1u) || !(b.alpha[midx(g, m, t)] > as)) continue;
          toff[nt] = off_code(dx, dy, dz);
          tw[nt] = b.alpha[midx(g, m, t)];
          sw += tw[nt];
          nt++;
        }
  }
  *swout = sw;
  return (sw > 0.0) ? nt : 0;
}

__device__ inline long long off_cell(const Grid& g, long long c, uint8_t code) {
  const int dz = code / 9 - 1, dy = (code / 3) % 3 - 1, dx = code % 3 - 1;
  return c + dx + g.st[1] * dy + g.st[2] * dz;
}

__device__ inline bool is_small(const Grid& g, const Bufs& b, const double* Qc, long long c, int m, double as) {
  if (as > 0.0 && as < g.mix_alpha) return true;
  if (as == 0.0)
    for (int v = 0; v < g.NV; v++)
      if (Qc[qidx(g, m, v, c)] != 0.0) return true;
  if (as > 0.0) {  // a non-physical state (rho <= 0 or p + pinf <= 0) mixes like a small cell
    double u[5], w[5];
    // a division by 1 returns its dividend: a whole cell skips them
    for (int v = 0; v < g.NV; v++) u[v] = as == 1.0 ? Qc[qidx(g, m, v, c)] : Qc[qidx(g, m, v, c)] / as;
    cons_to_prim<double>(g, m, g.D, u, w);
    if (!(w[0] > 0.0) || !(w[g.NV - 1] + g.pinf[m] > 0.0)) return true;
  }
  return false;
}

// per (band cell, material): small-cell test and, for a small cell, its
// targets and normalised weights (mixn: 0xff not small, else target count)
__device__ __forceinline__ void phase_mix_mark(const Grid& g, const Bufs& b, const double* Qc, int first_, int stride_) {
    const int nb = b.ctl->nband, N = g.N;
  unsigned long long nsmall = 0, nfail = 0;
  const int total = nb * N;
  for (int it = first_; it < total; it += stride_) {
    const int m = it / nb, k = it - m * nb;
    const long long c = b.band[k];
    const long long r = (long long)k * N + m;
    b.mixn[r] = 0xff;
    if (!((b.smask[c] >> m) & 1u)) continue;
    const double as = b.alpha[midx(g, m, c)];
    if (!is_small(g, b, Qc, c, m, as)) continue;
    nsmall++;
    uint8_t toff[MIX_MAXT];
    double tw[MIX_MAXT], sw;
    const int nt = mix_targets(g, b, c, m, as, toff, tw, &sw);
    if (nt == 0) nfail++;
    for (int t = 0; t < nt; t++) {
      b.mixoff[r * MIX_MAXT + t] = toff[t];
      b.mixbeta[r * MIX_MAXT + t] = tw[t] / sw;
      // tell the target which neighbour (by this offset code) mixes into it
      const long long tc = off_cell(g, c, toff[t]);
      atomicOr(&b.mixin[(long long)b.bandidx[tc] * N + m], 1u << toff[t]);
    }
    b.mixn[r] = (uint8_t)nt;
  }
  if (nsmall) atomicAdd(&b.ctl->cnt[C_SMALL], nsmall);
  if (nfail) atomicAdd(&b.ctl->cnt[C_MIXFAIL], nfail);
}
__global__ void k_mix_mark(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qc) {
  if (!ctl_active(b)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) b.ctl->mix_count = 0u;  // the list is filled by k_mix_weights
  phase_mix_mark(g, b, Qc, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Weight sum T of every (band cell, material). With cell volumes V (unit on
// Cartesian grids, r on a cylindrical one) a pair moves the content
// C = beta V_s V_t (a_s Q_t - a_t Q_s) / (a_s V_s + a_t V_t): the small cell's
// per-volume state moves towards the target's with weight
// beta a_t V_t / (a_s V_s + a_t V_t) and the target's towards the small
// cell's with weight beta a_s V_s / (a_s V_s + a_t V_t).
// T sums a cell's weights: its own pairs in target order, then the pairs of
// the neighbours that mix into it in (z, y, x) offset order.
template <int DD>
__device__ __forceinline__ void phase_mix_weights_d(const Grid& g, const Bufs& b, int first_, int stride_) {
  const int nb = b.ctl->nband, N = g.N;
  const int total = nb * N;
  for (int it = first_; it < total; it += stride_) {
    const int m = it / nb, k = it - m * nb;
    const long long c = b.band[k];
    const long long r = (long long)k * N + m;
    double T = 0.0;
    if ((b.smask[c] >> m) & 1u) {
      const double ac = b.alpha[midx(g, m, c)], vc = vfac(g, c);
      const int nown = b.mixn[r];
      for (int t = 0; t < (nown == 0xff ? 0 : nown); t++) {
        const long long tc = off_cell(g, c, b.mixoff[r * MIX_MAXT + t]);
        const double at = b.alpha[midx(g, m, tc)], vt = vfac(g, tc);
        T += b.mixbeta[r * MIX_MAXT + t] * (at * vt) / (ac * vc + at * vt);
      }
      // the neighbours that mix into this cell, in (z, y, x) offset order:
      // the set bits of mixin in increasing offset code
      unsigned inbits = b.mixin[r];
      if (inbits) {
        int q[3];
        coords(g, c, q);
        while (inbits) {
          const int code = __ffs(inbits) - 1;
          inbits &= inbits - 1u;
          const int dz = code / 9 - 1, dy = (code / 3) % 3 - 1, dx = code % 3 - 1;
          const int sx = q[0] - dx, sy = q[1] - dy, sz = q[2] - dz;
          if (!in_array(g, sx, sy, sz)) continue;
          const long long s = cell_at(g, sx, sy, sz);
          const int ks = b.bandidx[s];
          if (ks < 0) continue;
          const long long rs = (long long)ks * N + m;
          const int ns = b.mixn[rs];
          if (ns == 0xff) continue;
          for (int t = 0; t < ns; t++) {
            if (b.mixoff[rs * MIX_MAXT + t] != code) continue;
            const double as = b.alpha[midx(g, m, s)], vs = vfac(g, s);
            T += b.mixbeta[rs * MIX_MAXT + t] * (as * vs) / (as * vs + ac * vc);
          }
        }
      }
    }
    b.mixT[r] = T;
  }
}
// Scale of a pair exchange from the weight sums of its two cells: when a
// cell's T exceeds one its mixed state would leave the range of the states it
// mixes with, so the pair is scaled by min(1, 1/T_s, 1/T_t) (both sides by the
// same factor, so the exchange stays conservative). A small cell without
// volume has no per-volume state to bound: its pairs stay whole.
__device__ inline double mix_limit(double as, double Ts, double Tt) {
  if (as == 0.0) return 1.0;
  double f = 1.0;
  if (Ts > 1.0) f = fmin(f, 1.0 / Ts);
  if (Tt > 1.0) f = fmin(f, 1.0 / Tt);
  return f;
}

// ---- warp-cooperative mixing pairs (grid kernels). The pairs of an item are
// its own pairs as a small cell (in target order) followed by the pairs of
// the neighbours that mix into it (in increasing offset code: the (z, y, x)
// order above). The pairs of a warp's items are numbered consecutively and
// taken 32 at a time, one per lane, so that their FP64 divisions run on full
// warps; each item's lane then combines its pairs' values in that order with
// the operations of the one-lane functions above, so the results are theirs.
struct MixPair {
  bool ok;         // the pair exists (the neighbour has a state and targets this cell)
  bool own;        // the item is the pair's small cell
  long long p;     // the other cell of the pair
  long long rp;    // its item (band index * N + material)
  double beta;     // the pair's mixing weight
};
// pair jj of item r (cell c, material m; nown own pairs, inbits incoming bits)
__device__ __forceinline__ MixPair mix_pair(const Grid& g, const Bufs& b, long long r, long long c, int m, int nown,
                                            unsigned inbits, int jj) {
  MixPair P;
  P.ok = false;
  P.own = jj < nown;
  P.p = 0;
  P.rp = 0;
  P.beta = 0.0;
  const int N = g.N;
  if (P.own) {
    P.p = off_cell(g, c, b.mixoff[r * MIX_MAXT + jj]);
    P.rp = (long long)b.bandidx[P.p] * N + m;
    P.beta = b.mixbeta[r * MIX_MAXT + jj];
    P.ok = true;
    return P;
  }
  unsigned bits = inbits;  // the (jj - nown)-th set bit, counting from the lowest
  for (int i = nown; i < jj; i++) bits &= bits - 1u;
  const int code = __ffs(bits) - 1;
  const int dz = code / 9 - 1, dy = (code / 3) % 3 - 1, dx = code % 3 - 1;
  int q[3];
  coords(g, c, q);
  const int sx = q[0] - dx, sy = q[1] - dy, sz = q[2] - dz;
  if (!in_array(g, sx, sy, sz)) return P;
  const long long sc = cell_at(g, sx, sy, sz);
  const int ks = b.bandidx[sc];
  if (ks < 0) return P;
  const long long rs = (long long)ks * N + m;
  const int ns = b.mixn[rs];
  if (ns == 0xff) return P;
  for (int t = 0; t < ns; t++)  // a small cell's targets have distinct offsets
    if (b.mixoff[rs * MIX_MAXT + t] == code) {
      P.beta = b.mixbeta[rs * MIX_MAXT + t];
      P.ok = true;
      break;
    }
  P.p = sc;
  P.rp = rs;
  return P;
}
// per-lane table of the warp's items, read by the lanes that evaluate their pairs
struct MixItemSm {
  long long r, c;
  int m, nown, pre;
  unsigned inbits;
};
// exclusive prefix sum of the lanes' pair counts, and the warp's total
__device__ __forceinline__ int warp_excl_scan(int P, int lane, int& tot) {
  int incl = P;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  tot = __shfl_sync(0xffffffffu, incl, 31);
  return incl - P;
}
// mark the lanes of round rb whose pairs belong to this lane's item
__device__ __forceinline__ void mix_owner_map(uint8_t* owner, int pre, int P, int rb, int lane) {
  const int j0 = pre > rb ? pre : rb, j1 = pre + P < rb + 32 ? pre + P : rb + 32;
  for (int j = j0; j < j1; j++) owner[j - rb] = (uint8_t)lane;
}

// weight sums T and the list of the items that mix (grid kernel; first_ and
// stride_ warp-aligned, blockDim.x == BAND_THREADS)
__device__ __forceinline__ void mix_weights_coop(const Grid& g, const Bufs& b, int first_, int stride_) {
  __shared__ MixItemSm s_it[BAND_THREADS];
  __shared__ uint8_t s_own[BAND_THREADS];
  __shared__ double s_val[BAND_THREADS];
  __shared__ uint8_t s_ok[BAND_THREADS];
  const int nb = b.ctl->nband, N = g.N;
  const int total = nb * N;
  const int lane = threadIdx.x & 31, wb = threadIdx.x - lane;
  for (int base = first_ - lane; base < total; base += stride_) {
    const int it = base + lane;
    const bool valid = it < total;
    int m = 0, nown = 0, P = 0;
    long long c = 0, r = 0;
    unsigned inbits = 0;
    if (valid) {
      m = it / nb;
      const int k = it - m * nb;
      c = b.band[k];
      r = (long long)k * N + m;
      const int mn = b.mixn[r];
      const unsigned mi = b.mixin[r];
      if (mn != 0xff || mi != 0u) {
        // an item that mixes: small, or a target of a small neighbour
        b.mixlist[atomicAdd(&b.ctl->mix_count, 1u)] = (int)r;
        b.mixtouch[k] = 1;
      }
      if ((b.smask[c] >> m) & 1u) {
        nown = mn == 0xff ? 0 : mn;
        inbits = mi;
        P = nown + __popc(mi);
      }
    }
    int tot;
    const int pre = warp_excl_scan(P, lane, tot);
    s_it[threadIdx.x] = MixItemSm{r, c, m, nown, pre, inbits};
    double T = 0.0;
    for (int rb = 0; rb < tot; rb += 32) {
      __syncwarp();
      mix_owner_map(s_own + wb, pre, P, rb, lane);
      __syncwarp();
      double val = 0.0;
      bool ok = false;
      if (rb + lane < tot) {
        const MixItemSm o = s_it[wb + s_own[wb + lane]];
        const MixPair pr = mix_pair(g, b, o.r, o.c, o.m, o.nown, o.inbits, rb + lane - o.pre);
        if (pr.ok) {
          ok = true;
          const double ac = b.alpha[midx(g, o.m, o.c)], vc = vfac(g, o.c);
          const double ap = b.alpha[midx(g, o.m, pr.p)], vp = vfac(g, pr.p);
          val = pr.own ? pr.beta * (ap * vp) / (ac * vc + ap * vp) : pr.beta * (ap * vp) / (ap * vp + ac * vc);
        }
      }
      s_val[threadIdx.x] = val;
      s_ok[threadIdx.x] = ok ? 1 : 0;
      __syncwarp();
      const int j0 = pre > rb ? pre : rb, j1 = pre + P < rb + 32 ? pre + P : rb + 32;
      for (int j = j0; j < j1; j++)
        if (s_ok[wb + j - rb]) T += s_val[wb + j - rb];
    }
    if (valid) b.mixT[r] = T;
  }
}

// mixed states of the listed items into mixq (grid kernel; first_ and stride_
// warp-aligned, blockDim.x == BAND_THREADS)
template <int DD>
__device__ __forceinline__ void mix_compute_coop(const Grid& g, const Bufs& b, const double* Qc, int first_,
                                                 int stride_) {
  constexpr int NV = DD + 2;
  __shared__ MixItemSm s_it[BAND_THREADS];
  __shared__ uint8_t s_own[BAND_THREADS];
  __shared__ double s_x[NV][BAND_THREADS];
  __shared__ double s_f[BAND_THREADS], s_mul[BAND_THREADS];
  __shared__ int8_t s_sg[BAND_THREADS];
  const int N = g.N, total = (int)b.ctl->mix_count;
  const int lane = threadIdx.x & 31, wb = threadIdx.x - lane;
  for (int base = first_ - lane; base < total; base += stride_) {
    const int it = base + lane;
    const bool valid = it < total;
    int m = 0, nown = 0, P = 0;
    long long c = 0, r = 0;
    unsigned inbits = 0;
    bool live = false;
    if (valid) {
      r = b.mixlist[it];
      const int k = (int)(r / N);
      m = (int)(r - (long long)k * N);
      c = b.band[k];
      live = (b.smask[c] >> m) & 1u;
      if (!live) {
        for (int v = 0; v < NV; v++) b.mixq[r * NV + v] = Qc[qidx(g, m, v, c)];
      } else {
        const int mn = b.mixn[r];
        if (mn != 0xff) {
          nown = mn;
          if (mn == 0 && b.alpha[midx(g, m, c)] == 0.0 && m != b.chi[c]) atomicOr(&b.mixmerge[k], 1u << m);
        }
        inbits = b.mixin[r];
        P = nown + __popc(inbits);
      }
    }
    int tot;
    const int pre = warp_excl_scan(P, lane, tot);
    s_it[threadIdx.x] = MixItemSm{r, c, m, nown, pre, inbits};
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) acc[v] = 0.0;
    for (int rb = 0; rb < tot; rb += 32) {
      __syncwarp();
      mix_owner_map(s_own + wb, pre, P, rb, lane);
      __syncwarp();
      int8_t sg = 0;
      if (rb + lane < tot) {
        const MixItemSm o = s_it[wb + s_own[wb + lane]];
        const MixPair pr = mix_pair(g, b, o.r, o.c, o.m, o.nown, o.inbits, rb + lane - o.pre);
        if (pr.ok) {
          // small cell s and target t of the pair: the item is s (own) or t
          const long long cs = pr.own ? o.c : pr.p, ct = pr.own ? pr.p : o.c;
          const double as = b.alpha[midx(g, o.m, cs)], vs = vfac(g, cs);
          const double at = b.alpha[midx(g, o.m, ct)], vt = vfac(g, ct);
          const double f = pr.own ? mix_limit(as, b.mixT[o.r], b.mixT[pr.rp]) : mix_limit(as, b.mixT[pr.rp], b.mixT[o.r]);
#pragma unroll
          for (int v = 0; v < NV; v++)
            s_x[v][threadIdx.x] = (pr.beta * (as * Qc[qidx(g, o.m, v, ct)] - at * Qc[qidx(g, o.m, v, cs)])) / (as * vs + at * vt);
          s_f[threadIdx.x] = f;
          s_mul[threadIdx.x] = pr.own ? vt : vs;
          sg = pr.own ? 1 : -1;
        }
      }
      s_sg[threadIdx.x] = sg;
      __syncwarp();
      const int j0 = pre > rb ? pre : rb, j1 = pre + P < rb + 32 ? pre + P : rb + 32;
      for (int j = j0; j < j1; j++) {
        const int sl = wb + j - rb;
        const int8_t sj = s_sg[sl];
        if (sj == 0) continue;
        const double f = s_f[sl], mul = s_mul[sl];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          const double x = f * (s_x[v][sl] * mul);
          acc[v] = sj > 0 ? acc[v] + x : acc[v] - x;
        }
      }
    }
    if (valid && live)
      for (int v = 0; v < NV; v++) b.mixq[r * NV + v] = Qc[qidx(g, m, v, c)] + acc[v];
  }
}

// grid kernel: also lists the items that mix, for k_mix_compute and k_mix_scatter
__global__ void k_mix_weights(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  if (!ctl_active(b)) return;
  mix_weights_coop(g, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}


// new state of material m of every band cell: own exchanges minus the
// exchanges its small neighbours send to it (lexicographic neighbour order),
// each scaled by mix_limit
template <int DD>
__device__ __forceinline__ void mix_compute_item(const Grid& g, const Bufs& b, const double* Qc, int k, int m) {
    const int N = g.N, NV = DD + 2;
  {
    const long long c = b.band[k];
    const long long r = (long long)k * N + m;
    double* out = b.mixq + r * NV;
    if (!((b.smask[c] >> m) & 1u)) {
      for (int v = 0; v < NV; v++) out[v] = Qc[qidx(g, m, v, c)];
      return;
    }
    int q[3];
    coords(g, c, q);
    double acc[5] = {0, 0, 0, 0, 0};
    const int nown = b.mixn[r];
    if (nown != 0xff) {
      const double as = b.alpha[midx(g, m, c)];
      if (nown == 0 && as == 0.0 && m != b.chi[c]) atomicOr(&b.mixmerge[k], 1u << m);
      const double Tc = b.mixT[r], vs = vfac(g, c);
      for (int t = 0; t < (nown == 0xff ? 0 : nown); t++) {
        const long long tc = off_cell(g, c, b.mixoff[r * MIX_MAXT + t]);
        const double beta = b.mixbeta[r * MIX_MAXT + t];
        const double at = b.alpha[midx(g, m, tc)], vt = vfac(g, tc);
        const double f = mix_limit(as, Tc, b.mixT[(long long)b.bandidx[tc] * N + m]);
        for (int v = 0; v < NV; v++)
          acc[v] += f * ((beta * (as * Qc[qidx(g, m, v, tc)] - at * Qc[qidx(g, m, v, c)]) / (as * vs + at * vt)) * vt);
      }
    }
    // neighbours that mix into this cell (bits set by the marking pass), in
    // (z, y, x) offset order: the set bits in increasing offset code, so that
    // the lanes of a warp take their k-th neighbour together
    unsigned inbits = b.mixin[r];
    while (inbits) {
      const int code = __ffs(inbits) - 1;
      inbits &= inbits - 1u;
      const int dz = code / 9 - 1, dy = (code / 3) % 3 - 1, dx = code % 3 - 1;
      const int sx = q[0] - dx, sy = q[1] - dy, sz = q[2] - dz;
      if (!in_array(g, sx, sy, sz)) continue;
      const long long s = cell_at(g, sx, sy, sz);
      const int ks = b.bandidx[s];
      if (ks < 0) continue;
      const long long rs = (long long)ks * N + m;
      const int ns = b.mixn[rs];
      if (ns == 0xff) continue;
      for (int t = 0; t < ns; t++) {
        if (b.mixoff[rs * MIX_MAXT + t] != code) continue;
        const double beta = b.mixbeta[rs * MIX_MAXT + t];
        const double as = b.alpha[midx(g, m, s)], vs = vfac(g, s);
        const double at = b.alpha[midx(g, m, c)], vt = vfac(g, c);
        const double f = mix_limit(as, b.mixT[rs], b.mixT[r]);
        for (int v = 0; v < NV; v++)
          acc[v] -= f * ((beta * (as * Qc[qidx(g, m, v, c)] - at * Qc[qidx(g, m, v, s)]) / (as * vs + at * vt)) * vs);
      }
    }
    for (int v = 0; v < NV; v++) out[v] = Qc[qidx(g, m, v, c)] + acc[v];
  }
}
// every (band cell, material): the mixed state into mixq
template <int DD>
__device__ __forceinline__ void phase_mix_compute_d(const Grid& g, const Bufs& b, const double* Qc, int first_, int stride_) {
  const int nb = b.ctl->nband, N = g.N;
  const int total = nb * N;
  for (int it = first_; it < total; it += stride_) {
    const int m = it / nb, k = it - m * nb;
    mix_compute_item<DD>(g, b, Qc, k, m);
  }
}
// grid kernel: only the listed items (a fifth of the band or less; the others
// keep their state), their pairs spread over the lanes of each warp
__global__ void k_mix_compute(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* Qc) {
  if (!ctl_active(b)) return;
  const int first = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  if (g.D == 1) mix_compute_coop<1>(g, b, Qc, first, stride);
  else if (g.D == 2) mix_compute_coop<2>(g, b, Qc, first, stride);
  else mix_compute_coop<3>(g, b, Qc, first, stride);
}
// write the mixed states back; a material that lost all volume and has no
// same-material neighbour is merged into the cell's primary material
template <bool LIST>
__device__ __forceinline__ void phase_mix_scatter(const Grid& g, const Bufs& b, double* Qc, int first_, int stride_) {
    const int nb = b.ctl->nband, N = g.N, NV = g.NV;
  unsigned long long nmerge = 0;
  for (int k = first_; k < nb; k += stride_) {
    const long long c = b.band[k];
    double* in = b.mixq + (long long)k * N * NV;
    if (LIST) {
      // only cells with a listed item changed; the unlisted materials of such
      // a cell keep their state (mixq holds the listed ones only)
      if (!b.mixtouch[k]) continue;
      b.mixtouch[k] = 0;
      for (int m = 0; m < N; m++) {
        const long long r = (long long)k * N + m;
        if (b.mixn[r] == 0xff && b.mixin[r] == 0u)
          for (int v = 0; v < NV; v++) in[m * NV + v] = Qc[qidx(g, m, v, c)];
      }
    }
    const unsigned mb = b.mixmerge[k];
    if (mb) {
      const int pm = b.chi[c];
      for (int m = 0; m < N; m++) {
        if (!((mb >> m) & 1u)) continue;
        for (int v = 0; v < NV; v++) {
          in[pm * NV + v] = in[pm * NV + v] + in[m * NV + v];
          in[m * NV + v] = 0.0;
        }
        nmerge++;
      }
      b.mixmerge[k] = 0;
    }
    for (int m = 0; m < N; m++) {
      for (int v = 0; v < NV; v++) Qc[qidx(g, m, v, c)] = in[m * NV + v];
      b.mixin[(long long)k * N + m] = 0u;  // ready for the next marking pass
    }
  }
  if (nmerge) atomicAdd(&b.ctl->cnt[C_MERGE], nmerge);
}
__global__ void k_mix_scatter(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, double* Qc) {
  if (!ctl_active(b)) return;
  phase_mix_scatter<true>(g, b, Qc, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ------------------------------------------------- scale separation (a12)
// first_ and stride_ must be warp-aligned (lane l of a warp starts at a
// multiple of 32 plus l, stride a multiple of 32): the test of a candidate's
// 3^d block runs on the lanes of its warp, one block cell per lane.
__device__ __forceinline__ void phase_scale_sep(const Grid& g, const Bufs& b, double* Q, int first_, int stride_) {
    const int nb = b.ctl->nband, N = g.N, D = g.D;
  const double eps = g.eps_ss;
  unsigned long long nodd = 0, nmove = 0;
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const int rz = D >= 3 ? 1 : 0, ry = D >= 2 ? 1 : 0;
  const int nblock = (2 * rz + 1) * (2 * ry + 1) * 3;  // cells of the 3^d block
  for (int base = first_ - lane; base < nb; base += stride_) {
    const int k = base + lane;
    long long c = 0;
    int chi1 = 0;
    bool cand = false;
    if (k < nb) {
      c = b.band[k];
      b.phit[k] = b.phi[c];
      b.chit[k] = b.chi[c];
      if (b.gflag[c] & GF_MIXED) {
        int np = 0;
        for (int m = 0; m < N; m++)
          if (present(g, b, c, m)) np++;
        cand = np >= 2;
        chi1 = b.chi[c];
      }
    }
    // near_minus: some cell of the candidate's 3^d block whose simplex values
    // of phi^chi1 reach eps from both sides (an OR over the block): the cell
    // itself first, on its own lane (it holds two materials: usually a hit),
    // then the whole block of the remaining candidates, taken by the warp's
    // lanes together for each candidate in turn
    bool near_minus = false;
    if (cand) {
      double mn, mx;
      vertex_minmax(g, b.phi, b.chi, c, chi1, &mn, &mx);
      near_minus = mn - eps <= 0.0 && mx - eps >= 0.0;
    }
    unsigned pend = __ballot_sync(FULL, cand && !near_minus);
    while (pend) {
      const int src = __ffs(pend) - 1;
      pend &= pend - 1u;
      const long long cs = __shfl_sync(FULL, c, src);
      const int ch = __shfl_sync(FULL, chi1, src);
      bool hit = false;
      if (lane < nblock) {
        const int dx = lane % 3 - 1, dy = (lane / 3) % (2 * ry + 1) - ry, dz = lane / (3 * (2 * ry + 1)) - rz;
        double mn, mx;
        vertex_minmax(g, b.phi, b.chi, cs + dx + g.st[1] * dy + g.st[2] * dz, ch, &mn, &mx);
        hit = mn - eps <= 0.0 && mx - eps >= 0.0;
      }
      const bool any = __ballot_sync(FULL, hit) != 0u;
      if (lane == src) near_minus = any;
    }
    if (!cand) continue;
    int q[3];
    coords(g, c, q);
    if (near_minus) continue;
    nodd++;
    int chs = -1;
    for (int m = 0; m < N; m++) {
      if (m == chi1 || !((b.xsS[c] >> m) & 1u)) continue;
      if (chs < 0 || b.alpha[midx(g, m, c)] > b.alpha[midx(g, chs, c)]) chs = m;
    }
    double dmin = 0.0;
    bool found = false;
    const int sz = D >= 3 ? 3 : 0, sy = D >= 2 ? 3 : 0;
    for (int dz = -sz; dz <= sz; dz++)
      for (int dy = -sy; dy <= sy; dy++)
        for (int dx = -3; dx <= 3; dx++) {
          int p[3] = {q[0] + dx, q[1] + dy, q[2] + dz};
          if (!interior_q(g, p)) continue;
          const long long i0 = cell_at(g, p[0], p[1], p[2]);
          double mn, mx;
          vertex_minmax(g, b.phi, b.chi, i0, chs, &mn, &mx);
          if (!(mn + eps <= 0.0 && mx + eps >= 0.0)) continue;
          double n[3];
          normal_m(g, b.phi, b.chi, i0, chs, n);
          const double ps = phi_m(b.phi, b.chi, i0, chs);
          double dd = 0.0;
          for (int d = 0; d < D; d++) {
            const double xi0 = g.lo[d] + ((double)(p[d] - g.off[d]) + 0.5) * g.h[d];
            const double xc = g.lo[d] + ((double)(q[d] - g.off[d]) + 0.5) * g.h[d];
            const double pd = xi0 - (ps + eps) * n[d];
            const double df = xc - pd;
            dd += df * df;
          }
          dd = sqrt(dd);
          if (!found || dd < dmin) {
            dmin = dd;
            found = true;
          }
        }
    if (found) b.phit[k] = fabs(dmin - eps);
    b.chit[k] = (uint8_t)chs;
    // the cell now belongs to chi_1*; when chi_1* holds no content in it, the
    // content of chi_1 becomes chi_1*'s (totals kept, counted with the merges)
    if (Q[qidx(g, chs, 0, c)] == 0.0 && Q[qidx(g, chi1, 0, c)] > 0.0) {
      for (int v = 0; v < g.NV; v++) {
        Q[qidx(g, chs, v, c)] = Q[qidx(g, chi1, v, c)];
        Q[qidx(g, chi1, v, c)] = 0.0;
      }
      nmove++;
    }
  }
  if (nodd) atomicAdd(&b.ctl->cnt[C_ODDBALL], nodd);
  if (nmove) atomicAdd(&b.ctl->cnt[C_MERGE], nmove);
}
__global__ void k_scale_sep(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, double* Q) {
  if (!ctl_active(b)) return;
  phase_scale_sep(g, b, Q, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// --------------------------------------------- band distance maintenance
template <int DD>
__device__ __forceinline__ void reinit_items_d(const Grid& g, const Bufs& b, int first, int stride) {
  const int nb = b.ctl->nband, D = DD;
  for (int k = first; k < nb; k += stride) {
    const long long c = b.band[k];
    b.phit[k] = b.phi[c];
    b.chit[k] = b.chi[c];
    int q[3];
    coords(g, c, q);
    unsigned bits = 0;
    const int rz = D >= 3 ? 1 : 0, ry = D >= 2 ? 1 : 0;
    for (int dz = -rz; dz <= rz; dz++)
      for (int dy = -ry; dy <= ry; dy++)
        for (int dx = -1; dx <= 1; dx++)
          if (in_array(g, q[0] + dx, q[1] + dy, q[2] + dz))
            bits |= 1u << b.chi[cell_at(g, q[0] + dx, q[1] + dy, q[2] + dz)];
    if (popcount8(bits) >= 2) continue;
    double a[3] = {0, 0, 0}, hh[3] = {1, 1, 1}, w[3] = {1, 1, 1};
    for (int d = 0; d < D; d++) {
      const long long jm = c - g.st[d], jp = c + g.st[d];
      const double vm = interior_c(g, jm) ? b.phi[jm] : b.phi[c];
      const double vp = interior_c(g, jp) ? b.phi[jp] : b.phi[c];
      a[d] = fmin(vm, vp);
      hh[d] = g.h[d];
      w[d] = g.ih2[d];
    }
    for (int i = 1; i < D; i++)
      for (int j = i; j > 0 && a[j] < a[j - 1]; j--) {
        double t = a[j]; a[j] = a[j - 1]; a[j - 1] = t;
        t = hh[j]; hh[j] = hh[j - 1]; hh[j - 1] = t;
        t = w[j]; w[j] = w[j - 1]; w[j - 1] = t;
      }
    double ph = a[0] + hh[0];
    for (int kk = 1; kk < D; kk++) {
      if (ph <= a[kk]) break;
      double A = 0.0, B = 0.0, C = -1.0;
      for (int j = 0; j <= kk; j++) {
        A += w[j];
        B += w[j] * a[j];
        C += w[j] * a[j] * a[j];
      }
      const double disc = B * B - A * C;
      ph = (B + sqrt(disc > 0.0 ? disc : 0.0)) / A;
    }
    if (ph > g.cap) ph = g.cap;
    b.phit[k] = ph;
  }
}
__device__ __forceinline__ void reinit_items(const Grid& g, const Bufs& b, int first, int stride) {
  if (g.D == 1) reinit_items_d<1>(g, b, first, stride);
  else if (g.D == 2) reinit_items_d<2>(g, b, first, stride);
  else reinit_items_d<3>(g, b, first, stride);
}
__device__ __forceinline__ void scatter_items(const Bufs& b, int first, int stride) {
  const int nb = b.ctl->nband;
  for (int k = first; k < nb; k += stride) {
    const long long c = b.band[k];
    b.phi[c] = b.phit[k];
    b.chi[c] = b.chit[k];
  }
}
__global__ void k_reinit(const __grid_constant__ Grid g, const __grid_constant__ Bufs b) {
  if (!ctl_active(b)) return;
  reinit_items(g, b, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
// ------------------------------------------------------- totals and init
// one block per (m, v): fixed-order reduction over interior cells (strided
// per-thread sums, a butterfly in each warp, then the warps in order)
__global__ void k_totals(const __grid_constant__ Grid g, const double* Q, double* out) {
  const int mv = blockIdx.x;
  const int m = mv / g.NV, v = mv % g.NV;
  double s = 0.0;
  for (long long idx = threadIdx.x; idx < g.n_interior; idx += blockDim.x) {
    const long long c = interior_cell(g, idx);
    s += g.geom == 1 ? Q[qidx(g, m, v, c)] * vfac(g, c) : Q[qidx(g, m, v, c)];
  }
  s = warp_sum_fixed(s);
  __shared__ double red[NTHREADS / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
    out[mv] = t * g.V;
  }
}

// The free-surface ambient is not solved: its conserved state is
// alpha (fs_rho, 0, p(t)) with t = 0 (k = -2), the step's start (k = -1) or
// the time of stage k of the step.
__device__ __forceinline__ void phase_hold(const Grid& g, const Bufs& b, double* Qc, int k, long long first,
                                           long long stride) {
  const int F = g.fs_mat;
  if (F < 0) return;
  const double t = k == -2 ? 0.0 : (k == -1 ? b.ctl->t : b.ctl->t + g.rk_c[k] * b.ctl->dt);
  double w[5] = {0, 0, 0, 0, 0}, u[5];
  w[0] = g.fs_rho;
  w[g.D + 1] = fs_pressure(g, t);
  prim_to_cons<double>(g, F, g.D, w, u);
  for (long long idx = first; idx < g.n_interior; idx += stride) {
    const long long c = interior_cell(g, idx);
    const double a = alpha_of(g, b, c, F);
    for (int v = 0; v < g.NV; v++) Qc[qidx(g, F, v, c)] = a * u[v];
  }
}
__global__ void k_hold_ambient(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, double* Qc, int k) {
  if (k >= -1 && !ctl_active(b)) return;
  phase_hold(g, b, Qc, k, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}


// --------------------------------------------------- batched 1D instances
// One CTA owns one 1D instance and runs whole steps with block barriers
// between the phases: every phase calls the same per-item functions as the
// grid kernels, so each instance gets the grid path's arithmetic.

// aperture and WENO5-LLF flux of every face of a 1D instance (global-memory
// stencils; same arithmetic as the tiled kernel)
template <typename T>
__device__ __forceinline__ void flux1d_faces(const Grid& g, const Bufs& b, const double* Qs, T* Ff, double* Af,
                                             const BndBase& bb, int first, int stride, unsigned& err) {
  constexpr int NV = 3;
  const int N = g.N, n = g.n[0], nf = n + 1, off = g.off[0];
  const T eps = (T)g.weno_eps;
  for (int it = first; it < nf * N; it += stride) {
    const int m = it / nf, f = it - m * nf;
    const long long cR = off + f, cL = cR - 1;
    const bool lin = f >= 1, rin = f < n;
    const unsigned um = (lin ? b.smask[cL] : 0u) | (rin ? b.smask[cR] : 0u);
    double Af_ = 0.0;
    T Fh[NV] = {T(0), T(0), T(0)};
    if ((um >> m) & 1u) {
      Af_ = face_aperture(g, b, cL, cR, 0, m);
      if (Af_ > 0.0 && m != g.fs_mat) {
        if ((lin && !((b.smask[cL] >> m) & 1u)) || (rin && !((b.smask[cR] >> m) & 1u))) err |= ERR_BAND;
        const T mgm1 = T(g.gm1[m]), mgpi = T(g.gpi[m]), mgam = T(g.gamma[m]), mpinf = T(g.pinf[m]);
        const TaitK mtk = tait_of(g, m);
        T u[6][NV], un[6], pr[6], cs[6];
        bool avail = true, isbad = false;
        for (int q = 0; q < 6; q++) {
          const long long k = cL + (q - 2);
          const bool inner = k >= off && k < off + n;
          if (inner) {
            interior_uhat<T>(g, b, Qs, k, m, u[q]);
          } else {
            const T* Uh = (const T*)b.Uh;
            for (int v = 0; v < NV; v++) u[q][v] = Uh[qidx(g, m, v, k)];
          }
          if (isnan(u[q][0])) {
            avail = false;
            continue;
          }
          T vel[1];
          bool bq;
          stencil_prim<1, T>(u[q], mgm1, mgpi, mgam, mpinf, mtk, vel, pr[q], cs[q], bq);
          un[q] = vel[0];
          isbad = isbad || bq;
        }
        if (!avail) {
          err |= ERR_BAND;
        } else {
          if (isbad) err |= ERR_NEGATIVE;
          const T a = face_flux_regs<1, T>(u, un, pr, cs, 0, eps, Fh);
          if (g.positivity) {
            PosArgs pa;
            pa.on = 1;
            pa.dt2d = 2.0 * b.ctl->dt;
            pa.gm1 = g.gm1[m];
            pa.gpi = g.gpi[m];
            pa.pinf = g.pinf[m];
            pa.tait = mtk.on;
            pp_limit<1, T>(u[2], u[3], un[2], un[3], pr[2], pr[3], a, 0, pa, (T)(pa.dt2d * g.rh[0]), Fh);
          }
        }
      }
    }
    Af[(long long)m * nf + f] = Af_;
    for (int v = 0; v < NV; v++) Ff[((long long)m * NV + v) * nf + f] = Fh[v];
    if (f == 0 || f == n) {
      const long long fid = f == 0 ? bb.base[0] : bb.base[1];
      const double sgn = f == 0 ? 1.0 : -1.0;
      const double fa = g.geom == 1 ? face_r(g, off + f) : g.farea[0];
      for (int v = 0; v < NV; v++) b.bflux[((fid * g.N) + m) * NV + v] = sgn * (Af_ * (double)Fh[v] * fa);
    }
  }
}

// RK stage update of every (cell, material) of a 1D instance
template <typename T>
__device__ __forceinline__ void flux1d_update(const Grid& g, const Bufs& b, const double* Qs, const double* Qn,
                                              double* Qout, double beta, double omb, const T* Ff, const double* Af,
                                              int first, int stride, unsigned& err) {
  constexpr int NV = 3;
  const int N = g.N, n = g.n[0], nf = n + 1, off = g.off[0];
  const double dt = b.ctl->dt;
  for (int it = first; it < n * N; it += stride) {
    const int m = it / n, i = it - m * n;
    const long long c = off + i;
    if (!((b.smask[c] >> m) & 1u)) continue;
    const bool cut = (b.gflag[c] & GF_CUT) != 0;
    // cylindrical grid: faces weighted by their radii, volume r_i h, and the
    // source p alpha / r_i of the radial momentum (the stage's stencil state)
    const bool cyl = g.geom == 1;
    double rlo = 0.0, rhi = 0.0, rvc = 0.0, psrc = 0.0;
    if (cyl) {
      const double rc = cell_r(g, (int)c), a = alpha_of(g, b, c, m);
      rlo = face_r(g, (int)c);
      rhi = face_r(g, (int)c + 1);
      rvc = 1.0 / (rc * g.h[0]);
      if (a > 0.0) {
        T u[NV], w[NV];
        interior_uhat<T>(g, b, Qs, c, m, u);
        cons_to_prim<T>(g, m, 1, u, w);
        psrc = (double)w[2] * a / rc;
      }
    }
    for (int v = 0; v < NV; v++) {
      double L = 0.0;
      const double fl = (double)Ff[((long long)m * NV + v) * nf + i], fh = (double)Ff[((long long)m * NV + v) * nf + i + 1];
      if (cyl) {
        L = (Af[(long long)m * nf + i] * fl * rlo - Af[(long long)m * nf + i + 1] * fh * rhi) * rvc;
        if (cut) L = L + b.X[qidx(g, m, v, c)] * rvc;
        if (v == 1) L = L + psrc;
      } else {
        L = L + (Af[(long long)m * nf + i] * fl - Af[(long long)m * nf + i + 1] * fh) * g.rh[0];
        if (cut) L = L + b.X[qidx(g, m, v, c)] * g.rV;
      }
      if (m == g.fs_mat) L = 0.0;  // the ambient is not solved
      const long long qi = qidx(g, m, v, c);
      const double qv = beta * Qn[qi] + omb * (Qs[qi] + dt * L);
      if (!isfinite(qv)) err |= ERR_NONFINITE;
      Qout[qi] = qv;
    }
  }
}

template <typename T, int BS>
__global__ void __launch_bounds__(BS) k_batched(const BatchEntry* tab, const int* order, int n_steps) {
  const BatchEntry& E = tab[order[blockIdx.x]];
  const Grid& g = E.g;
  const Bufs& b = E.b;
  const int t = threadIdx.x, nt = BS;
  T* Ff = (T*)E.Fface;
  double* Af = E.Aface;
  for (int step = 0; step < n_steps; step++) {
    if (t == 0) {
      Ctl* c = b.ctl;
      c->active = (c->t < c->t_end && c->err == 0) ? 1 : 0;
      c->nband = 0;
      c->lam_bits = 0ull;
    }
    __syncthreads();
    if (!*(volatile int*)&b.ctl->active) break;
    phase_bc_phichi(g, b, t, nt);
    __syncthreads();
    phase_xs(g, b, t, nt);
    __syncthreads();
    phase_dilate(g, b, b.xs, b.mtmp, 0, t, nt);
    __syncthreads();
    phase_band(g, b, b.mtmp, t, nt);
    __syncthreads();
    phase_geom_mat_d<1>(g, b, t, nt);
    __syncthreads();
    phase_geom_cell<false>(g, b, b.Q[0], (const double*)nullptr, t, nt);
    __syncthreads();
    if (g.fs_mat >= 0) {
      phase_hold(g, b, b.Q[0], -1, t, nt);
      __syncthreads();
    }
    phase_band_save(g, b, t, nt);
    __syncthreads();
    for (int s = 0; s < g.rk; s++) {
      const double* Qs = b.Q[s];
      double* Qo = s == g.rk - 1 ? b.Q[0] : b.Q[s + 1];
      const double beta = g.rk_beta[s];
      phase_prim<T>(g, b, Qs, t, nt);
      __syncthreads();
      int cur = 0;
      for (int k = 0; k < g.ext_sweeps; k++) {
        if (cur) extend_items_d<T, 1>(g, b, b.W1, b.W0, b.f1, b.f0, t, nt);
        else extend_items_d<T, 1>(g, b, b.W0, b.W1, b.f0, b.f1, t, nt);
        cur ^= 1;
        __syncthreads();
      }
      phase_cons<T>(g, b, Qs, cur ? b.W1 : b.W0, cur ? b.f1 : b.f0, t, nt);
      __syncthreads();
      phase_bc_uhat_d<T, 1>(g, b, Qs, t, nt);
      __syncthreads();
      // the exchange of stage 0 comes first: the bound of the step reads the
      // free-surface velocities it sets
      phase_interface_d<T, 1>(g, b, Qs, s, t, nt);
      __syncthreads();
      if (s == 0) {
        unsigned err = 0;
        const double lam = block_max(dt_items_d<T, 1>(g, b, Qs, t, nt, err));
        if (err) atomicOr(&b.ctl->err, err);
        if (t == 0) {
          Ctl* c = b.ctl;
          c->lam = lam;
          double dt = g.cfl / lam;
          int last = 0;
          if (c->t + dt >= c->t_end) {
            dt = c->t_end - c->t;
            last = 1;
          }
          c->dt = dt;
          c->last = last;
        }
        __syncthreads();
      }
      int vc = 0;
      for (int k = 0; k < g.vel_sweeps; k++) {
        if (vc) extend_vel_items_d<1>(g, b, b.vel1, b.vel0, b.vf1, b.vf0, t, nt);
        else extend_vel_items_d<1>(g, b, b.vel0, b.vel1, b.vf0, b.vf1, t, nt);
        vc ^= 1;
        __syncthreads();
      }
      unsigned err = 0;
      flux1d_faces<T>(g, b, Qs, Ff, Af, E.bb, t, nt, err);
      __syncthreads();
      flux1d_update<T>(g, b, Qs, b.Q[0], Qo, beta, 1.0 - beta, Ff, Af, t, nt, err);
      if (err) atomicOr(&b.ctl->err, err);
      __syncthreads();
      for (int mv = t; mv < g.N * g.NV; mv += nt) {
        double sum = 0.0;
        for (int f = 0; f < E.nbnd; f++) sum += b.bflux[(long long)f * g.N * g.NV + mv];
        b.ctl->ledger[mv / g.NV][mv % g.NV] += g.rk_lw[s] * b.ctl->dt * sum;
      }
      __syncthreads();
      phase_levelset_d<1, false>(g, b, vc ? b.vel1 : b.vel0, beta, 1.0 - beta, t, nt);
      __syncthreads();
      phase_levelset_R(g, b, t, nt);
      __syncthreads();
      phase_bc_phichi(g, b, t, nt);
      __syncthreads();
      phase_geom_mat_d<1>(g, b, t, nt);
      __syncthreads();
      phase_geom_cell<false>(g, b, (const double*)Qo, (const double*)nullptr, t, nt);
      __syncthreads();
      if (g.fs_mat >= 0) {
        phase_hold(g, b, Qo, s + 1, t, nt);
        __syncthreads();
      }
      phase_mix_mark(g, b, (const double*)Qo, t, nt);
      __syncthreads();
      phase_mix_weights_d<1>(g, b, t, nt);
      __syncthreads();
      phase_mix_compute_d<1>(g, b, (const double*)Qo, t, nt);
      __syncthreads();
      phase_mix_scatter<false>(g, b, Qo, t, nt);
      __syncthreads();
    }
    if (t == 0) {
      Ctl* c = b.ctl;
      c->t = c->last ? c->t_end : c->t + c->dt;
      c->cnt[C_STEPS] += 1;
    }
    __syncthreads();
    if (g.scale_sep) {
      phase_scale_sep(g, b, b.Q[0], t, nt);
      __syncthreads();
      phase_scatter_phichi(g, b, t, nt);
      __syncthreads();
      phase_bc_phichi(g, b, t, nt);
      __syncthreads();
    }
    if (g.reinit) {
      for (int k = 0; k < g.reinit_iters; k++) {
        reinit_items_d<1>(g, b, t, nt);
        __syncthreads();
        scatter_items(b, t, nt);
        __syncthreads();
      }
      phase_bc_phichi(g, b, t, nt);
      __syncthreads();
    }
  }
}

// end times of every instance of a batch
__global__ void k_set_tend_all(const BatchEntry* tab, int n, double t_end) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) tab[i].b.ctl->t_end = t_end;
}

}  // namespace
}  // namespace msf
