// msf_adjoint_common.cuh -- precision-independent adjoint kernels of one
// TVD-RK3 step at frozen interface evolution: ghost-extension sweeps
// (transposed), primitive recovery, mixing, boundary states, the RK
// combination, and the bookkeeping of the replay (fill levels, band volume
// fractions). Included once, by the FP64 unit, after msf_adjoint.cuh.
#pragma once

#include "msf_adjoint.cuh"

namespace msf {
namespace {

__global__ void k_adj_begin(const __grid_constant__ Bufs b, const double* tdt) {
  Ctl* t = b.ctl;
  t->active = 1;
  t->nband = 0;
  t->lam_bits = 0ull;
  t->dt = *tdt;
  t->last = 0;
}
__global__ void k_adj_end(const __grid_constant__ Bufs b, const double* tt) {
  Ctl* t = b.ctl;
  t->t = *tt;
  t->last = 0;
}

// sweep at which each ghost state was first filled: k = 0 marks the real
// states (flags of the primitive recovery), k >= 1 the output flags of sweep k
__global__ void k_adj_level(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                            const __grid_constant__ AdjBufs a, const uint8_t* f, int k) {
  const int nb = b.ctl->nband, N = g.N;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nb * N; it += gridDim.x * blockDim.x) {
    const int m = it / nb, kk = it - m * nb;
    const long long c = b.band[kk];
    const long long i = midx(g, m, c);
    if (!((b.smask[c] >> m) & 1u)) {
      a.lvl[i] = 0xff;
    } else if (k == 0) {
      a.lvl[i] = f[i] ? 0 : 0xff;
    } else if (f[i] && a.lvl[i] == 0xff) {
      a.lvl[i] = (uint8_t)k;
    }
  }
}

// transpose of extension sweep k: a state updated in sweep k took the
// upwind-weighted (else plain) mean of its neighbours filled before sweep k;
// every other state was carried over unchanged
__global__ void k_adj_ext(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                          const __grid_constant__ AdjBufs a, const double* lin, double* lout, int k) {
  const int nb = b.ctl->nband, N = g.N, NV = g.NV, D = g.D;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nb * N; it += gridDim.x * blockDim.x) {
    const int m = it / nb, kk = it - m * nb;
    const long long c = b.band[kk];
    if (!((b.smask[c] >> m) & 1u)) continue;
    const int lj = a.lvl[midx(g, m, c)];
    const bool keep = lj == 0 || lj > k;
    double out[5];
    for (int v = 0; v < NV; v++) out[v] = keep ? lin[qidx(g, m, v, c)] : 0.0;
    if (lj <= k - 1) {
      int q[3];
      coords(g, c, q);
      for (int d = 0; d < D; d++)
        for (int s = 0; s < 2; s++) {
          if (!nb_interior(g, q, d, s)) continue;
          const long long i = s ? c + g.st[d] : c - g.st[d];
          if (b.bandidx[i] < 0 || !((b.smask[i] >> m) & 1u)) continue;
          const int li = a.lvl[midx(g, m, i)];
          if (li == 0 || li > k) continue;
          double n[3];
          stored_normal(g, b, i, m, n);
          int qi[3];
          coords(g, i, qi);
          double sw = 0.0, wij = 0.0;
          int cnt = 0;
          for (int d2 = 0; d2 < D; d2++)
            for (int s2 = 0; s2 < 2; s2++) {
              if (!nb_interior(g, qi, d2, s2)) continue;
              const long long l = s2 ? i + g.st[d2] : i - g.st[d2];
              if (b.bandidx[l] < 0 || !((b.smask[l] >> m) & 1u) || a.lvl[midx(g, m, l)] > k - 1) continue;
              double w = s2 ? n[d2] : -n[d2];
              w = w > 0.0 ? w : 0.0;
              sw += w;
              cnt++;
              if (l == c) wij = w;
            }
          const double coef = sw > 0.0 ? wij / sw : 1.0 / (double)cnt;
          if (coef == 0.0) continue;
          for (int v = 0; v < NV; v++) out[v] += coef * lin[qidx(g, m, v, i)];
        }
    }
    for (int v = 0; v < NV; v++) lout[qidx(g, m, v, c)] = out[v];
  }
}

// real band states: W = cons_to_prim(Q / alpha)
__global__ void k_adj_prim(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                           const __grid_constant__ AdjBufs a, const double* Qs, const double* lw) {
  const int nb = b.ctl->nband, N = g.N, NV = g.NV, D = g.D;
  __shared__ double s_de[2 * MAXM];
  eos_block_init(s_de, N);
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nb * N; it += gridDim.x * blockDim.x) {
    const int m = it / nb, kk = it - m * nb;
    const long long c = b.band[kk];
    if (!((b.smask[c] >> m) & 1u) || !b.isreal[midx(g, m, c)]) continue;
    double gw[5];
    bool any = false;
    for (int v = 0; v < NV; v++) {
      gw[v] = lw[qidx(g, m, v, c)];
      any = any || gw[v] != 0.0;
    }
    if (!any) continue;
    const double al = b.alpha[midx(g, m, c)];
    double u[5], gu[5] = {0, 0, 0, 0, 0}, ge[2] = {0, 0};
    for (int v = 0; v < NV; v++) u[v] = Qs[qidx(g, m, v, c)] / al;
    c2p_reverse(g, m, D, u, gw, gu, ge);
    for (int v = 0; v < NV; v++) a.LQ[qidx(g, m, v, c)] += gu[v] / al;
    atomicAdd(&s_de[2 * m], ge[0]);
    atomicAdd(&s_de[2 * m + 1], ge[1]);
  }
  eos_block_flush(s_de, a.deos, N);
}

// mixing adjoint, part 1: transpose of the merge of a material that lost
// all volume into the cell's primary (its state became part of the primary's)
__global__ void k_adj_mix_merge(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                                const __grid_constant__ AdjBufs a, int st, const uint8_t* chi_next) {
  const int nb = b.ctl->nband, N = g.N, NV = g.NV;
  const uint8_t* mixn = a.mixn[st];
  const double* ab = a.aband[st + 1];
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nb * N; it += gridDim.x * blockDim.x) {
    const int m = it / nb, kk = it - m * nb;
    const long long c = b.band[kk];
    const long long r = (long long)kk * N + m;
    int src = m;
    const int nown = mixn[r];
    if (nown == 0 && ab[r] == 0.0 && m != chi_next[c]) src = chi_next[c];
    for (int v = 0; v < NV; v++) a.mixt[r * NV + v] = a.LA[qidx(g, src, v, c)];
  }
}

// mixing adjoint, part 2: transpose of the pairwise exchanges
// M = f beta (a_s Q_t - a_t Q_s) / (a_s + a_t), Q_s += M, Q_t -= M, with the
// pair scale f = mix_limit(a_s, T_s, T_t) of the recorded weight sums (f and
// the volume fractions do not depend on Q at frozen interface evolution)
__global__ void k_adj_mix_exchange(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                                   const __grid_constant__ AdjBufs a, int st) {
  const int nb = b.ctl->nband, N = g.N, NV = g.NV, D = g.D;
  const uint8_t* mixn = a.mixn[st];
  const uint8_t* mixoff = a.mixoff[st];
  const double* mixbeta = a.mixbeta[st];
  const double* mixT = a.mixT[st];
  const double* ab = a.aband[st + 1];
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nb * N; it += gridDim.x * blockDim.x) {
    const int m = it / nb, kk = it - m * nb;
    const long long c = b.band[kk];
    const long long r = (long long)kk * N + m;
    const double* lx = a.mixt + r * NV;
    double out[5];
    for (int v = 0; v < NV; v++) out[v] = lx[v];
    if ((b.smask[c] >> m) & 1u) {
      const int nown = mixn[r];
      const double ax = ab[r];
      if (nown != 0xff)
        for (int t = 0; t < nown; t++) {
          const long long tc = off_cell(g, c, mixoff[r * MIX_MAXT + t]);
          const long long rt = (long long)b.bandidx[tc] * N + m;
          const double at = ab[rt];
          const double kap = mix_limit(ax, mixT[r], mixT[rt]) * mixbeta[r * MIX_MAXT + t] / (ax + at);
          for (int v = 0; v < NV; v++) out[v] += kap * at * (a.mixt[rt * NV + v] - lx[v]);
        }
      int q[3];
      coords(g, c, q);
      const int rz = D >= 3 ? 1 : 0, ry = D >= 2 ? 1 : 0;
      for (int dz = -rz; dz <= rz; dz++)
        for (int dy = -ry; dy <= ry; dy++)
          for (int dx = -1; dx <= 1; dx++) {
            if (dx == 0 && dy == 0 && dz == 0) continue;
            const int sx = q[0] - dx, sy = q[1] - dy, sz = q[2] - dz;
            if (!in_array(g, sx, sy, sz)) continue;
            const long long s = cell_at(g, sx, sy, sz);
            const int ks = b.bandidx[s];
            if (ks < 0) continue;
            const long long rs = (long long)ks * N + m;
            const int ns = mixn[rs];
            if (ns == 0xff) continue;
            const uint8_t code = off_code(dx, dy, dz);
            for (int t = 0; t < ns; t++) {
              if (mixoff[rs * MIX_MAXT + t] != code) continue;
              const double as = ab[rs];
              const double kap = mix_limit(as, mixT[rs], mixT[r]) * mixbeta[rs * MIX_MAXT + t] / (as + ax);
              for (int v = 0; v < NV; v++) out[v] += kap * as * (a.mixt[rs * NV + v] - lx[v]);
            }
          }
    }
    for (int v = 0; v < NV; v++) a.LA[qidx(g, m, v, c)] = out[v];
  }
}

// boundary states: the adjoint of a halo state goes to its source cell
// (sign of the normal momentum flipped at reflective sides) or, for an
// inflow side, to the inflow primitive state and the EOS
__global__ void k_adj_bc(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                         const __grid_constant__ AdjBufs a) {
  const int N = g.N, NV = g.NV, D = g.D;
  __shared__ double s_de[2 * MAXM];
  eos_block_init(s_de, N);
  long long per[3] = {0, 0, 0}, total = 0;
  for (int d = 0; d < D; d++) {
    per[d] = 2LL * G * (g.n_interior / g.n[d]);
    total += per[d];
  }
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int d = 0;
    long long r0 = idx;
    while (r0 >= per[d]) { r0 -= per[d]; d++; }
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
      double gu[5];
      bool any = false;
      for (int v = 0; v < NV; v++) {
        gu[v] = a.LU[qidx(g, m, v, c)];
        any = any || gu[v] != 0.0;
      }
      if (!any) continue;
      if (type == 2 && m == g.inflow_mat[d][side]) {
        double w[5], gw[5] = {0, 0, 0, 0, 0}, ge[2] = {0, 0};
        for (int v = 0; v < NV; v++) w[v] = g.inflow_prim[d][side][v];
        p2c_reverse(g, m, D, w, gu, gw, ge);
        for (int v = 0; v < NV; v++) atomicAdd(&a.dinf[(d * 2 + side) * 5 + v], gw[v]);
        atomicAdd(&s_de[2 * m], ge[0]);
        atomicAdd(&s_de[2 * m + 1], ge[1]);
        continue;
      }
      const bool used = b.bandidx[sc] >= 0 ? (((b.smask[sc] >> m) & 1u) != 0) : (b.chi[sc] == m);
      if (!used) continue;
      if (flip) gu[1 + d] = -gu[1 + d];
      for (int v = 0; v < NV; v++)
        if (gu[v] != 0.0) atomicAdd(&a.LU[qidx(g, m, v, sc)], gu[v]);
    }
  }
  eos_block_flush(s_de, a.deos, N);
}

// RK combination Q^(s+1) = beta Q^n + (1 - beta) (Q^(s) + dt L(Q^(s))) of the
// updated states; states the stage does not update keep their buffer value
// (for the last stage that value is Q^n itself)
__global__ void k_adj_combine(const __grid_constant__ Grid g, const __grid_constant__ Bufs b,
                              const __grid_constant__ AdjBufs a, double beta, double omb, int last_stage) {
  const int N = g.N, NV = g.NV;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.n_interior;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, idx);
    const bool inb = b.bandidx[c] >= 0;
    for (int m = 0; m < N; m++) {
      const bool upd = (b.smask[c] >> m) & 1u;
      for (int v = 0; v < NV; v++) {
        const long long i = qidx(g, m, v, c);
        const double lt = a.LA[i];
        if (upd) {
          a.LN[i] += beta * lt;
          const double gq = inb ? a.LQ[i] : (b.chi[c] == m ? a.LU[i] : 0.0);
          a.LA[i] = omb * lt + gq;
        } else {
          if (last_stage) a.LN[i] += lt;
          a.LA[i] = 0.0;
        }
      }
    }
  }
}

// band volume fractions: save after a geometry pass, or restore them
__global__ void k_adj_alpha(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, double* ab, int save) {
  const int nb = b.ctl->nband, N = g.N;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nb * N; it += gridDim.x * blockDim.x) {
    const int m = it / nb, kk = it - m * nb;
    const long long c = b.band[kk];
    const long long r = (long long)kk * N + m;
    if (save) ab[r] = b.alpha[midx(g, m, c)];
    else b.alpha[midx(g, m, c)] = ab[r];
  }
}

// adjoint in / out: dir 0 copies lam_out (interior SoA) into LA and clears
// LN; dir 1 writes lam_in = LA + LN; dir 2 scatters an interior SoA state
// (lout) into a padded state array (lin)
__global__ void k_adj_io(const __grid_constant__ Grid g, const __grid_constant__ AdjBufs a, const double* lout,
                         double* lin, int dir) {
  const int N = g.N, NV = g.NV;
  const long long ni = g.n_interior;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ni;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = interior_cell(g, idx);
    for (int m = 0; m < N; m++)
      for (int v = 0; v < NV; v++) {
        const long long i = qidx(g, m, v, c), o = ((long long)m * NV + v) * ni + idx;
        if (dir == 0) {
          a.LA[i] = lout[o];
          a.LN[i] = 0.0;
        } else if (dir == 2) {
          lin[i] = lout[o];
        } else {
          lin[o] = a.LA[i] + a.LN[i];
        }
      }
  }
}

}  // namespace

static int adj_grid_blocks(long long n) {
  long long b = (n + NTHREADS - 1) / NTHREADS;
  if (b > 1216) b = 1216;
  if (b < 1) b = 1;
  return (int)b;
}

void launch_adj_begin(const Bufs& b, const double* tdt, cudaStream_t s) { k_adj_begin<<<1, 1, 0, s>>>(b, tdt); }
void launch_adj_end(const Bufs& b, const double* tt, cudaStream_t s) { k_adj_end<<<1, 1, 0, s>>>(b, tt); }
void launch_adj_level(const Grid& g, const Bufs& b, const AdjBufs& a, const uint8_t* f, int k, int nblk,
                      cudaStream_t s) {
  k_adj_level<<<nblk, BAND_THREADS, 0, s>>>(g, b, a, f, k);
}
void launch_adj_ext(const Grid& g, const Bufs& b, const AdjBufs& a, const double* lin, double* lout, int k, int nblk,
                    cudaStream_t s) {
  k_adj_ext<<<nblk, BAND_THREADS, 0, s>>>(g, b, a, lin, lout, k);
}
void launch_adj_prim(const Grid& g, const Bufs& b, const AdjBufs& a, const double* Qs, const double* lw, int nblk,
                     cudaStream_t s) {
  k_adj_prim<<<nblk, BAND_THREADS, 0, s>>>(g, b, a, Qs, lw);
}
void launch_adj_mix(const Grid& g, const Bufs& b, const AdjBufs& a, int stage, const uint8_t* chi_next, int nblk,
                    cudaStream_t s) {
  k_adj_mix_merge<<<nblk, BAND_THREADS, 0, s>>>(g, b, a, stage, chi_next);
  k_adj_mix_exchange<<<nblk, BAND_THREADS, 0, s>>>(g, b, a, stage);
}
void launch_adj_bc(const Grid& g, const Bufs& b, const AdjBufs& a, cudaStream_t s) {
  k_adj_bc<<<adj_grid_blocks(g.ncell - g.n_interior), NTHREADS, 0, s>>>(g, b, a);
}
void launch_adj_combine(const Grid& g, const Bufs& b, const AdjBufs& a, double beta, double omb, int last_stage,
                        cudaStream_t s) {
  k_adj_combine<<<adj_grid_blocks(g.n_interior), NTHREADS, 0, s>>>(g, b, a, beta, omb, last_stage);
}
void launch_adj_alpha(const Grid& g, const Bufs& b, double* ab, int save, int nblk, cudaStream_t s) {
  k_adj_alpha<<<nblk, BAND_THREADS, 0, s>>>(g, b, ab, save);
}
void launch_adj_io(const Grid& g, const AdjBufs& a, const double* lout, double* lin, int dir, cudaStream_t s) {
  k_adj_io<<<adj_grid_blocks(g.n_interior), NTHREADS, 0, s>>>(g, a, lout, lin, dir);
}

}  // namespace msf
