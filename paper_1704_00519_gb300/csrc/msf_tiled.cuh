// msf_tiled.cuh -- temporally blocked ghost-state extension of
// two-dimensional grids.
//
// The ghost-state extension (Sec. 2.3.2) is K Jacobi sweeps with a one-cell
// stencil. One CTA loads a 16 x 16 tile plus a K-cell halo into shared memory
// and runs all K sweeps there: a value near the region edge may be wrong (its
// outer neighbours are missing), but the error moves one cell per sweep, so
// after K sweeps the tile itself holds exactly what K global sweeps give. Each
// cell's arithmetic repeats the one-sweep kernel (msf_kernels.cuh) operation
// by operation. Used for the FP32-bulk form: the halo triples the arithmetic
// and concentrates it on the SMs that hold band tiles, which the FP32 pipes
// absorb but the FP64 pipes (1/58 of the FP32 rate on this part) do not; FP64
// sweeps stay one launch per sweep, spread over every SM. Included after
// msf_kernels.cuh.
#pragma once

#include "msf_tiled.h"

namespace msf {
namespace {

struct TileGeo {
  int x0, y0, H, SX, SY, R;
};
__device__ inline TileGeo tile_geo(const Grid& g, int K) {
  TileGeo t;
  const int nbx = (g.n[0] + TILED_T - 1) / TILED_T;
  const int bx = blockIdx.x % nbx, by = blockIdx.x / nbx;
  t.x0 = g.off[0] + bx * TILED_T;
  t.y0 = g.off[1] + by * TILED_T;
  t.H = K;
  t.SX = TILED_T + 2 * K;
  t.SY = TILED_T + 2 * K;
  t.R = t.SX * t.SY;
  return t;
}
__device__ inline bool tile_interior(const Grid& g, int gx, int gy) {
  return gx >= g.off[0] && gx < g.off[0] + g.n[0] && gy >= g.off[1] && gy < g.off[1] + g.n[1];
}
// does the tile's own 16 x 16 block hold a band cell (thread t looks at cell t)
__device__ inline bool tile_has_band(const Grid& g, const Bufs& b, const TileGeo& t) {
  const int gx = t.x0 + (int)threadIdx.x % TILED_T, gy = t.y0 + (int)threadIdx.x / TILED_T;
  bool mine = tile_interior(g, gx, gy) && b.bandidx[cell_at(g, gx, gy, 0)] >= 0;
  return __syncthreads_or(mine) != 0;
}

// ---------------------------------------------------- ghost-state extension
template <typename T>
__global__ void __launch_bounds__(TILED_T* TILED_T)
    k_extend_tiled(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const void* Win, void* Wout,
                   const uint8_t* fin, uint8_t* fout, int K) {
  if (!ctl_active(b)) return;
  const TileGeo tg = tile_geo(g, K);
  if (!tile_has_band(g, b, tg)) return;
  constexpr int NV = 4;  // two dimensions
  const int R = tg.R, SX = tg.SX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* nx = (double*)smem_raw;                 // [R]
  double* ny = nx + R;                            // [R]
  T* W = (T*)(ny + R);                            // [2][NV][R]
  uint8_t* f = (uint8_t*)(W + 2 * NV * R);        // [2][R]
  uint8_t* ok = f + 2 * R;                        // [R]
  uint8_t* real = ok + R;                         // [R]
  __shared__ unsigned s_uni;
  if (threadIdx.x == 0) s_uni = 0;
  __syncthreads();
  {
    const int gx = tg.x0 + (int)threadIdx.x % TILED_T, gy = tg.y0 + (int)threadIdx.x / TILED_T;
    if (tile_interior(g, gx, gy)) {
      const long long c = cell_at(g, gx, gy, 0);
      if (b.bandidx[c] >= 0) atomicOr(&s_uni, (unsigned)b.smask[c]);
    }
  }
  __syncthreads();
  const unsigned uni = s_uni;
  const T* Wi = (const T*)Win;
  T* Wo = (T*)Wout;
  for (int m = 0; m < g.N; m++) {
    if (!((uni >> m) & 1u)) continue;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      const int gx = tg.x0 - tg.H + r % SX, gy = tg.y0 - tg.H + r / SX;
      uint8_t v = 0;
      if (tile_interior(g, gx, gy)) {
        const long long c = cell_at(g, gx, gy, 0);
        v = (b.bandidx[c] >= 0 && ((b.smask[c] >> m) & 1u)) ? 1 : 0;
        if (v) {
          real[r] = b.isreal[midx(g, m, c)];
          f[r] = fin[midx(g, m, c)];
          for (int q = 0; q < NV; q++) W[q * R + r] = W[(NV + q) * R + r] = Wi[qidx(g, m, q, c)];
          nx[r] = b.nrm[((long long)m * 3 + 0) * g.ncell + c];
          ny[r] = b.nrm[((long long)m * 3 + 1) * g.ncell + c];
        }
      }
      ok[r] = v;
    }
    __syncthreads();
    for (int k = 0; k < K; k++) {
      const int cur = k & 1, nxt = cur ^ 1;
      T* Wc = W + cur * NV * R;
      T* Wn = W + nxt * NV * R;
      const uint8_t* fc = f + cur * R;
      uint8_t* fn = f + nxt * R;
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        if (!ok[r]) continue;
        if (real[r]) {
          fn[r] = 1;
          continue;
        }
        const int sx = r % SX, sy = r / SX;
        T acc[NV] = {T(0), T(0), T(0), T(0)}, acc2[NV] = {T(0), T(0), T(0), T(0)};
        T sw = T(0);
        int cnt = 0;
        for (int d = 0; d < 2; d++)
          for (int s = 0; s < 2; s++) {
            const int ax = d == 0 ? sx + (s ? 1 : -1) : sx, ay = d == 1 ? sy + (s ? 1 : -1) : sy;
            if (ax < 0 || ax >= SX || ay < 0 || ay >= tg.SY) continue;
            const int j = ax + SX * ay;
            if (!ok[j] || !fc[j]) continue;
            const double nd = d == 0 ? nx[r] : ny[r];
            T w = (T)(s ? nd : -nd);
            w = w > T(0) ? w : T(0);
            for (int q = 0; q < NV; q++) {
              const T x = Wc[q * R + j];
              acc[q] += w * x;
              acc2[q] += x;
            }
            sw += w;
            cnt++;
          }
        if (sw > T(0)) {
          for (int q = 0; q < NV; q++) Wn[q * R + r] = acc[q] / sw;
          fn[r] = 1;
        } else if (cnt > 0) {
          for (int q = 0; q < NV; q++) Wn[q * R + r] = acc2[q] / (T)cnt;
          fn[r] = 1;
        } else {
          for (int q = 0; q < NV; q++) Wn[q * R + r] = Wc[q * R + r];
          fn[r] = fc[r];
        }
      }
      __syncthreads();
    }
    {
      const int fin_buf = K & 1;
      const int lx = (int)threadIdx.x % TILED_T, ly = (int)threadIdx.x / TILED_T;
      const int r = (lx + tg.H) + SX * (ly + tg.H);
      const int gx = tg.x0 + lx, gy = tg.y0 + ly;
      if (ok[r] && tile_interior(g, gx, gy)) {
        const long long c = cell_at(g, gx, gy, 0);
        for (int q = 0; q < NV; q++) Wo[qidx(g, m, q, c)] = W[(fin_buf * NV + q) * R + r];
        fout[midx(g, m, c)] = f[fin_buf * R + r];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------- interface-velocity extension
// K sweeps of the interface-velocity extension (extend_vel_items), sums in T:
// the FP32-bulk form's interface velocity comes from an FP32 HLLC state, so
// FP32 sums lose nothing; the level-set values that pick the upwind side stay
// FP64
template <typename T>
__global__ void __launch_bounds__(TILED_T* TILED_T)
    k_extend_vel_tiled(const __grid_constant__ Grid g, const __grid_constant__ Bufs b, const double* vin,
                       double* vout, const uint8_t* fin, uint8_t* fout, int K) {
  if (!ctl_active(b)) return;
  const TileGeo tg = tile_geo(g, K);
  if (!tile_has_band(g, b, tg)) return;
  const int R = tg.R, SX = tg.SX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* ph = (double*)smem_raw;      // [R]
  T* V = (T*)(ph + R);                 // [2][2][R]
  uint8_t* f = (uint8_t*)(V + 4 * R);  // [2][R]
  uint8_t* ok = f + 2 * R;             // [R]
  uint8_t* cut = ok + R;               // [R]
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const int gx = tg.x0 - tg.H + r % SX, gy = tg.y0 - tg.H + r / SX;
    uint8_t v = 0;
    if (tile_interior(g, gx, gy)) {
      const long long c = cell_at(g, gx, gy, 0);
      v = b.bandidx[c] >= 0 ? 1 : 0;
      if (v) {
        cut[r] = (b.gflag[c] & GF_CUT) ? 1 : 0;
        f[r] = fin[c];
        for (int e = 0; e < 2; e++) V[e * R + r] = V[(2 + e) * R + r] = (T)vin[e * g.ncell + c];
        ph[r] = b.phi[c];
      }
    }
    ok[r] = v;
  }
  __syncthreads();
  for (int k = 0; k < K; k++) {
    const int cur = k & 1, nxt = cur ^ 1;
    const T* Vc = V + cur * 2 * R;
    T* Vn = V + nxt * 2 * R;
    const uint8_t* fc = f + cur * R;
    uint8_t* fn = f + nxt * R;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      if (!ok[r]) continue;
      if (cut[r]) {
        for (int e = 0; e < 2; e++) Vn[e * R + r] = Vc[e * R + r];
        fn[r] = 1;
        continue;
      }
      const int sx = r % SX, sy = r / SX;
      T acc[2] = {T(0), T(0)}, acc2[2] = {T(0), T(0)};
      int cnt = 0, cnt2 = 0;
      for (int d = 0; d < 2; d++)
        for (int s = 0; s < 2; s++) {
          const int ax = d == 0 ? sx + (s ? 1 : -1) : sx, ay = d == 1 ? sy + (s ? 1 : -1) : sy;
          if (ax < 0 || ax >= SX || ay < 0 || ay >= tg.SY) continue;
          const int j = ax + SX * ay;
          if (!ok[j] || !fc[j]) continue;
          for (int e = 0; e < 2; e++) acc2[e] += Vc[e * R + j];
          cnt2++;
          if (ph[j] < ph[r]) {
            for (int e = 0; e < 2; e++) acc[e] += Vc[e * R + j];
            cnt++;
          }
        }
      uint8_t filled = 0;
      for (int e = 0; e < 2; e++) Vn[e * R + r] = Vc[e * R + r];
      if (cnt > 0) {
        for (int e = 0; e < 2; e++) Vn[e * R + r] = acc[e] / (T)cnt;
        filled = 1;
      } else if (cnt2 > 0) {
        for (int e = 0; e < 2; e++) Vn[e * R + r] = acc2[e] / (T)cnt2;
        filled = 1;
      } else if (fc[r]) {
        filled = 1;
      }
      fn[r] = filled;
    }
    __syncthreads();
  }
  const int fb = K & 1;
  const int lx = (int)threadIdx.x % TILED_T, ly = (int)threadIdx.x / TILED_T;
  const int r = (lx + tg.H) + SX * (ly + tg.H);
  const int gx = tg.x0 + lx, gy = tg.y0 + ly;
  if (ok[r] && tile_interior(g, gx, gy)) {
    const long long c = cell_at(g, gx, gy, 0);
    for (int e = 0; e < 2; e++) vout[e * g.ncell + c] = (double)V[(fb * 2 + e) * R + r];
    vout[2 * g.ncell + c] = vin[2 * g.ncell + c];
    fout[c] = f[fb * R + r];
  }
}

}  // namespace

template <typename T>
static cudaError_t l_extend_tiled(const Grid& g, const Bufs& b, const void* Win, void* Wout, const uint8_t* fin,
                                  uint8_t* fout, int K, cudaStream_t s) {
  const int SX = TILED_T + 2 * K, R = SX * SX;
  const size_t bytes = (size_t)R * (2 * sizeof(double) + 2 * 4 * sizeof(T) + 4);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_extend_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const int nbx = (g.n[0] + TILED_T - 1) / TILED_T, nby = (g.n[1] + TILED_T - 1) / TILED_T;
  k_extend_tiled<T><<<nbx * nby, TILED_T * TILED_T, bytes, s>>>(g, b, Win, Wout, fin, fout, K);
  return cudaGetLastError();
}
template <typename T>
static cudaError_t l_extend_vel_tiled(const Grid& g, const Bufs& b, const double* vin, double* vout,
                                      const uint8_t* fin, uint8_t* fout, int K, cudaStream_t s) {
  const int SX = TILED_T + 2 * K, R = SX * SX;
  const size_t bytes = (size_t)R * (sizeof(double) + 4 * sizeof(T) + 4);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_extend_vel_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const int nbx = (g.n[0] + TILED_T - 1) / TILED_T, nby = (g.n[1] + TILED_T - 1) / TILED_T;
  k_extend_vel_tiled<T><<<nbx * nby, TILED_T * TILED_T, bytes, s>>>(g, b, vin, vout, fin, fout, K);
  return cudaGetLastError();
}
template <typename T>
static TiledOps make_tiled_ops() {
  TiledOps o;
  o.extend = l_extend_tiled<T>;
  o.extend_vel = l_extend_vel_tiled<T>;
  return o;
}


}  // namespace msf
