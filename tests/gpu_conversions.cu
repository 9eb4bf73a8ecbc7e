// Test-only kernels: the integer-pipe conversions and sign tests of the
// library's device header against the hardware instructions they replace,
// bit for bit. Built by tests/test_gpu_fp32_copy.py with the flags of each
// kernel unit (the FP32-bulk unit's fast-math flags change the hardware
// conversions of subnormals, which the integer paths hand back to them).
#include <cstdint>
#include <cuda_runtime.h>

#include "../paper_1704_00519_gb300/csrc/msf_device.cuh"

namespace {

struct Result {
  unsigned long long checked, bad;
  unsigned long long first_bad;  // the first pattern that differed (bits)
};

__device__ void record(Result* r, unsigned long long pattern) {
  if (atomicAdd(&r->bad, 1ull) == 0ull) r->first_bad = pattern;
}

// every binary32 pattern: f2d_bits against the hardware widening
__global__ void k_f2d_all(Result* r) {
  unsigned long long n = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < (1ull << 32);
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float x = __uint_as_float((unsigned)i);
    const double a = msf::f2d_bits(x), b = (double)x;
    if (__double_as_longlong(a) != __double_as_longlong(b)) record(r, i);
    n++;
  }
  atomicAdd(&r->checked, n);
}

__device__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// binary64 pattern k of the test set: for k < 2^24 a structured pattern
// (every sign and exponent with fractions at and around the rounding
// boundaries of the narrowing), otherwise a random one
__device__ unsigned long long pattern64(unsigned long long k) {
  if (k < (1ull << 24)) {
    const unsigned long long se = k >> 12;  // sign and exponent (12 bits)
    const unsigned f = (unsigned)(k & 0xfffu);
    // the 29 dropped bits: 0, 1, half - 1, half, half + 1, all ones, and
    // random; the 23 kept bits: 0, 1, all ones, random (even and odd)
    const unsigned long long h = splitmix64(k);
    const unsigned long long drops[8] = {0ull, 1ull, 0x0fffffffull, 0x10000000ull, 0x10000001ull, 0x1fffffffull,
                                         h & 0x1fffffffull, (h >> 29) & 0x1fffffffull};
    const unsigned long long kept[8] = {0ull, 1ull, 0x7fffffull, 0x7ffffeull, (h >> 7) & 0x7fffffull,
                                        ((h >> 7) & 0x7fffffull) | 1ull, ((h >> 7) & 0x7fffffull) & ~1ull, 2ull};
    const unsigned long long frac = (kept[(f >> 3) & 7] << 29) | drops[f & 7];
    return (se << 52) | frac;
  }
  return splitmix64(k * 0x632be59bd9b4e019ull);
}

// d2f_bits against the hardware narrowing; finite_bits, pos_bits, neg_bits
// and lt_bits against isfinite, x > 0, x < 0 and x < y
__global__ void k_d2f(Result* r, unsigned long long count) {
  unsigned long long n = 0;
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < count;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long p = pattern64(k);
    const double x = __longlong_as_double((long long)p);
    const float a = msf::d2f_bits(x), b = (float)x;
    bool ok = __float_as_uint(a) == __float_as_uint(b);
    ok = ok && msf::finite_bits(x) == (bool)isfinite(x);
    ok = ok && msf::pos_bits(x) == (x > 0.0);
    ok = ok && msf::neg_bits(x) == (x < 0.0);
    const double y = __longlong_as_double((long long)pattern64(k + 1));  // a neighbouring pattern
    ok = ok && msf::lt_bits(x, y) == (x < y) && msf::lt_bits(y, x) == (y < x) && !msf::lt_bits(x, x);
    ok = ok && msf::lt_bits(x, -x) == (x < -x) && msf::lt_bits(-x, x) == (-x < x);  // +0 against -0 too
    if (!ok) record(r, p);
    n++;
  }
  atomicAdd(&r->checked, n);
}

}  // namespace

// which = 0: every binary32 pattern through f2d_bits; which = 1: `count`
// binary64 patterns through d2f_bits and the sign tests. out[0] = patterns
// checked, out[1] = mismatches, out[2] = the first mismatching pattern.
extern "C" int conv_check(int which, unsigned long long count, unsigned long long* out) {
  Result* d = nullptr;
  if (cudaMalloc(&d, sizeof(Result)) != cudaSuccess) return 1;
  cudaMemset(d, 0, sizeof(Result));
  if (which == 0) k_f2d_all<<<4864, 256>>>(d);
  else k_d2f<<<4864, 256>>>(d, count);
  Result h{};
  cudaError_t e = cudaMemcpy(&h, d, sizeof(Result), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return 2;
  out[0] = h.checked;
  out[1] = h.bad;
  out[2] = h.first_bad;
  return 0;
}
