// Shared device helpers of the MLMC level-batch library: the counter-based
// generator, uniforms, Box-Muller, block reductions and launch constants.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mlmc {

// ---------------------------------------------------------------- Philox --
// Philox4x64-10 of Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
// as easy as 1, 2, 3" (SC'11): ten rounds of two 64x64 -> 128-bit products on
// a four-word counter, key bumped by two Weyl constants between rounds.
constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

// Stream ids of the counter word c3.
constexpr uint64_t kStreamInterface = 0;
constexpr uint64_t kStreamLayerZ = 1;
constexpr uint64_t kStreamField0 = 2;

struct Words4 {
  uint64_t w0, w1, w2, w3;
};

// Counter (call, sample, level, stream), key (seed, 0).
__host__ __device__ __forceinline__ Words4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                                         uint64_t c3, uint64_t k0) {
  uint64_t k1 = 0;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
#ifdef __CUDA_ARCH__
    const uint64_t hi0 = __umul64hi(kPhiloxM0, c0);
    const uint64_t hi1 = __umul64hi(kPhiloxM1, c2);
#else
    const uint64_t hi0 = (uint64_t)(((unsigned __int128)kPhiloxM0 * c0) >> 64);
    const uint64_t hi1 = (uint64_t)(((unsigned __int128)kPhiloxM1 * c2) >> 64);
#endif
    const uint64_t lo0 = kPhiloxM0 * c0;
    const uint64_t lo1 = kPhiloxM1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0;
    const uint64_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return Words4{c0, c1, c2, c3};
}

// u = ((w >> 12) + 1/2) 2^-52: exact in FP64, strictly inside (0, 1).
__device__ __forceinline__ double uniform52(uint64_t w) {
  return __dmul_rn(__dadd_rn((double)(w >> 12), 0.5), 0x1p-52);
}

// Box-Muller pair from two uniforms: (r cos 2 pi ub, r sin 2 pi ub),
// r = sqrt(-2 ln ua).
__device__ __forceinline__ void box_muller(double ua, double ub, double& re, double& im) {
  const double rad = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  re = rad * c;
  im = rad * s;
}

// FP32 version for the mixed-precision field path, from the words directly,
// with no FP64 arithmetic (GB300's FP64 rate is a small fraction of its FP32
// rate).  u = (K + 1/2) 2^-52, K = w >> 12, as in uniform52():
//  - ln u_a: above 1/2 as log1p(-(1 - u_a)) with 1 - u_a = (2^52 - 1 - K + 1/2)
//    2^-52 formed in integers, so u_a close to 1 keeps its distance from 1;
//    below 1/2 as ln u_a;
//  - 2 u_b = k + x with k the nearest integer and x in [-1/2, 1/2] formed in
//    integers, and sincos(pi (k + x)) = (-1)^k sincos(pi x).
// Absolute error of the normals ~1e-6.
__device__ __forceinline__ void box_muller_words(uint64_t wa, uint64_t wb, float& re, float& im) {
  const uint64_t Ka = wa >> 12, Kb = wb >> 12;
  float lg;
  if (Ka >= (1ull << 51)) {
    const uint64_t Kc = ((1ull << 52) - 1) - Ka;  // 1 - u = (Kc + 1/2) 2^-52
    lg = log1pf(-((float)(2 * Kc + 1) * 0x1p-53f));
  } else {
    lg = logf((float)(2 * Ka + 1) * 0x1p-53f);
  }
  const float rad = sqrtf(-2.0f * lg);
  const uint64_t k = (Kb + (1ull << 50)) >> 51;              // nearest integer to 2 u_b
  const long long D = (long long)(2 * Kb + 1) - (long long)(k << 52);  // 2^52 x, |x| <= 1/2
  float s, c;
  sincospif((float)D * 0x1p-52f, &s, &c);
  const float sg = (k & 1) ? -1.0f : 1.0f;
  re = sg * rad * c;
  im = sg * rad * s;
}

// ------------------------------------------- table-driven FP64 Box-Muller --
// FP64 -2 ln u and (cos, sin)(2 pi u) by table-driven argument reduction (the
// method of P. T. P. Tang, "Table-driven implementation of the logarithm
// function in IEEE floating-point arithmetic", ACM TOMS 16 (1990), and the
// analogous reduction for the trigonometric functions), with Taylor
// polynomials on the reduced interval, working from the integer K = w >> 12
// of u = (K + 1/2) 2^-52 = (2K + 1) 2^-53 so that no integer-to-FP64
// conversion and no scaling of u is needed.  Tables hold exact-argument
// values from the CUDA math library, computed once per context
// (bm_tables_kernel):
//   sc[j] = (cos(2 pi j/1024), sin(2 pi j/1024)), j < 1024;
//   lg[3t .. 3t+2] = (F_t, -2/F_t, -2 ln F_t), F_t = 1/2 + (t + 1/2)/2048,
//     t < 1024;
//   lg[3072 + e] = 2 e ln 2, e = 0 .. 52.
constexpr int kSinCosTab = 1024;
constexpr int kLogTab = 1024;
constexpr int kLogExpTab = 53;
constexpr int kBmLgDoubles = 3 * kLogTab + kLogExpTab;

struct BmTables {
  const double2* sc;
  const double* lg;
};

// -2 ln u for u = (2K + 1) 2^-53 (K < 2^52): N = 2K + 1 = v 2^(53 - e) with
// v in [1/2, 1) read off the bits of N (e = 0 .. 52); v = F_t (1 + r),
// |r| <= 1/2048; with s = -2 r, -2 ln(1 + r) = s + s^2/4 + s^3/12 + s^4/32
// (truncation |s|^5/80 < 1.2e-17), so -2 ln u = 2 e ln 2 - 2 ln F_t + that.
// s = (v - F_t)(-2/F_t) is the exact difference times the rounded factor, so
// the absolute error stays ~1e-19 near u = 1.
__device__ __forceinline__ double tab_m2log(uint64_t K, const double* __restrict__ lg) {
  const uint64_t N = 2 * K + 1;
  const int lz = __clzll((long long)N);  // 11 .. 63
  const uint64_t Nn = N << lz;            // leading one at bit 63; the low lz bits are zero
  const int e = lz - 11;
  const double v = __longlong_as_double((long long)((1022ull << 52) | ((Nn >> 11) & ((1ull << 52) - 1))));
  const int t = (int)((Nn >> 53) & (kLogTab - 1));
  const double F = __ldg(lg + 3 * t), m2iF = __ldg(lg + 3 * t + 1), m2lF = __ldg(lg + 3 * t + 2);
  const double sv = (v - F) * m2iF;
  double q = fma(sv, 1.0 / 32.0, 1.0 / 12.0);
  q = fma(q, sv, 0.25);
  const double l1 = fma(q, sv * sv, sv);
  return __ldg(lg + 3 * kLogTab + e) + (m2lF + l1);
}

// r (cos 2 pi u, sin 2 pi u) for u = (2K + 1) 2^-53, K = w >> 12: u = j/1024
// + b with the nearest j (integer arithmetic, exact), theta = 2 pi b =
// (2D + 1) pi 2^-52 with |theta| <= pi/1024 (2D + 1 is exact in FP64).  The
// angle addition in tangent form, cos(a + theta) = cos(theta) (cos a -
// tan(theta) sin a) and sin(a + theta) = cos(theta) (sin a + tan(theta)
// cos a), with the tabulated (cos a, sin a) and Taylor polynomials of
// tan(theta) to theta^5 and cos(theta) to theta^4 (truncation < 2e-18);
// r cos(theta) scales both.
__device__ __forceinline__ void tab_polar(uint64_t w, double r, const double2* __restrict__ sc, double& x,
                                          double& y) {
  const long long K = (long long)(w >> 12);
  const long long j = (K + (1LL << 41)) >> 42;
  const long long D = K - (j << 42);
  const double th = (double)(2 * D + 1) * 0x1.921fb54442d18p-51;  // pi 2^-52
  const double t2 = th * th;
  const double tn = fma(th * t2, fma(t2, 2.0 / 15.0, 1.0 / 3.0), th);  // tan(theta)
  const double rc = r * fma(t2, fma(t2, 1.0 / 24.0, -0.5), 1.0);      // r cos(theta)
  const double2 cs = __ldg(sc + (j & (kSinCosTab - 1)));
  x = rc * fma(-tn, cs.y, cs.x);
  y = rc * fma(tn, cs.x, cs.y);
}

// Box-Muller pair from two words (same definition as box_muller()), each
// normal times `scale` (folded into the radius).
__device__ __forceinline__ void box_muller_tab(uint64_t wa, uint64_t wb, const BmTables& tb, double& re,
                                               double& im, double scale = 1.0) {
  const double rad = sqrt(tab_m2log(wa >> 12, tb.lg)) * scale;
  tab_polar(wb, rad, tb.sc, re, im);
}

__device__ __forceinline__ void box_muller_tab(uint64_t wa, uint64_t wb, const BmTables&, float& re,
                                               float& im, float scale = 1.0f) {
  box_muller_words(wa, wb, re, im);
  re *= scale;
  im *= scale;
}

// ------------------------------------------------------------ reductions --
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block in a fixed order (deterministic).  `red` is a shared
// buffer of 2*66 elements; `parity` alternates between calls (of block_sum
// and block_sum2 alike) so that a call never overwrites slots that a slow
// thread may still read from the previous call.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red, int& parity) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  T* buf = red + 66 * parity;
  parity ^= 1;
  v = warp_sum(v);
  if (lane == 0) buf[warp] = v;
  __syncthreads();
  if (warp == 0) {
    T t = lane < nw ? buf[lane] : T(0);
    t = warp_sum(t);
    if (lane == 0) buf[32] = t;
  }
  __syncthreads();
  return buf[32];
}

// Two sums at once (fewer barriers).
template <typename T>
__device__ __forceinline__ void block_sum2(T& a, T& b, T* red, int& parity) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  T* buf = red + 66 * parity;
  parity ^= 1;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    buf[warp] = a;
    buf[33 + warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    T ta = lane < nw ? buf[lane] : T(0);
    T tb = lane < nw ? buf[33 + lane] : T(0);
    ta = warp_sum(ta);
    tb = warp_sum(tb);
    if (lane == 0) {
      buf[32] = ta;
      buf[65] = tb;
    }
  }
  __syncthreads();
  a = buf[32];
  b = buf[65];
}

__host__ __device__ __forceinline__ int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

}  // namespace mlmc
