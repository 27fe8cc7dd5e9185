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

__device__ __forceinline__ void box_muller(double ua, double ub, float& re, float& im) {
  const float rad = sqrtf(-2.0f * logf((float)ua));
  float s, c;
  sincospif(2.0f * (float)ub, &s, &c);
  re = rad * c;
  im = rad * s;
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
