// Layer geometry of one sample, shared by the 2-D and 3-D solver kernels
// (internal header): the random interfaces (Sec. 2) or the line ends of the
// three-layer example (Sec. 3.4), the Ex. 1 layer constants, and the layer
// of a point.
#pragma once
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace mlmc {

__device__ __forceinline__ int layer_at(const double* eta, int n_if, double y) {
  int t = 0;
  for (int s = 0; s < n_if; ++s) t += (eta[s] <= y) ? 1 : 0;
  return t;
}

// Layer of the point (x, y): geometry 0 counts the interfaces at or below y;
// geometry 1 counts the lines (0, e2)-(1, e3) and (0, e0)-(1, e1) at or below
// it, the line height e_a + ((e_b - e_a) x) rounded once per operation.
__device__ __forceinline__ int layer_at_point(int geometry, const double* eta, int n_if, double x, double y) {
  if (geometry != 1) return layer_at(eta, n_if, y);
  const double lower = __dadd_rn(eta[2], __dmul_rn(__dadd_rn(eta[3], -eta[2]), x));
  const double upper = __dadd_rn(eta[0], __dmul_rn(__dadd_rn(eta[1], -eta[0]), x));
  return (lower <= y ? 1 : 0) + (upper <= y ? 1 : 0);
}

// Interfaces of one sample (sorted; geometry 1: the four line ends, in order)
// and, for Ex. 1, the layer constants.
__device__ inline void sample_layers(const SolveArgs& a, uint64_t sample, double* eta, double* kc) {
  const int n_if = a.geometry == 1 ? 0 : a.n_layers - 1;
  const double width = __dadd_rn(a.if_hi, -a.if_lo);
  if (a.geometry == 1) {
    const Words4 w = philox4x64_10(0, sample, (uint64_t)a.level, kStreamInterface, a.seed);
    const uint64_t ws[4] = {w.w0, w.w1, w.w2, w.w3};
    for (int t = 0; t < 4; ++t)
      eta[t] = __dadd_rn(a.line_lo[t], __dmul_rn(__dadd_rn(a.line_hi[t], -a.line_lo[t]), uniform52(ws[t])));
  }
  for (int t = 0; t < n_if; ++t) {
    const Words4 w = philox4x64_10((uint64_t)(t >> 2), sample, (uint64_t)a.level, kStreamInterface,
                                   a.seed);
    const uint64_t wt = (t & 3) == 0 ? w.w0 : (t & 3) == 1 ? w.w1 : (t & 3) == 2 ? w.w2 : w.w3;
    eta[t] = __dadd_rn(a.if_lo, __dmul_rn(width, uniform52(wt)));
  }
  for (int t = 1; t < n_if; ++t) {  // insertion sort, ascending
    const double v = eta[t];
    int s = t - 1;
    while (s >= 0 && eta[s] > v) {
      eta[s + 1] = eta[s];
      --s;
    }
    eta[s + 1] = v;
  }
  if (a.ksrc == KSRC_CONST) {
    for (int t = 0; t < a.n_layers; t += 4) {
      const Words4 w = philox4x64_10((uint64_t)(t >> 2), sample, (uint64_t)a.level, kStreamLayerZ,
                                     a.seed);
      double z[4];
      box_muller(uniform52(w.w0), uniform52(w.w1), z[0], z[1]);
      box_muller(uniform52(w.w2), uniform52(w.w3), z[2], z[3]);
      for (int u = 0; u < 4 && t + u < a.n_layers; ++u)
        kc[t + u] = exp(a.mu[t + u] + a.sigma[t + u] * z[u]);
    }
  }
}

}  // namespace mlmc
