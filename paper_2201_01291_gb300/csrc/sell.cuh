// SELL-32 row product shared by the FP64 Krylov kernels.
#pragma once
#include "avip_internal.h"

namespace avip {

// One row of y = A v over the SELL-32 structure (diagonal first, then ascending columns).
// Slots are fetched in groups of 8 so that the column loads, the value loads and the
// dependent gathers of a group are all in flight together.
__device__ __forceinline__ double sell_row_dot(const SellView& A, int slice, int lane, int row,
                                               const double* __restrict__ v) {
  constexpr int U = 8;
  const int base = __ldg(A.sl_ptr + slice) + lane;
  const int w = __ldg(A.sl_w + slice);
  const int rl = __ldg(A.rlen + row);
  double acc = 0.0;
  for (int k0 = 0; k0 < w; k0 += U) {
    int c[U];
    double av[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      c[u] = row;
      av[u] = 0.0;
      if (k < rl) {
        c[u] = __ldg(A.col + base + k * kSlice);
        av[u] = __ldg(A.aval + base + k * kSlice);
      }
    }
    double xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = (k0 + u < rl) ? __ldcg(v + c[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < rl) acc = fma(av[u], xv[u], acc);
  }
  return acc;
}

// The same for a SELL-32 matrix given as SellMatT (the multigrid level operators), accumulated
// in the value type.  The gathered vector is read through L2 (it was written by other blocks
// in an earlier phase).
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
__device__ __forceinline__ T sellmat_row_dot(const SellMatT<T>& M, int slice, int lane, int row,
                                             const T* __restrict__ v) {
  constexpr int U = 8;
  const int base = __ldg(M.sl_ptr + slice) + lane;
  const int w = __ldg(M.sl_w + slice);
  const int rl = __ldg(M.rlen + row);
  T acc = T(0);
  for (int k0 = 0; k0 < w; k0 += U) {
    int c[U];
    T av[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      c[u] = 0;
      av[u] = T(0);
      if (k < rl) {
        c[u] = __ldg(M.col + base + k * kSlice);
        av[u] = __ldg(M.val + base + k * kSlice);
      }
    }
    T xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = (k0 + u < rl) ? __ldcg(v + c[u]) : T(0);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < rl) acc = fma_t(av[u], xv[u], acc);
  }
  return acc;
}

}  // namespace avip
