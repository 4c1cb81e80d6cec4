// Mixed-precision Poisson solve: FP32 inner Jacobi-PCG with FP64 iterative refinement.
//
// Outer loop (FP64): r = b' - A x with the FP64 matrix and the FP64 iterate, stop when
// ||r||_2 <= rtol ||b'||_2 (this is also the final true-residual test), otherwise solve
// A e = r / ||r|| in FP32 to a relative reduction inner_rtol and correct x += ||r|| e in FP64.
// Inner loop (FP32): the same CG recurrences as the FP64 kernel on the symmetrically
// Jacobi-scaled matrix (z = r), FP32 matrix values and vectors, FP32 products and FP32
// compensated (Kahan) per-thread accumulation of the dot products; the per-thread partials
// are combined across the grid in FP64 by the deterministic grid reduction.
// On GB300 the FP32 pipe is ~58x faster than FP64 and FP32 values halve the matrix and
// vector traffic, so the inner iterations are bound by memory latency and synchronisation
// instead of FP64 issue.  Only the outer residual and the correction run in FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "avip_internal.h"
#include "grid_sync.cuh"

namespace avip {

struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ float sell_row_dot32(const SellView& A, const float* __restrict__ aval, int slice,
                                                int lane, int row, const float* __restrict__ v) {
  constexpr int U = 8;
  const int base = __ldg(A.sl_ptr + slice) + lane;
  const int w = __ldg(A.sl_w + slice);
  const int rl = __ldg(A.rlen + row);
  float acc = 0.f;
  for (int k0 = 0; k0 < w; k0 += U) {
    int c[U];
    float av[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      c[u] = row;
      av[u] = 0.f;
      if (k < rl) {
        c[u] = __ldg(A.col + base + k * kSlice);
        av[u] = __ldg(aval + base + k * kSlice);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = (k0 + u < rl) ? __ldcg(v + c[u]) : 0.f;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < rl) acc = fmaf(av[u], xv[u], acc);
  }
  return acc;
}

__device__ __forceinline__ double sell_row_dot64(const SellView& A, int slice, int lane, int row,
                                                 const double* __restrict__ v) {
  constexpr int U = 8;
  const int base = __ldg(A.sl_ptr + slice) + lane;
  const int w = __ldg(A.sl_w + slice);
  const int rl = __ldg(A.rlen + row);
  double acc = 0.0;
  for (int k0 = 0; k0 < w; k0 += U) {
    int c[U];
    double av[U], xv[U];
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
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = (k0 + u < rl) ? __ldcg(v + c[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < rl) acc = fma(av[u], xv[u], acc);
  }
  return acc;
}

template <int TPB>
__global__ void __launch_bounds__(TPB, (TPB <= 512 ? 1024 / TPB : 1)) pcg_mixed_kernel(PcgArgs a) {
  if (solve_skipped(a.sc)) return;  // an earlier stage of this run failed beyond repair
  __shared__ double smem[2 * 32 * 4];
  const int lane = threadIdx.x & 31;
  constexpr int wpb = TPB / 32;
  const int gwarp = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  const int N = a.A.N, nsl = a.A.nslices;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
  FlagSync fs{a.flags, a.parts, a.sync, 0u, a.spin_ns, (int)gridDim.x, (int)blockIdx.x};
  double one[1];

  // ---- x = D^1/2 phi (warm start) and b'
  const double gain = dirichlet_gain(a);
  const int hist = history_length(a);
  double bb[1] = {0.0};
  for (int s = gwarp; s < nsl; s += nwarps) {
    const int i = s * kSlice + lane;
    if (i >= N) continue;
    a.x[i] = a.dsq[i] * predict_phi(a, i, hist);
    double b;
    if (a.use_density_rhs) {
      double rho = 0.0;
      if (a.rhs_src)
        rho = a.rhs_src[i];
      else
        for (int k = 0; k < a.ns; ++k) rho = fma(a.q[k], nb[(size_t)k * a.Npad + i], rho);
      b = fma(a.rhs_scale[i], rho, gain * a.lift[i]);
      a.b[i] = b;
    } else {
      b = a.b[i];
    }
    if (a.rhs_scale[i] != 0.0) bb[0] = fma(b, b, bb[0]);  // free rows only: a Dirichlet row holds its value exactly
    else a.x[i] = b;  // a Dirichlet unit row takes its (possibly ramped) value exactly
  }
  if (!grid_allsum<1>(bb, fs, smem)) goto timeout;
  {
    const double thresh = a.rtol * a.rtol * bb[0];
    int it = 0, outer = 0, status = AVIP_OK;
    double rr64 = 0.0;
    while (true) {
      // ---- FP64 residual of the FP64 iterate (x complete: a reduction separates its writes)
      double r2[1] = {0.0};
      for (int s = gwarp; s < nsl; s += nwarps) {
        const int i = s * kSlice + lane;
        if (i >= N) continue;
        const double r = a.b[i] - sell_row_dot64(a.A, s, lane, i, a.x);
        a.r[i] = r;
        r2[0] = fma(r, r, r2[0]);
      }
      if (!grid_allsum<1>(r2, fs, smem)) goto timeout;
      rr64 = r2[0];
      if (!isfinite(rr64)) {  // non-finite right-hand side or iterate: stop, never loop on NaN
        status = AVIP_ENAN;
        break;
      }
      if (rr64 <= thresh || bb[0] == 0.0) break;
      if (it >= a.max_iter) {
        status = AVIP_ENOTCONV;
        break;
      }
      ++outer;
      const int it_outer = it;
      const double rnorm = sqrt(rr64);
      const double rscale = 1.0 / rnorm;
      // ---- FP32 right-hand side r / ||r||, e = 0
      double g0[1];
      {
        Kahan k;
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          const float r = (float)(a.r[i] * rscale);
          a.r32[i] = r;
          a.e32[i] = 0.f;
          a.p32[i] = 0.f;
          a.q32[i] = 0.f;
          k.add(r * r);
        }
        g0[0] = k.value();
      }
      if (!grid_allsum<1>(g0, fs, smem)) goto timeout;
      const double inner_thresh = a.inner_rtol * a.inner_rtol * g0[0];
      double rr = g0[0];
      float beta = 0.f;
      // ---- FP32 inner CG
      while (rr > inner_thresh && it < a.max_iter) {
        Kahan kpq;
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          const float w = sell_row_dot32(a.A, a.aval32, s, lane, i, a.r32);
          const float qn = fmaf(beta, a.q32[i], w);
          const float pn = fmaf(beta, a.p32[i], a.r32[i]);
          a.q32[i] = qn;
          a.p32[i] = pn;
          kpq.add(pn * qn);
        }
        double pq[1] = {kpq.value()};
        const double rr_now = rr;
        if (!grid_allsum<1, 1>(pq, one, fs, smem, [rr_now](const double* t, double* e) { e[0] = rr_now / t[0]; }))
          goto timeout;
        const float alpha = (float)one[0];
        Kahan krr;
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          a.e32[i] = fmaf(alpha, a.p32[i], a.e32[i]);
          const float r = fmaf(-alpha, a.q32[i], a.r32[i]);
          a.r32[i] = r;
          krr.add(r * r);
        }
        double rn[1] = {krr.value()};
        double bs[1];
        if (!grid_allsum<1, 1>(rn, bs, fs, smem, [rr_now](const double* t, double* e) { e[0] = t[0] / rr_now; }))
          goto timeout;
        beta = (float)bs[0];
        rr = rn[0];
        ++it;
      }
      if (it == it_outer) {  // the inner solve could not start: no progress is possible
        status = AVIP_ENOTCONV;
        break;
      }
      // ---- FP64 correction x += ||r|| e
      for (int s = gwarp; s < nsl; s += nwarps) {
        const int i = s * kSlice + lane;
        if (i >= N) continue;
        a.x[i] = fma(rnorm, (double)a.e32[i], a.x[i]);
      }
      double z0[1] = {0.0};
      if (!grid_allsum<1>(z0, fs, smem)) goto timeout;  // x complete before the next residual
    }
    for (int s = gwarp; s < nsl; s += nwarps) {
      const int i = s * kSlice + lane;
      if (i < N) a.phi[i] = a.dsqinv[i] * (bb[0] == 0.0 ? a.b[i] : a.x[i]);  // free b == 0: x = b
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.res->pcg_iters = it;
      advance_history(a);
      a.res->pcg_status = status;
      a.res->pcg_relres = bb[0] > 0.0 ? sqrt(rr64 / bb[0]) : 0.0;
      a.res->pcg_bnorm = sqrt(bb[0]);
      a.res->pcg_outer = outer;
      if (status != AVIP_OK && a.sc->status == AVIP_OK) a.sc->status = status;
    }
    return;
  }
timeout:
  if (threadIdx.x == 0) {
    atomicExch(&a.sync->abort, 1);
    a.res->pcg_status = AVIP_ETIMEOUT;
    atomicCAS(&a.sc->status, AVIP_OK, AVIP_ETIMEOUT);
  }
}

static const void* mixed_kernel_ptr(int tpb) {
  switch (tpb) {
    case 256: return (const void*)pcg_mixed_kernel<256>;
    case 512: return (const void*)pcg_mixed_kernel<512>;
    case 1024: return (const void*)pcg_mixed_kernel<1024>;
    default: return (const void*)pcg_mixed_kernel<768>;
  }
}

PcgPlan pcg_mixed_plan(int nslices, int requested_tpb) {
  PcgPlan pl;
  pl.kind = 4;
  pl.tpb = (requested_tpb == 256 || requested_tpb == 512 || requested_tpb == 1024) ? requested_tpb : 768;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mixed_kernel_ptr(pl.tpb), pl.tpb, 0);
  const int wpb = pl.tpb / kSlice;
  pl.blocks = std::max(1, std::min(occ * sms, (nslices + wpb - 1) / wpb));
  return pl;
}

cudaError_t launch_pcg_mixed(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.blocks);
  cfg.blockDim = dim3(pl.tpb);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* kargs[] = {const_cast<PcgArgs*>(&args)};
  return cudaLaunchKernelExC(&cfg, mixed_kernel_ptr(pl.tpb), kargs);
}

}  // namespace avip
