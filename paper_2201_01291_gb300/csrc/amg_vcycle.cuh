// Smoothed-aggregation AMG V-cycle shared by the whole-GPU cooperative solvers (grid-wide
// barriers) and the batched solver (one thread-block cluster per instance, cluster barriers).
//
// `Ops` supplies the synchronisation of the participating threads: barrier() completes every
// vector written before it, sum(v) returns the sum of v over all participants (and is a
// barrier too); both return false if a wait was abandoned.  gwarp / nwarps number the
// participating warps.
#pragma once
#include <cooperative_groups.h>

#include "avip_internal.h"
#include "grid_sync.cuh"
#include "sell.cuh"

namespace avip {

// Per-thread accumulation of a dot product: FP64 fused multiply-adds, or compensated (Kahan)
// FP32 sums in the mixed-precision solve.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float y = a * b - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// One V-cycle: x0 = M b0 (level 0 takes b0 and x0 instead of the hierarchy's own vectors).
// On entry b0 and d_0 = D^-1 b0 / theta_0 are complete (written before the last barrier).
// Returns b0.x0 in rz (grid-reduced, also the barrier after which x0 is complete); false if a
// wait was abandoned.  T = double, or float for the inner solve of the mixed-precision path.
template <typename T, class Ops>
__device__ bool vcycle(const AmgDevT<T>* __restrict__ H, const T* __restrict__ b0, T* __restrict__ x0, Ops& ops,
                       int gwarp, int nwarps, int lane, double& rz) {
  const int nl = H->nlev;
  for (int l = 0; l + 1 < nl; ++l) {
    const AmgLevelT<T>* __restrict__ L = H->L + l;
    const SellMatT<T> A = L->A;
    const int n = L->n;
    const T* __restrict__ dinv = L->dinv;
    const T* __restrict__ b = l == 0 ? b0 : L->b;
    T* __restrict__ x = l == 0 ? x0 : L->x;
    T* __restrict__ d = L->d;
    T* __restrict__ r = L->r;
    {
      const T c1 = (T)L->c1, c2 = (T)L->c2;
      // second Chebyshev step from x = d0: r1 = b - A d0, x = d0 + c1 d0 + c2 D^-1 r1
      for (int sl = gwarp; sl < A.nslices; sl += nwarps) {
        const int i = sl * kSlice + lane;
        if (i >= n) continue;
        const T di = d[i];
        const T r1 = b[i] - sellmat_row_dot(A, sl, lane, i, (const T*)d);
        x[i] = di + fma_t(c1, di, c2 * dinv[i] * r1);
      }
    }
    if (!ops.barrier()) return false;
    // residual
    for (int sl = gwarp; sl < A.nslices; sl += nwarps) {
      const int i = sl * kSlice + lane;
      if (i >= n) continue;
      r[i] = b[i] - sellmat_row_dot(A, sl, lane, i, (const T*)x);
    }
    if (!ops.barrier()) return false;
    {  // restriction, and the first Chebyshev direction of the next level
      const AmgLevelT<T>* __restrict__ C = H->L + l + 1;
      const SellMatT<T> R = L->R;
      const int nc = C->n;
      const T c_inv_theta = (T)C->inv_theta;
      const T* __restrict__ cdinv = C->dinv;
      T* __restrict__ cb = C->b;
      T* __restrict__ cd = C->d;
      for (int sl = gwarp; sl < R.nslices; sl += nwarps) {
        const int j = sl * kSlice + lane;
        if (j >= nc) continue;
        const T bj = sellmat_row_dot(R, sl, lane, j, (const T*)r);
        cb[j] = bj;
        cd[j] = cdinv[j] * bj * c_inv_theta;
      }
    }
    if (!ops.barrier()) return false;
  }
  {  // coarsest level: dense inverse, one warp per row (a one-level hierarchy ends here: b0.x0)
    const AmgLevelT<T>* __restrict__ C = H->L + nl - 1;
    const int n = H->nc;
    const T* __restrict__ cinv = H->cinv;
    const T* __restrict__ cb = nl == 1 ? b0 : C->b;
    T* __restrict__ cx = nl == 1 ? x0 : C->x;
    DotAcc<T> acc;
    for (int row = gwarp; row < n; row += nwarps) {
      T s = T(0);
      for (int k = lane; k < n; k += 32) s = fma_t(__ldg(cinv + (size_t)row * n + k), __ldcg(cb + k), s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        cx[row] = s;
        if (nl == 1) acc.add(__ldcg(cb + row), s);
      }
    }
    if (nl == 1) {
      double av[1] = {acc.value()};
      if (!ops.sum(av)) return false;
      rz = av[0];
    } else if (!ops.barrier()) {
      return false;
    }
  }
  for (int l = nl - 2; l >= 0; --l) {
    const AmgLevelT<T>* __restrict__ L = H->L + l;
    const SellMatT<T> A = L->A;
    const int n = L->n;
    const T* __restrict__ dinv = L->dinv;
    const T* __restrict__ b = l == 0 ? b0 : L->b;
    T* __restrict__ x = l == 0 ? x0 : L->x;
    T* __restrict__ d = L->d;
    T* __restrict__ r = L->r;
    {  // prolongation
      const SellMatT<T> P = L->P;
      const T* __restrict__ cx = H->L[l + 1].x;
      for (int sl = gwarp; sl < A.nslices; sl += nwarps) {
        const int i = sl * kSlice + lane;
        if (i >= n) continue;
        x[i] += sellmat_row_dot(P, sl, lane, i, cx);
      }
    }
    if (!ops.barrier()) return false;
    const T inv_theta = (T)L->inv_theta, c1 = (T)L->c1, c2 = (T)L->c2;
    // first post-smoothing step: r = b - A x, d = D^-1 r / theta (x updated in the next phase)
    for (int sl = gwarp; sl < A.nslices; sl += nwarps) {
      const int i = sl * kSlice + lane;
      if (i >= n) continue;
      const T ri = b[i] - sellmat_row_dot(A, sl, lane, i, (const T*)x);
      r[i] = ri;
      d[i] = dinv[i] * ri * inv_theta;
    }
    if (!ops.barrier()) return false;
    // second step: r1 = r - A d, x += d + c1 d + c2 D^-1 r1
    DotAcc<T> acc;
    for (int sl = gwarp; sl < A.nslices; sl += nwarps) {
      const int i = sl * kSlice + lane;
      if (i >= n) continue;
      const T di = d[i];
      const T r1 = r[i] - sellmat_row_dot(A, sl, lane, i, (const T*)d);
      const T xi = x[i] + di + fma_t(c1, di, c2 * dinv[i] * r1);
      x[i] = xi;
      if (l == 0) acc.add(b[i], xi);
    }
    if (l == 0) {
      double av[1] = {acc.value()};
      if (!ops.sum(av)) return false;
      rz = av[0];
    } else if (!ops.barrier()) {
      return false;
    }
  }
  return true;
}

// CG preconditioned by the V-cycle on the scaled system (the whole solve of kinds 8 and the
// batched AMG solve): warm start, b', true-residual checks and restarts, phi = D^-1/2 x.
// `leader` is the one thread that writes the solve statistics.  Returns false if a wait was
// abandoned (grid barriers only).
template <class Ops>
__device__ bool amg_cg_solve(const PcgArgs& a, Ops& ops, int gwarp, int nwarps, int lane, bool leader) {
  constexpr int kMaxRestarts = 8;
  const int N = a.A.N, nsl = a.A.nslices;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
  const AmgDev* __restrict__ H = a.amg;
  const double* __restrict__ dinv0 = H->L[0].dinv;
  double* __restrict__ d0 = H->L[0].d;
  double* __restrict__ z = a.z;  // preconditioned residual (the V-cycle's finest solution)
  const double inv_theta0 = H->L[0].inv_theta;

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
  if (!ops.sum(bb)) return false;
  {
    const double thresh = a.rtol * a.rtol * bb[0];
    double rz = 0.0, rr_true = 0.0;
    bool check = true, fresh = true;
    int it = 0, restarts = 0, status = AVIP_OK;
    if (bb[0] == 0.0) {
      for (int s = gwarp; s < nsl; s += nwarps) {
        const int i = s * kSlice + lane;
        if (i < N) a.x[i] = a.b[i];  // free b == 0: x = b
      }
    } else {
      while (true) {
        if (check || it >= a.max_iter) {
          // ---- true residual r = b' - A x (x complete); first Chebyshev direction of level 0
          double r2[1] = {0.0};
          for (int s = gwarp; s < nsl; s += nwarps) {
            const int i = s * kSlice + lane;
            if (i >= N) continue;
            const double r = a.b[i] - sell_row_dot(a.A, s, lane, i, a.x);
            a.r[i] = r;
            d0[i] = dinv0[i] * r * inv_theta0;
            r2[0] = fma(r, r, r2[0]);
          }
          if (!ops.sum(r2)) return false;
          rr_true = r2[0];
          if (rr_true <= thresh) break;
          if (!isfinite(rr_true)) {  // non-finite data: stop at once
            status = AVIP_ENAN;
            break;
          }
          if (it >= a.max_iter || (it > 0 && restarts >= kMaxRestarts)) {
            status = AVIP_ENOTCONV;
            break;
          }
          if (it > 0) ++restarts;
          fresh = true;
          check = false;
        }
        // ---- z = M r (r and the level-0 direction complete)
        double rz_new = 0.0;
        if (!vcycle(H, (const double*)a.r, z, ops, gwarp, nwarps, lane, rz_new)) return false;
        if (!(rz_new > 0.0) || !isfinite(rz_new)) {  // the preconditioned residual lost positivity
          if (it == 0 || restarts >= kMaxRestarts) {
            status = AVIP_ENOTCONV;
            break;
          }
          ++it;
          check = true;
          continue;
        }
        const double beta = fresh ? 0.0 : rz_new / rz;
        rz = rz_new;
        fresh = false;
        // ---- phase A: w = A z, q = w + beta q, p = z + beta p, p.q -> alpha
        double pq[1] = {0.0};
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          const double zi = __ldcg(z + i);  // with one level, z rows come from other warps
          const double w = sell_row_dot(a.A, s, lane, i, z);
          const double qn = beta == 0.0 ? w : fma(beta, a.q_ap[i], w);
          const double pn = beta == 0.0 ? zi : fma(beta, a.p[i], zi);
          a.q_ap[i] = qn;
          a.p[i] = pn;
          pq[0] = fma(pn, qn, pq[0]);
        }
        if (!ops.sum(pq)) return false;
        const double alpha = rz / pq[0];
        // ---- phase B: x += alpha p, r -= alpha q, r.r; first direction of level 0
        double rn[1] = {0.0};
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          a.x[i] = fma(alpha, a.p[i], a.x[i]);
          const double r = fma(-alpha, a.q_ap[i], a.r[i]);
          a.r[i] = r;
          d0[i] = dinv0[i] * r * inv_theta0;
          rn[0] = fma(r, r, rn[0]);
        }
        if (!ops.sum(rn)) return false;
        check = rn[0] <= thresh || !isfinite(rn[0]);
        ++it;
      }
    }
    // ---- phi = D^-1/2 x
    for (int s = gwarp; s < nsl; s += nwarps) {
      const int i = s * kSlice + lane;
      if (i < N) a.phi[i] = a.dsqinv[i] * a.x[i];
    }
    if (leader) {
      a.res->pcg_iters = it;
      if (a.phi1) *a.hist = *a.hist < 2 ? *a.hist + 1 : 2;
      a.res->pcg_status = status;
      a.res->pcg_relres = bb[0] > 0.0 ? sqrt(rr_true / bb[0]) : 0.0;
      a.res->pcg_bnorm = sqrt(bb[0]);
      if (status != AVIP_OK && a.sc->status == AVIP_OK) a.sc->status = status;
    }
    return true;
  }
}


// Mixed-precision solve with the FP32 hierarchy (kind 10 and the batched mixed form): FP64
// outer residual and correction, FP32 inner CG preconditioned by the FP32 V-cycle.
template <class Ops>
__device__ bool amg_mixed_solve(const PcgArgs& a, Ops& ops, int gwarp, int nwarps, int lane, bool leader) {
  const int N = a.A.N, nsl = a.A.nslices;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
  const AmgDevT<float>* __restrict__ H = a.amg32;
  const SellMatT<float> A32 = H->L[0].A;
  const float* __restrict__ dinv0 = H->L[0].dinv;
  float* __restrict__ d0 = H->L[0].d;
  const float inv_theta0 = (float)H->L[0].inv_theta;
  float* __restrict__ r32 = a.r32;
  float* __restrict__ e32 = a.e32;
  float* __restrict__ p32 = a.p32;
  float* __restrict__ q32 = a.q32;
  float* __restrict__ z32 = a.z32;

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
  if (!ops.sum(bb)) return false;
  {
    const double thresh = a.rtol * a.rtol * bb[0];
    int it = 0, outer = 0, status = AVIP_OK;
    double rr64 = 0.0;
    while (true) {
      // ---- FP64 residual of the FP64 iterate (x complete)
      double r2[1] = {0.0};
      for (int s = gwarp; s < nsl; s += nwarps) {
        const int i = s * kSlice + lane;
        if (i >= N) continue;
        const double r = a.b[i] - sell_row_dot(a.A, s, lane, i, a.x);
        a.r[i] = r;
        r2[0] = fma(r, r, r2[0]);
      }
      if (!ops.sum(r2)) return false;
      rr64 = r2[0];
      if (!isfinite(rr64)) {
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
      const double rnorm = sqrt(rr64), rscale = 1.0 / rnorm;
      // ---- FP32 right-hand side r / ||r||, e = 0, first V-cycle direction
      double g0[1];
      {
        DotAcc<float> k;
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          const float r = (float)(a.r[i] * rscale);
          r32[i] = r;
          e32[i] = 0.f;
          d0[i] = dinv0[i] * r * inv_theta0;
          k.add(r, r);
        }
        g0[0] = k.value();
      }
      if (!ops.sum(g0)) return false;
      const double inner_thresh = a.inner_rtol * a.inner_rtol * g0[0];
      double rr = g0[0], rz = 0.0;
      bool fresh = true;
      while (rr > inner_thresh && it < a.max_iter) {
        double rz_new = 0.0;
        if (!vcycle(H, (const float*)r32, z32, ops, gwarp, nwarps, lane, rz_new)) return false;
        if (!(rz_new > 0.0) || !isfinite(rz_new)) break;  // refine with what the inner solve has
        const float beta = fresh ? 0.f : (float)(rz_new / rz);
        rz = rz_new;
        fresh = false;
        DotAcc<float> kpq;
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          const float zi = __ldcg(z32 + i);
          const float w = sellmat_row_dot(A32, s, lane, i, (const float*)z32);
          const float qn = beta == 0.f ? w : fmaf(beta, q32[i], w);  // (restart: old p, q unused)
          const float pn = beta == 0.f ? zi : fmaf(beta, p32[i], zi);
          q32[i] = qn;
          p32[i] = pn;
          kpq.add(pn, qn);
        }
        double pq[1] = {kpq.value()};
        if (!ops.sum(pq)) return false;
        const float alpha = (float)(rz / pq[0]);
        DotAcc<float> krr;
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          e32[i] = fmaf(alpha, p32[i], e32[i]);
          const float r = fmaf(-alpha, q32[i], r32[i]);
          r32[i] = r;
          d0[i] = dinv0[i] * r * inv_theta0;
          krr.add(r, r);
        }
        double rn[1] = {krr.value()};
        if (!ops.sum(rn)) return false;
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
        a.x[i] = fma(rnorm, (double)e32[i], a.x[i]);
      }
      double z0[1] = {0.0};
      if (!ops.sum(z0)) return false;  // x complete before the next residual
    }
    for (int s = gwarp; s < nsl; s += nwarps) {
      const int i = s * kSlice + lane;
      if (i < N) a.phi[i] = a.dsqinv[i] * (bb[0] == 0.0 ? a.b[i] : a.x[i]);  // free b == 0: x = b
    }
    if (leader) {
      a.res->pcg_iters = it;
      if (a.phi1) *a.hist = *a.hist < 2 ? *a.hist + 1 : 2;
      a.res->pcg_outer = outer;
      a.res->pcg_status = status;
      a.res->pcg_relres = bb[0] > 0.0 ? sqrt(rr64 / bb[0]) : 0.0;
      a.res->pcg_bnorm = sqrt(bb[0]);
      if (status != AVIP_OK && a.sc->status == AVIP_OK) a.sc->status = status;
    }
    return true;
  }
}


// Grid-wide synchronisation of a cooperative launch (counter barrier of grid_sync.cuh).
struct GridOps {
  FlagSync& fs;
  double* smem;
  __device__ bool barrier() { return grid_barrier(fs); }
  template <int NV>
  __device__ bool sum(double (&v)[NV]) {
    return grid_allsum<NV>(v, fs, smem);
  }
};

// Synchronisation of one thread-block cluster: hardware cluster barrier (release / acquire at
// cluster scope, so global-memory writes of the cluster are visible after it) and sums through
// distributed shared memory (at most 32 CTAs; deterministic: fixed shuffle tree over the ranks).
// `part` (2 x 4 doubles), `wsum` (32 x 4 doubles) and `res` (4 doubles) are the calling CTA's
// shared scratch.
struct ClusterOps {
  cooperative_groups::cluster_group cl;
  double* part;  // [2][4]: this CTA's partials, double-buffered
  double* wsum;  // [32][4]: warp partials
  double* res;   // [4]: cluster totals for this CTA's threads
  unsigned seq;
  __device__ bool barrier() {
    cl.sync();
    return true;
  }
  template <int NV>
  __device__ bool sum(double (&v)[NV]) {
    static_assert(NV <= 4, "cluster sum: at most 4 values");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) wsum[warp * 4 + k] = t;
    }
    __syncthreads();
    const int buf = seq & 1;
    ++seq;
    if (threadIdx.x < NV) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += wsum[w * 4 + threadIdx.x];
      part[buf * 4 + threadIdx.x] = t;
    }
    cl.sync();
    // warp 0 gathers the C partials (lane r reads rank r) and reduces them with a fixed
    // shuffle tree; the totals reach the other warps through shared memory
    if (warp == 0) {
      const int C = (int)cl.num_blocks();
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double t = lane < C ? *cl.map_shared_rank(part + buf * 4 + k, lane) : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) res[k] = t;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = res[k];
    return true;
  }
};

}  // namespace avip
