// Cluster-resident Jacobi-PCG (FP64) for meshes that fit in the shared memory of one
// thread-block cluster.
//
// One cluster of C CTAs (C = 16 when the device allows non-portable clusters, else 8) solves
// the whole system.  CTA `rank` owns a contiguous range of SELL-32 slices; its rows' vectors
// x, r, p, q, b and (when it fits) its slice of the matrix stay in that CTA's shared memory
// for the whole solve.  Each CTA also keeps a halo: the x and r entries of rows owned by other
// CTAs that its rows reference.  Halo entries are *pushed*: when a row updates r (or x) it
// stores the new value straight into the halo slots of the CTAs that read it, through
// distributed shared memory (fire-and-forget stores), and the cluster barrier that follows
// makes them visible.  Every read of an iteration is therefore a local shared-memory read.
// Reductions are pushed the same way: every CTA writes its partial into every CTA's slot
// table, one cluster barrier, then each CTA adds the C partials locally in rank order
// (identical totals everywhere; deterministic).  A reduction costs one hardware cluster
// barrier (~0.3 us on GB300) instead of the ~3.5 us of a grid-wide reduction, which is what
// bounds small meshes with the persistent grid kernels.
//
// The same symmetric Jacobi scaling and CG recurrences as the grid-wide kernel are used.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "avip_internal.h"
#include "amg_vcycle.cuh"

namespace cg = cooperative_groups;

namespace avip {

constexpr int kClusterTPB = 512;
constexpr size_t kClusterSmemMax = 212 * 1024;  // dynamic part; the static part below is ~9 KB

// Static shared memory of the cluster solves (declared once per kernel).
struct ClusterShared {
  double part[2][16][4];        // reduction partials [parity][source rank][value]
  double thr[2 * kClusterTPB];  // per-thread values of a block reduction
  double res[8];                // reduced totals and epilogue results
};

// Shared memory per CTA: xs[R + H], rs[R + H], ps[R], qs[R] (FP64), then, when the matrix
// fits, vals[max_elems] (FP64) and cols[max_elems] (int32 local indices).  b' stays in global
// memory (read only at the start and by the true-residual passes).
// One complete solve of the system described by (a, L) by the calling cluster.
__device__ void cluster_solve(const PcgArgs& a, const ClusterLayout& L, ClusterShared& sh) {
  if (solve_skipped(a.sc)) return;  // every CTA of the cluster reads the same status
  extern __shared__ __align__(16) double dsm[];
  auto& s_part = sh.part;
  auto& s_thr = sh.thr;
  auto& s_res = sh.res;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int R = L.rows, H = L.hmax;
  double* xs = dsm;
  double* rs = xs + R + H;
  double* ps = rs + R + H;
  double* qs = ps + R;
  double* vals = qs + R;
  int32_t* cols = reinterpret_cast<int32_t*>(vals + (L.mat_smem ? L.max_elems : 0));
  const int N = a.A.N, nsl = a.A.nslices;
  const int s0 = rank * L.spc, s1 = min(nsl, s0 + L.spc);
  const int e0 = s0 < nsl ? __ldg(a.A.sl_ptr + s0) : 0;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
  unsigned seq = 0;

  // one row of A v, all reads local (own rows and pushed halo)
  auto row_dot = [&](int s, int l, int i, const double* v) -> double {
    const int w = __ldg(a.A.sl_w + s);
    const int rl = __ldg(a.A.rlen + i);
    const int base = __ldg(a.A.sl_ptr + s) + l - e0;
    double acc0 = 0.0, acc1 = 0.0;  // two chains halve the dependent FP64 latency
    for (int k = 0; k < w; k += 2) {
      if (k < rl) {
        const int e = base + k * kSlice;
        const int c = L.mat_smem ? cols[e] : __ldg(L.colL + e0 + e);
        const double av = L.mat_smem ? vals[e] : __ldg(a.A.aval + e0 + e);
        acc0 = fma(av, v[c], acc0);
      }
      if (k + 1 < rl) {
        const int e = base + (k + 1) * kSlice;
        const int c = L.mat_smem ? cols[e] : __ldg(L.colL + e0 + e);
        const double av = L.mat_smem ? vals[e] : __ldg(a.A.aval + e0 + e);
        acc1 = fma(av, v[c], acc1);
      }
    }
    return acc0 + acc1;
  };
  // push the value of own row i into the halo slots of the CTAs that read it
  auto push = [&](double* v, int i, double val) {
    const int p1 = __ldg(L.push_ptr + i + 1);
    for (int k = __ldg(L.push_ptr + i); k < p1; ++k) {
      const unsigned d = (unsigned)__ldg(L.push_dst + k);
      *cl.map_shared_rank(v + R + (int)(d & 0xffffffu), (int)(d >> 24)) = val;
    }
  };
  // cluster-wide sum of NV values with an epilogue evaluated once per CTA
  auto csum = [&](int NV, double* v, auto epi) {
    const int par = (++seq) & 1;
    // per-thread values -> shared memory -> warp 0 adds them (few warp-wide FP64 adds)
    for (int k = 0; k < NV; ++k) s_thr[k * kClusterTPB + threadIdx.x] = v[k];
    __syncthreads();
    if (warp == 0) {
      double bt[4] = {0.0, 0.0, 0.0, 0.0};
      for (int k = 0; k < NV; ++k) {
        constexpr int W = kClusterTPB / 32;
        double t[W];
#pragma unroll
        for (int w = 0; w < W; ++w) t[w] = s_thr[k * kClusterTPB + w * 32 + lane];
#pragma unroll
        for (int h = W / 2; h > 0; h >>= 1)
#pragma unroll
          for (int w = 0; w < h; ++w) t[w] += t[w + h];
        double u = t[0];
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        bt[k] = u;
      }
      // lane d pushes this CTA's partial into CTA d's table
      if (lane < C) {
        double* dst = cl.map_shared_rank(&s_part[par][rank][0], lane);
        for (int k = 0; k < NV; ++k) dst[k] = bt[k];
      }
    }
    cl.sync();  // all partials (and all pushed halo values) are visible
    if (warp == 0) {
      for (int k = 0; k < NV; ++k) {
        double t = lane < C ? s_part[par][lane][k] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_res[k] = t;
      }
      if (lane == 0) epi(s_res, s_res + 4);
    }
    __syncthreads();
    for (int k = 0; k < NV; ++k) v[k] = s_res[k];
  };
  auto none = [](const double*, double*) {};

  // ---- load the matrix slices, x = D^1/2 phi (pushed to the halos), b'
  if (L.mat_smem && s0 < nsl) {
    const int e1 = __ldg(a.A.sl_ptr + s1);
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      cols[e - e0] = __ldg(L.colL + e);
      vals[e - e0] = __ldg(a.A.aval + e);
    }
  }
  const double gain = dirichlet_gain(a);
  const int hist = history_length(a);
  double bb[1] = {0.0};
  for (int li = threadIdx.x; li < R; li += blockDim.x) {
    const int i = s0 * kSlice + li;
    double x = 0.0, b = 0.0;
    if (i < N) {
      x = a.dsq[i] * predict_phi(a, i, hist);
      if (a.use_density_rhs) {
        double rho = 0.0;
        if (a.rhs_src)
          rho = a.rhs_src[i];
        else
          for (int k = 0; k < a.ns; ++k) rho = fma(a.q[k], nb[(size_t)k * a.Npad + i], rho);
        b = fma(a.rhs_scale[i], rho, gain * a.lift[i]);
      } else {
        b = a.b[i];
      }
      if (a.rhs_scale[i] != 0.0) bb[0] = fma(b, b, bb[0]);  // free rows only: a Dirichlet row holds its value exactly
      else x = b;  // a Dirichlet unit row takes its (possibly ramped) value exactly
      push(xs, i, x);
      a.b[i] = b;
    }
    xs[li] = x;
    rs[li] = ps[li] = qs[li] = 0.0;
  }
  csum(1, bb, none);  // also the barrier after which x (own and halo) may be read
  const double thresh = a.rtol * a.rtol * bb[0];
  double rr = 0.0, beta = 0.0, rr_true = 0.0;
  bool check = true;
  int it = 0, restarts = 0, status = AVIP_OK;
  if (bb[0] == 0.0) {
    for (int li = threadIdx.x; li < R; li += blockDim.x) {  // free b == 0: x = b
      const int i = s0 * kSlice + li;
      xs[li] = i < N ? a.b[i] : 0.0;
    }
  } else {
    while (true) {
      if (check || it >= a.max_iter) {
        // ---- true residual r = b' - A x
        double r2[1] = {0.0};
        for (int s = s0 + warp; s < s1; s += nw) {
          const int i = s * kSlice + lane;
          const int li = i - s0 * kSlice;
          if (i >= N) continue;
          const double r = a.b[i] - row_dot(s, lane, i, xs);
          rs[li] = r;
          ps[li] = 0.0;
          qs[li] = 0.0;
          push(rs, i, r);
          r2[0] = fma(r, r, r2[0]);
        }
        csum(1, r2, none);
        rr_true = r2[0];
        if (rr_true <= thresh) break;
        if (!isfinite(rr_true)) {  // non-finite data: stop at once
          status = AVIP_ENAN;
          break;
        }
        if (it >= a.max_iter || (it > 0 && restarts >= 8)) {
          status = AVIP_ENOTCONV;
          break;
        }
        if (it > 0) ++restarts;
        rr = rr_true;
        beta = 0.0;
        check = false;
      }
      // ---- phase A: q = A r + beta q, p = r + beta p, p.q
      double pq[1] = {0.0};
      for (int s = s0 + warp; s < s1; s += nw) {
        const int i = s * kSlice + lane;
        const int li = i - s0 * kSlice;
        if (i >= N) continue;
        const double w = row_dot(s, lane, i, rs);
        const double qn = fma(beta, qs[li], w);
        const double pn = fma(beta, ps[li], rs[li]);
        qs[li] = qn;
        ps[li] = pn;
        pq[0] = fma(pn, qn, pq[0]);
      }
      const double rr_now = rr;
      csum(1, pq, [rr_now](const double* t, double* e) { e[0] = rr_now / t[0]; });
      const double alpha = s_res[4];
      // ---- phase B: update own rows, push r to the halos that read it
      double rn[1] = {0.0};
      for (int s = s0 + warp; s < s1; s += nw) {
        const int i = s * kSlice + lane;
        const int li = i - s0 * kSlice;
        if (i >= N) continue;
        xs[li] = fma(alpha, ps[li], xs[li]);
        const double r = fma(-alpha, qs[li], rs[li]);
        rs[li] = r;
        push(rs, i, r);
        rn[0] = fma(r, r, rn[0]);
      }
      csum(1, rn, [rr_now, thresh](const double* t, double* e) {
        e[0] = t[0] / rr_now;
        e[1] = (t[0] <= thresh || !isfinite(t[0])) ? 1.0 : 0.0;
      });
      beta = s_res[4];
      check = s_res[5] != 0.0;
      rr = rn[0];
      ++it;
      if (check || it >= a.max_iter) {
        // the true residual reads x of the halo: push it, then a barrier
        for (int s = s0 + warp; s < s1; s += nw) {
          const int i = s * kSlice + lane;
          if (i < N) push(xs, i, xs[i - s0 * kSlice]);
        }
        cl.sync();
      }
    }
  }
  // ---- phi = D^-1/2 x
  for (int li = threadIdx.x; li < R; li += blockDim.x) {
    const int i = s0 * kSlice + li;
    if (i < N) {
      a.phi[i] = a.dsqinv[i] * xs[li];
      a.x[i] = xs[li];
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    a.res->pcg_iters = it;
    advance_history(a);
    a.res->pcg_status = status;
    a.res->pcg_relres = bb[0] > 0.0 ? sqrt(rr_true / bb[0]) : 0.0;
    a.res->pcg_bnorm = sqrt(bb[0]);
    if (status != AVIP_OK && a.sc->status == AVIP_OK) a.sc->status = status;
  }
  cl.sync();  // no CTA leaves while another may still write into its shared memory
}

struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Mixed precision in one cluster: FP32 inner CG (FP32 matrix slices and vectors in shared
// memory, Kahan-compensated FP32 dot products), FP64 iterative refinement (FP64 iterate in
// shared memory, FP64 residual with the FP64 matrix read from global memory).
// Shared memory per CTA: x64[R + H] (FP64), r64[R] (FP64), r32[R + H], e32[R], p32[R], q32[R]
// (FP32), then vals32[max_elems] (FP32) and cols[max_elems] (int32) when the matrix fits.
__device__ void cluster_solve_mixed(const PcgArgs& a, const ClusterLayout& L, ClusterShared& sh) {
  if (solve_skipped(a.sc)) return;  // every CTA of the cluster reads the same status
  extern __shared__ __align__(16) double dsm[];
  auto& s_part = sh.part;
  auto& s_thr = sh.thr;
  auto& s_res = sh.res;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = (int)cl.num_blocks();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int R = L.rows, H = L.hmax;
  double* x64 = dsm;
  double* r64 = x64 + R + H;
  float* r32 = reinterpret_cast<float*>(r64 + R);
  float* e32 = r32 + R + H;
  float* p32 = e32 + R;
  float* q32 = p32 + R;
  float* vals = q32 + R;
  int32_t* cols = reinterpret_cast<int32_t*>(vals + (L.mat_smem ? L.max_elems : 0));
  const int N = a.A.N, nsl = a.A.nslices;
  const int s0 = rank * L.spc, s1 = min(nsl, s0 + L.spc);
  const int e0 = s0 < nsl ? __ldg(a.A.sl_ptr + s0) : 0;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
  unsigned seq = 0;

  auto colof = [&](int e) -> int { return L.mat_smem ? cols[e] : __ldg(L.colL + e0 + e); };
  auto row_dot32 = [&](int s, int l, int i, const float* v) -> float {
    const int w = __ldg(a.A.sl_w + s);
    const int rl = __ldg(a.A.rlen + i);
    const int base = __ldg(a.A.sl_ptr + s) + l - e0;
    float acc = 0.f;
    for (int k = 0; k < w; ++k) {
      if (k < rl) {
        const int e = base + k * kSlice;
        const float av = L.mat_smem ? vals[e] : __ldg(a.aval32 + e0 + e);
        acc = fmaf(av, v[colof(e)], acc);
      }
    }
    return acc;
  };
  auto row_dot64 = [&](int s, int l, int i, const double* v) -> double {
    const int w = __ldg(a.A.sl_w + s);
    const int rl = __ldg(a.A.rlen + i);
    const int base = __ldg(a.A.sl_ptr + s) + l - e0;
    double acc = 0.0;
    for (int k = 0; k < w; ++k) {
      if (k < rl) {
        const int e = base + k * kSlice;
        acc = fma(__ldg(a.A.aval + e0 + e), v[colof(e)], acc);
      }
    }
    return acc;
  };
  auto push64 = [&](double* v, int i, double val) {
    const int p1 = __ldg(L.push_ptr + i + 1);
    for (int k = __ldg(L.push_ptr + i); k < p1; ++k) {
      const unsigned d = (unsigned)__ldg(L.push_dst + k);
      *cl.map_shared_rank(v + R + (int)(d & 0xffffffu), (int)(d >> 24)) = val;
    }
  };
  auto push32 = [&](float* v, int i, float val) {
    const int p1 = __ldg(L.push_ptr + i + 1);
    for (int k = __ldg(L.push_ptr + i); k < p1; ++k) {
      const unsigned d = (unsigned)__ldg(L.push_dst + k);
      *cl.map_shared_rank(v + R + (int)(d & 0xffffffu), (int)(d >> 24)) = val;
    }
  };
  auto csum = [&](int NV, double* v, auto epi) {
    const int par = (++seq) & 1;
    for (int k = 0; k < NV; ++k) s_thr[k * kClusterTPB + threadIdx.x] = v[k];
    __syncthreads();
    if (warp == 0) {
      double bt[4] = {0.0, 0.0, 0.0, 0.0};
      for (int k = 0; k < NV; ++k) {
        constexpr int W = kClusterTPB / 32;
        double t[W];
#pragma unroll
        for (int w = 0; w < W; ++w) t[w] = s_thr[k * kClusterTPB + w * 32 + lane];
#pragma unroll
        for (int h = W / 2; h > 0; h >>= 1)
#pragma unroll
          for (int w = 0; w < h; ++w) t[w] += t[w + h];
        double u = t[0];
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        bt[k] = u;
      }
      if (lane < C) {
        double* dst = cl.map_shared_rank(&s_part[par][rank][0], lane);
        for (int k = 0; k < NV; ++k) dst[k] = bt[k];
      }
    }
    cl.sync();
    if (warp == 0) {
      for (int k = 0; k < NV; ++k) {
        double t = lane < C ? s_part[par][lane][k] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_res[k] = t;
      }
      if (lane == 0) epi(s_res, s_res + 4);
    }
    __syncthreads();
    for (int k = 0; k < NV; ++k) v[k] = s_res[k];
  };
  auto none = [](const double*, double*) {};

  if (L.mat_smem && s0 < nsl) {
    const int e1 = __ldg(a.A.sl_ptr + s1);
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      cols[e - e0] = __ldg(L.colL + e);
      vals[e - e0] = __ldg(a.aval32 + e);
    }
  }
  const double gain = dirichlet_gain(a);
  const int hist = history_length(a);
  double bb[1] = {0.0};
  for (int li = threadIdx.x; li < R; li += blockDim.x) {
    const int i = s0 * kSlice + li;
    double x = 0.0;
    if (i < N) {
      x = a.dsq[i] * predict_phi(a, i, hist);
      double b;
      if (a.use_density_rhs) {
        double rho = 0.0;
        if (a.rhs_src)
          rho = a.rhs_src[i];
        else
          for (int k = 0; k < a.ns; ++k) rho = fma(a.q[k], nb[(size_t)k * a.Npad + i], rho);
        b = fma(a.rhs_scale[i], rho, gain * a.lift[i]);
      } else {
        b = a.b[i];
      }
      a.b[i] = b;
      if (a.rhs_scale[i] != 0.0) bb[0] = fma(b, b, bb[0]);  // free rows only: a Dirichlet row holds its value exactly
      else x = b;  // a Dirichlet unit row takes its (possibly ramped) value exactly
      push64(x64, i, x);
    }
    x64[li] = x;
    r64[li] = 0.0;
    r32[li] = e32[li] = p32[li] = q32[li] = 0.f;
  }
  csum(1, bb, none);
  const double thresh = a.rtol * a.rtol * bb[0];
  int it = 0, outer = 0, status = AVIP_OK;
  double rr64 = 0.0;
  if (bb[0] == 0.0)
    for (int li = threadIdx.x; li < R; li += blockDim.x) {  // free b == 0: x = b
      const int i = s0 * kSlice + li;
      x64[li] = i < N ? a.b[i] : 0.0;
    }
  while (bb[0] != 0.0) {
    // ---- FP64 residual of the FP64 iterate
    double r2[1] = {0.0};
    for (int s = s0 + warp; s < s1; s += nw) {
      const int i = s * kSlice + lane;
      const int li = i - s0 * kSlice;
      if (i >= N) continue;
      const double r = a.b[i] - row_dot64(s, lane, i, x64);
      r64[li] = r;
      r2[0] = fma(r, r, r2[0]);
    }
    csum(1, r2, none);
    rr64 = r2[0];
    if (!isfinite(rr64)) {  // non-finite right-hand side or iterate: stop, never loop on NaN
      status = AVIP_ENAN;
      break;
    }
    if (rr64 <= thresh) break;
    if (it >= a.max_iter) {
      status = AVIP_ENOTCONV;
      break;
    }
    ++outer;
    const int it_outer = it;
    const double rnorm = sqrt(rr64), rscale = 1.0 / rnorm;
    double g0[1];
    {
      KahanF k;
      for (int s = s0 + warp; s < s1; s += nw) {
        const int i = s * kSlice + lane;
        const int li = i - s0 * kSlice;
        if (i >= N) continue;
        const float r = (float)(r64[li] * rscale);
        r32[li] = r;
        e32[li] = p32[li] = q32[li] = 0.f;
        push32(r32, i, r);
        k.add(r * r);
      }
      g0[0] = k.value();
    }
    csum(1, g0, none);
    const double inner_thresh = a.inner_rtol * a.inner_rtol * g0[0];
    double rr = g0[0];
    float beta = 0.f;
    while (rr > inner_thresh && it < a.max_iter) {
      KahanF kpq;
      for (int s = s0 + warp; s < s1; s += nw) {
        const int i = s * kSlice + lane;
        const int li = i - s0 * kSlice;
        if (i >= N) continue;
        const float w = row_dot32(s, lane, i, r32);
        const float qn = fmaf(beta, q32[li], w);
        const float pn = fmaf(beta, p32[li], r32[li]);
        q32[li] = qn;
        p32[li] = pn;
        kpq.add(pn * qn);
      }
      double pq[1] = {kpq.value()};
      const double rr_now = rr;
      csum(1, pq, [rr_now](const double* t, double* e) { e[0] = rr_now / t[0]; });
      const float alpha = (float)s_res[4];
      KahanF krr;
      for (int s = s0 + warp; s < s1; s += nw) {
        const int i = s * kSlice + lane;
        const int li = i - s0 * kSlice;
        if (i >= N) continue;
        e32[li] = fmaf(alpha, p32[li], e32[li]);
        const float r = fmaf(-alpha, q32[li], r32[li]);
        r32[li] = r;
        push32(r32, i, r);
        krr.add(r * r);
      }
      double rn[1] = {krr.value()};
      csum(1, rn, [rr_now](const double* t, double* e) { e[0] = t[0] / rr_now; });
      beta = (float)s_res[4];
      rr = rn[0];
      ++it;
    }
    if (it == it_outer) {  // the inner solve could not start: no progress is possible
      status = AVIP_ENOTCONV;
      break;
    }
    // ---- FP64 correction, pushed to the halos before the next residual
    for (int s = s0 + warp; s < s1; s += nw) {
      const int i = s * kSlice + lane;
      const int li = i - s0 * kSlice;
      if (i >= N) continue;
      const double x = fma(rnorm, (double)e32[li], x64[li]);
      x64[li] = x;
      push64(x64, i, x);
    }
    cl.sync();
  }
  for (int li = threadIdx.x; li < R; li += blockDim.x) {
    const int i = s0 * kSlice + li;
    if (i < N) {
      a.phi[i] = a.dsqinv[i] * x64[li];
      a.x[i] = x64[li];
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    a.res->pcg_iters = it;
    advance_history(a);
    a.res->pcg_outer = outer;
    a.res->pcg_status = status;
    a.res->pcg_relres = bb[0] > 0.0 ? sqrt(rr64 / bb[0]) : 0.0;
    a.res->pcg_bnorm = sqrt(bb[0]);
    if (status != AVIP_OK && a.sc->status == AVIP_OK) a.sc->status = status;
  }
  cl.sync();
}

__global__ void __launch_bounds__(kClusterTPB, 1) pcg_cluster_mixed_kernel(PcgArgs a, ClusterLayout L) {
  __shared__ ClusterShared sh;
  cluster_solve_mixed(a, L, sh);
}

__global__ void __launch_bounds__(kClusterTPB, 1) pcg_cluster_kernel(PcgArgs a, ClusterLayout L) {
  __shared__ ClusterShared sh;
  cluster_solve(a, L, sh);
}

// AMG-preconditioned CG of one instance on one cluster: the rows of every level are shared by
// the cluster's warps, barriers are cluster barriers and sums go through distributed shared
// memory (the same V-cycle and CG as the whole-GPU kernel, solver kind 8).
template <class Ops = ClusterOps>
__device__ void cluster_amg_solve(const PcgArgs& a, double* part, double* wsum) {
  if (solve_skipped(a.sc)) return;  // every CTA of the cluster reads the same status
  cg::cluster_group cl = cg::this_cluster();
  Ops ops{cl, part, wsum, wsum + 32 * 4, 0u};
  const int wpb = (int)(blockDim.x >> 5), rank = (int)cl.block_rank();
  const int gw = rank * wpb + (int)(threadIdx.x >> 5), nw = (int)cl.num_blocks() * wpb, lane = (int)(threadIdx.x & 31);
  if (a.amg32)  // FP32 hierarchy (default), else FP64
    amg_cg_solve<float>(a, a.amg32, a.z, ops, gw, nw, lane, rank == 0 && threadIdx.x == 0);
  else
    amg_cg_solve<double>(a, a.amg, a.z, ops, gw, nw, lane, rank == 0 && threadIdx.x == 0);
  cl.sync();  // the next instance reuses the sum buffers
}

// (wsum holds 32 x 4 warp partials followed by the 4 totals.)

// The same for a mixed-precision instance with an FP32 hierarchy (solver kind 10).
template <class Ops = ClusterOps>
__device__ void cluster_amg_mixed_solve(const PcgArgs& a, double* part, double* wsum) {
  if (solve_skipped(a.sc)) return;
  cg::cluster_group cl = cg::this_cluster();
  Ops ops{cl, part, wsum, wsum + 32 * 4, 0u};
  const int wpb = (int)(blockDim.x >> 5), rank = (int)cl.block_rank();
  amg_mixed_solve(a, ops, rank * wpb + (int)(threadIdx.x >> 5), (int)cl.num_blocks() * wpb,
                  (int)(threadIdx.x & 31), rank == 0 && threadIdx.x == 0);
  cl.sync();
}

// Batched, persistent: every resident cluster solves instances order[c], order[c + nclusters],
// ... (the order is sorted by decreasing size, so the largest solves start first).  Instances
// that carry an AMG hierarchy (solver kinds 8 and 10) are solved with it (FP64 CG, or the
// mixed-precision solve), the others with the shared-memory Jacobi-PCG (FP64 or mixed).
__global__ void __launch_bounds__(kClusterTPB, 1) pcg_cluster_batch_kernel(const PcgArgs* __restrict__ args,
                                                                            const ClusterLayout* __restrict__ lays,
                                                                            const int32_t* __restrict__ order,
                                                                            int count) {
  __shared__ ClusterShared sh;
  __shared__ double s_amg_part[2 * 4], s_amg_wsum[32 * 4 + 4];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int cid = blockIdx.x / C, ncl = gridDim.x / C;
  for (int j = cid; j < count; j += ncl) {
    const int k = order[j];
    const PcgArgs a = args[k];
    const ClusterLayout L = lays[k];
    if ((a.amg || a.amg32) && !a.amg_mixed)
      cluster_amg_solve(a, s_amg_part, s_amg_wsum);
    else if (a.amg32)
      cluster_amg_mixed_solve(a, s_amg_part, s_amg_wsum);
    else if (L.mixed)
      cluster_solve_mixed(a, L, sh);
    else
      cluster_solve(a, L, sh);
  }
}

// Largest cluster (16 or 8 CTAs) the device schedules for this kernel with `smem` bytes of
// dynamic shared memory per CTA; 0 if none.
static int cluster_size_supported(size_t smem) {
  cudaFuncSetAttribute(pcg_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(pcg_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterSmemMax);
  cudaFuncSetAttribute(pcg_cluster_mixed_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(pcg_cluster_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterSmemMax);
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kClusterTPB);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, pcg_cluster_kernel, &cfg) == cudaSuccess && n > 0) return c;
    cudaGetLastError();
  }
  return 0;
}

// Plan a cluster solve for the mesh, or return kind 0 if it does not fit.  The cluster kernel
// runs on C SMs only, so it is chosen only for meshes small enough that the grid-wide
// reduction latency, not FP64 throughput, would dominate (n_rows <= max_rows).  Fills the
// host arrays of the layout: local column indices, halo push lists.
PcgPlan pcg_cluster_plan_fixed(const HostMesh& m, int C, ClusterLayout* out, ClusterHost* hd, int mixed) {
  PcgPlan pl;
  pl.kind = 0;
  const int spc = (m.nslices + C - 1) / C;
  const int R = spc * kSlice;
  auto owner = [&](int c) { return (c / kSlice) / spc; };
  // halo slots per CTA: sorted distinct remote columns
  std::vector<std::vector<int32_t>> halo(C);
  int max_elems = 0;
  for (int r = 0; r < C; ++r) {
    const int s0 = r * spc, s1 = std::min(m.nslices, s0 + spc);
    if (s0 >= s1) continue;
    max_elems = std::max(max_elems, m.sl_ptr[s1] - m.sl_ptr[s0]);
    for (int s = s0; s < s1; ++s)
      for (int l = 0; l < kSlice; ++l) {
        const int i = s * kSlice + l;
        if (i >= m.N) continue;
        for (int k = 0; k < m.rlen[i]; ++k) {
          const int c = m.col[(int64_t)m.sl_ptr[s] + (int64_t)k * kSlice + l];
          if (owner(c) != r) halo[r].push_back(c);
        }
      }
    std::sort(halo[r].begin(), halo[r].end());
    halo[r].erase(std::unique(halo[r].begin(), halo[r].end()), halo[r].end());
  }
  int H = 0;
  for (auto& h : halo) H = std::max<int>(H, (int)h.size());
  const size_t vec = mixed ? (sizeof(double) * (2 * (size_t)R + (size_t)H) + sizeof(float) * (4 * (size_t)R + (size_t)H))
                           : sizeof(double) * (4 * (size_t)R + 2 * (size_t)H);
  const size_t mat = ((mixed ? sizeof(float) : sizeof(double)) + sizeof(int32_t)) * (size_t)max_elems;
  const int mat_smem = vec + mat <= kClusterSmemMax ? 1 : 0;
  const size_t smem = vec + (mat_smem ? mat : 0);
  if (smem > kClusterSmemMax) return pl;
  // local column indices and push lists
  hd->colL.assign(m.col.size(), 0);
  std::vector<std::vector<uint32_t>> dst(m.N);
  for (int r = 0; r < C; ++r) {
    const int s0 = r * spc, s1 = std::min(m.nslices, s0 + spc);
    for (int s = s0; s < s1; ++s)
      for (int l = 0; l < kSlice; ++l) {
        const int i = s * kSlice + l;
        if (i >= m.N) continue;
        for (int k = 0; k < m.rlen[i]; ++k) {
          const int64_t e = (int64_t)m.sl_ptr[s] + (int64_t)k * kSlice + l;
          const int c = m.col[e];
          if (owner(c) == r) {
            hd->colL[e] = c - r * R;
          } else {
            const int slot = (int)(std::lower_bound(halo[r].begin(), halo[r].end(), c) - halo[r].begin());
            hd->colL[e] = R + slot;
          }
        }
      }
    for (size_t h = 0; h < halo[r].size(); ++h) dst[halo[r][h]].push_back(((uint32_t)r << 24) | (uint32_t)h);
  }
  hd->push_ptr.assign(m.N + 1, 0);
  hd->push_dst.clear();
  for (int i = 0; i < m.N; ++i) {
    for (uint32_t d : dst[i]) hd->push_dst.push_back((int32_t)d);
    hd->push_ptr[i + 1] = (int32_t)hd->push_dst.size();
  }
  out->spc = spc;
  out->rows = R;
  out->hmax = H;
  out->max_elems = max_elems;
  out->mat_smem = mat_smem;
  out->mixed = mixed;
  pl.kind = mixed ? 6 : 5;
  pl.tpb = kClusterTPB;
  pl.blocks = C;
  pl.maxs = (int)smem;  // dynamic shared memory bytes
  return pl;
}

PcgPlan pcg_cluster_plan(const HostMesh& m, int max_rows, ClusterLayout* out, ClusterHost* hd, int mixed) {
  PcgPlan pl;
  pl.kind = 0;
  if (m.N > max_rows) return pl;
  for (int C : {16, 8}) {
    ClusterLayout L{};
    ClusterHost H;
    PcgPlan p = pcg_cluster_plan_fixed(m, C, &L, &H, mixed);
    if (p.kind == 0 || cluster_size_supported((size_t)p.maxs) < C) continue;
    *out = L;
    *hd = std::move(H);
    return p;
  }
  return pl;
}

cudaError_t launch_pcg_cluster(const PcgArgs& args, const PcgPlan& pl, const ClusterLayout& L, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.blocks);
  cfg.blockDim = dim3(pl.tpb);
  cfg.dynamicSmemBytes = (size_t)pl.maxs;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.blocks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (L.mixed) return cudaLaunchKernelEx(&cfg, pcg_cluster_mixed_kernel, args, L);
  return cudaLaunchKernelEx(&cfg, pcg_cluster_kernel, args, L);
}

// Standalone AMG solve on one thread-block cluster (solver kind 11): small and mid-size meshes
// whose solve is too short to occupy the whole GPU (FP64 CG with an FP32 or FP64 hierarchy, or
// the mixed-precision solve).  Other work, such as other requests of a server, can run beside it.
// 512 threads per CTA for small meshes, 768 above kAmgClusterWideRows rows (measured on one
// 16-CTA cluster: 150k nodes 218 -> 185 us per CG iteration, mixed 188 -> 155; 4k nodes 26.3 ->
// 28.5, so small meshes keep 512).
constexpr int kAmgClusterWideRows = 20000;
template <int TPB, class Ops>
__global__ void __launch_bounds__(TPB, 1) pcg_amg_cluster_kernel(PcgArgs a) {
  __shared__ double s_amg_part[2 * 4], s_amg_wsum[32 * 4 + 4];
  if (a.amg_mixed)
    cluster_amg_mixed_solve<Ops>(a, s_amg_part, s_amg_wsum);
  else
    cluster_amg_solve<Ops>(a, s_amg_part, s_amg_wsum);
}
static const void* amg_cluster_kernel_ptr(int tpb) {
  return tpb == 768 ? (const void*)pcg_amg_cluster_kernel<768, ClusterOpsT<6, 4>>
                    : (const void*)pcg_amg_cluster_kernel<kClusterTPB, ClusterOps>;
}

// Cluster of the standalone AMG cluster kernel for a mesh of n rows: `want` CTAs (2, 4, 8 or
// 16) when schedulable, else the largest schedulable of 16 and 8 (want = 0: 16, else 8); kind 0
// if none.
PcgPlan amg_cluster_plan(int want, int n) {
  PcgPlan pl;
  pl.kind = 0;
  const int tpb = n > kAmgClusterWideRows ? 768 : kClusterTPB;
  const void* fn = amg_cluster_kernel_ptr(tpb);
  cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c : {want, 16, 8}) {
    if (c <= 0) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(tpb);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) == cudaSuccess && nc > 0) {
      pl.kind = 11;
      pl.tpb = tpb;
      pl.blocks = c;
      pl.maxs = 0;
      return pl;
    }
    cudaGetLastError();
  }
  return pl;
}

cudaError_t launch_pcg_amg_cluster(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.blocks);
  cfg.blockDim = dim3(pl.tpb);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = pl.blocks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* kargs[] = {const_cast<PcgArgs*>(&args)};
  return cudaLaunchKernelExC(&cfg, amg_cluster_kernel_ptr(pl.tpb), kargs);
}

// Clusters of size C that can be resident at once with `smem` bytes per CTA.
int cluster_batch_capacity(int C, size_t smem) {
  cudaFuncSetAttribute(pcg_cluster_batch_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(pcg_cluster_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterSmemMax);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kClusterTPB);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, pcg_cluster_batch_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}


cudaError_t launch_pcg_cluster_batch(const PcgArgs* args, const ClusterLayout* lays, const int32_t* order, int count,
                                     int C, int nclusters, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * nclusters);
  cfg.blockDim = dim3(kClusterTPB);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, pcg_cluster_batch_kernel, args, lays, order, count);
}

}  // namespace avip
