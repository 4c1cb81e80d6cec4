// Jacobi-preconditioned conjugate gradients for K phi = b (the Poisson system of Eq.
// poisson_discretization_cartesian with Dirichlet unknowns eliminated), FP64.
//
// Jacobi preconditioning is applied symmetrically: CG runs on A = D^-1/2 K D^-1/2 with
// x = D^1/2 phi and b' = D^-1/2 b.  Its iterates are exactly those of Jacobi-PCG on K, but the
// preconditioned residual is the residual itself, so one vector, one multiply and one dot
// product per row and iteration disappear; on GB300, where the FP64 pipe issues one warp-wide
// FMA per ~16 cycles per SM, that is a direct saving.  The stopping test is on the scaled
// residual of the free rows: ||b' - A x||_2 <= rtol ||b'||_2, both norms over the rows that
// are not Dirichlet rows (those are unit rows whose residual is zero from the start).
//
// One cooperative, persistent launch runs the whole solve: assembly of b' from the densities,
// the initial residual, every iteration, the final true-residual check and phi = D^-1/2 x.
// Each warp owns SELL-32 slices (32 consecutive Morton-ordered rows), so every matrix load is
// coalesced and the gathered neighbour values are mostly cache hits.
//
// Iteration (two grid reductions, see grid_sync.cuh):
//   phase A   w = A r (gather r),  q <- w + beta q,  p <- r + beta p,  sum p.q
//             -> alpha = r.r / p.q, derived once per block
//   phase B   x += alpha p;  r -= alpha q;  sum r.r
//             -> beta = r.r' / r.r and the stop test, once per block
// q = A p is carried by the recurrence A(r + beta p) = A r + beta A p, so only r is gathered
// and p, q are updated in place by the thread that owns the row.  Convergence is tested on
// the recursive residual and confirmed on the true residual; if the true residual is still
// too large the iteration restarts from it (bounded number of restarts).
#include <cuda_runtime.h>

#include <algorithm>

#include "avip_internal.h"
#include "grid_sync.cuh"
#include "sell.cuh"

namespace avip {

constexpr int kMaxRestarts = 8;
constexpr int kResTPB = 512;  // block size of the register-resident kernels (one block per SM)

template <int TPB>
__global__ void __launch_bounds__(TPB, (TPB <= 512 ? 1024 / TPB : 1)) pcg_fp64_kernel(PcgArgs a) {
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
  // x must be complete before the residual gathers it: this reduction is also the barrier
  if (!grid_allsum<1>(bb, fs, smem)) goto timeout;
  {
    const double thresh = a.rtol * a.rtol * bb[0];
    double rr = 0.0, beta = 0.0, rr_true = 0.0;
    bool check = true;  // the first pass computes the initial (true) residual
    int it = 0, restarts = 0, status = AVIP_OK;
    if (bb[0] == 0.0) {
      // free b == 0: the solution is x = b (0 on free rows, the value on Dirichlet rows)
      for (int s = gwarp; s < nsl; s += nwarps) {
        const int i = s * kSlice + lane;
        if (i < N) a.x[i] = a.b[i];
      }
    } else {
      while (true) {
        if (check || it >= a.max_iter) {
          // ---- true residual r = b' - A x; (re)start from it
          double r2[1] = {0.0};
          for (int s = gwarp; s < nsl; s += nwarps) {
            const int i = s * kSlice + lane;
            if (i >= N) continue;
            const double r = a.b[i] - sell_row_dot(a.A, s, lane, i, a.x);
            a.r[i] = r;
            a.p[i] = 0.0;
            a.q_ap[i] = 0.0;
            r2[0] = fma(r, r, r2[0]);
          }
          if (!grid_allsum<1>(r2, fs, smem)) goto timeout;
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
          rr = rr_true;
          beta = 0.0;
          check = false;
        }
        // ---- phase A (r was completed before the last reduction, which is the barrier)
        double pq[1] = {0.0};
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          const double w = sell_row_dot(a.A, s, lane, i, a.r);
          const double qn = fma(beta, a.q_ap[i], w);
          const double pn = fma(beta, a.p[i], a.r[i]);
          a.q_ap[i] = qn;
          a.p[i] = pn;
          pq[0] = fma(pn, qn, pq[0]);
        }
        const double rr_now = rr;
        if (!grid_allsum<1, 1>(pq, one, fs, smem, [rr_now](const double* t, double* e) { e[0] = rr_now / t[0]; }))
          goto timeout;
        const double alpha = one[0];
        // ---- phase B (every gather of r in phase A finished before the reduction above)
        double rn[1] = {0.0};
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          a.x[i] = fma(alpha, a.p[i], a.x[i]);
          const double r = fma(-alpha, a.q_ap[i], a.r[i]);
          a.r[i] = r;
          rn[0] = fma(r, r, rn[0]);
        }
        double bs[2];
        if (!grid_allsum<1, 2>(rn, bs, fs, smem, [rr_now, thresh](const double* t, double* e) {
              e[0] = t[0] / rr_now;
              e[1] = (t[0] <= thresh || !isfinite(t[0])) ? 1.0 : 0.0;
            }))
          goto timeout;
        beta = bs[0];
        check = bs[1] != 0.0;
        rr = rn[0];
        ++it;
      }
    }
    // ---- phi = D^-1/2 x
    for (int s = gwarp; s < nsl; s += nwarps) {
      const int i = s * kSlice + lane;
      if (i < N) a.phi[i] = a.dsqinv[i] * a.x[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.res->pcg_iters = it;
      advance_history(a);
      a.res->pcg_status = status;
      a.res->pcg_relres = bb[0] > 0.0 ? sqrt(rr_true / bb[0]) : 0.0;
      a.res->pcg_bnorm = sqrt(bb[0]);
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

// ------------------------------------------------------------------------------------------
// Register-resident variant: each warp owns MAXS consecutive slices for the whole solve and
// keeps, for each of its rows, the CG vectors p, q (= A p) and x in registers and the slice
// metadata (element base, slice width, row length) too.  Only r lives in memory (neighbours
// gather it).  Per row and iteration the memory traffic drops to the matrix row, the r
// gathers and one r read-modify-write; the FP64 work is 13 operations.  The launch uses one
// block per SM at most; it needs gridDim.x * warps * MAXS >= slices.
template <int TPB, int MAXS>
__global__ void __launch_bounds__(TPB, 1) pcg_fp64_res_kernel(PcgArgs a) {
  if (solve_skipped(a.sc)) return;  // an earlier stage of this run failed beyond repair
  __shared__ double smem[2 * 32 * 4];
  const int lane = threadIdx.x & 31;
  constexpr int wpb = TPB / 32;
  const int gwarp = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int N = a.A.N, nsl = a.A.nslices;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
  FlagSync fs{a.flags, a.parts, a.sync, 0u, a.spin_ns, (int)gridDim.x, (int)blockIdx.x};
  double one[1];

  int base[MAXS], wid[MAXS], rl[MAXS];
  double p[MAXS], q[MAXS], x[MAXS];
#pragma unroll
  for (int j = 0; j < MAXS; ++j) {
    const int s = gwarp * MAXS + j;
    const int i = s * kSlice + lane;
    wid[j] = 0;
    rl[j] = 0;
    base[j] = 0;
    p[j] = q[j] = x[j] = 0.0;
    if (s < nsl) {
      base[j] = __ldg(a.A.sl_ptr + s) + lane;
      wid[j] = __ldg(a.A.sl_w + s);
      rl[j] = i < N ? __ldg(a.A.rlen + i) : 0;
    }
  }
  // one row of A v with the cached metadata; returns the diagonal gather in vd
  auto row_dot = [&](int j, const double* __restrict__ v, int i, double& vd) -> double {
    constexpr int U = 8;
    double acc = 0.0;
    vd = 0.0;
    for (int k0 = 0; k0 < wid[j]; k0 += U) {
      int c[U];
      double av[U], xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + u;
        c[u] = i;
        av[u] = 0.0;
        if (k < rl[j]) {
          c[u] = __ldg(a.A.col + base[j] + k * kSlice);
          av[u] = __ldg(a.A.aval + base[j] + k * kSlice);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) xv[u] = (k0 + u < rl[j]) ? v[c[u]] : 0.0;
      if (k0 == 0) vd = xv[0];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k0 + u < rl[j]) acc = fma(av[u], xv[u], acc);
    }
    return acc;
  };

  // ---- x = D^1/2 phi (warm start) and b'
  const double gain = dirichlet_gain(a);
  const int hist = history_length(a);
  double bb[1] = {0.0};
#pragma unroll
  for (int j = 0; j < MAXS; ++j) {
    const int i = (gwarp * MAXS + j) * kSlice + lane;
    if (rl[j] == 0) continue;
    x[j] = a.dsq[i] * predict_phi(a, i, hist);
    a.x[i] = x[j];
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
    else {  // a Dirichlet unit row takes its (possibly ramped) value exactly
      x[j] = b;
      a.x[i] = b;
    }
  }
  if (!grid_allsum<1>(bb, fs, smem)) goto timeout;
  {
    const double thresh = a.rtol * a.rtol * bb[0];
    double rr = 0.0, beta = 0.0, rr_true = 0.0;
    bool check = true;
    int it = 0, restarts = 0, status = AVIP_OK;
    if (bb[0] == 0.0) {
#pragma unroll
      for (int j = 0; j < MAXS; ++j)
        if (rl[j] != 0) x[j] = a.b[(gwarp * MAXS + j) * kSlice + lane];  // free b == 0: x = b
    } else {
      while (true) {
        if (check || it >= a.max_iter) {
          // ---- true residual r = b' - A x (x was stored before the last reduction)
          double r2[1] = {0.0};
#pragma unroll
          for (int j = 0; j < MAXS; ++j) {
            const int i = (gwarp * MAXS + j) * kSlice + lane;
            if (rl[j] == 0) continue;
            double xd;
            const double r = a.b[i] - row_dot(j, a.x, i, xd);
            a.r[i] = r;
            p[j] = 0.0;
            q[j] = 0.0;
            r2[0] = fma(r, r, r2[0]);
          }
          if (!grid_allsum<1>(r2, fs, smem)) goto timeout;
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
          rr = rr_true;
          beta = 0.0;
          check = false;
        }
        // ---- phase A
        double pq[1] = {0.0};
#pragma unroll
        for (int j = 0; j < MAXS; ++j) {
          const int i = (gwarp * MAXS + j) * kSlice + lane;
          if (rl[j] == 0) continue;
          double ri;
          const double w = row_dot(j, a.r, i, ri);
          q[j] = fma(beta, q[j], w);
          p[j] = fma(beta, p[j], ri);
          pq[0] = fma(p[j], q[j], pq[0]);
        }
        const double rr_now = rr;
        if (!grid_allsum<1, 1>(pq, one, fs, smem, [rr_now](const double* t, double* e) { e[0] = rr_now / t[0]; }))
          goto timeout;
        const double alpha = one[0];
        // ---- phase B: all loads of r issued before the first store (no aliasing stall)
        double rn[1] = {0.0};
        double rv[MAXS];
#pragma unroll
        for (int j = 0; j < MAXS; ++j) {
          const int i = (gwarp * MAXS + j) * kSlice + lane;
          rv[j] = rl[j] != 0 ? __ldcg(a.r + i) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < MAXS; ++j) {
          const int i = (gwarp * MAXS + j) * kSlice + lane;
          if (rl[j] == 0) continue;
          x[j] = fma(alpha, p[j], x[j]);
          const double r = fma(-alpha, q[j], rv[j]);
          a.r[i] = r;
          rn[0] = fma(r, r, rn[0]);
        }
        double bs[2];
        if (!grid_allsum<1, 2>(rn, bs, fs, smem, [rr_now, thresh](const double* t, double* e) {
              e[0] = t[0] / rr_now;
              e[1] = (t[0] <= thresh || !isfinite(t[0])) ? 1.0 : 0.0;
            }))
          goto timeout;
        beta = bs[0];
        check = bs[1] != 0.0;
        rr = rn[0];
        ++it;
        if (check || it >= a.max_iter) {
          // the true residual gathers x: publish it (the next reduction orders it)
#pragma unroll
          for (int j = 0; j < MAXS; ++j) {
            const int i = (gwarp * MAXS + j) * kSlice + lane;
            if (rl[j] != 0) a.x[i] = x[j];
          }
          double z0[1] = {0.0};
          if (!grid_allsum<1>(z0, fs, smem)) goto timeout;
        }
      }
    }
    // ---- phi = D^-1/2 x
#pragma unroll
    for (int j = 0; j < MAXS; ++j) {
      const int i = (gwarp * MAXS + j) * kSlice + lane;
      if (rl[j] != 0) a.phi[i] = a.dsqinv[i] * x[j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.res->pcg_iters = it;
      advance_history(a);
      a.res->pcg_status = status;
      a.res->pcg_relres = bb[0] > 0.0 ? sqrt(rr_true / bb[0]) : 0.0;
      a.res->pcg_bnorm = sqrt(bb[0]);
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

// Block sizes of the streaming kernel; index 0 is the default.
static const int kPcgSizes[] = {768, 256, 512, 1024};

static const void* pcg_kernel_ptr(int tpb) {
  switch (tpb) {
    case 256: return (const void*)pcg_fp64_kernel<256>;
    case 512: return (const void*)pcg_fp64_kernel<512>;
    case 1024: return (const void*)pcg_fp64_kernel<1024>;
    default: return (const void*)pcg_fp64_kernel<768>;
  }
}

static const void* pcg_res_kernel_ptr(int maxs) {
  switch (maxs) {
    case 1: return (const void*)pcg_fp64_res_kernel<kResTPB, 1>;
    case 2: return (const void*)pcg_fp64_res_kernel<kResTPB, 2>;
    case 4: return (const void*)pcg_fp64_res_kernel<kResTPB, 4>;
    default: return (const void*)pcg_fp64_res_kernel<kResTPB, 8>;
  }
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

static int occupancy(const void* k, int tpb) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, tpb, 0);
  return occ;
}

// Choose the kernel and grid.  kind: 0 = automatic (register-resident when the mesh fits in
// one block per SM, else streaming), 1 = streaming, 2 = register-resident.
PcgPlan pcg_plan(int nslices, int kind, int requested_tpb) {
  PcgPlan pl;
  const int sms = sm_count();
  if (kind == 0 || kind == 2) {
    constexpr int wpb = kResTPB / kSlice;
    for (int maxs : {1, 2, 4, 8}) {
      const int blocks = (nslices + wpb * maxs - 1) / (wpb * maxs);
      const int occ = occupancy(pcg_res_kernel_ptr(maxs), kResTPB);
      if (occ > 0 && blocks <= sms * occ) {
        pl.kind = 2;
        pl.tpb = kResTPB;
        pl.maxs = maxs;
        pl.blocks = blocks;
        return pl;
      }
    }
  }
  pl.kind = 1;
  pl.tpb = requested_tpb;
  bool known = false;
  for (int s : kPcgSizes) known |= (s == requested_tpb);
  if (!known) pl.tpb = kPcgSizes[0];
  pl.maxs = 0;
  const int wpb = pl.tpb / kSlice;
  const int want = (nslices + wpb - 1) / wpb;
  pl.blocks = std::max(1, std::min(occupancy(pcg_kernel_ptr(pl.tpb), pl.tpb) * sms, want));
  return pl;
}

// Launch helper (host).  The plan's grid never exceeds the co-resident limit of its kernel.
cudaError_t launch_pcg_fp64(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pl.blocks);
  cfg.blockDim = dim3(pl.tpb);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* kargs[] = {const_cast<PcgArgs*>(&args)};
  const void* k = pl.kind == 2 ? pcg_res_kernel_ptr(pl.maxs) : pcg_kernel_ptr(pl.tpb);
  return cudaLaunchKernelExC(&cfg, k, kargs);
}

}  // namespace avip
