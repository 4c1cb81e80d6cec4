// BiCGStab for the non-symmetric Poisson system of the axisymmetric configuration (the radius
// in the dual-contour integrals breaks the symmetry of K, so conjugate gradients no longer
// apply), FP64, one cooperative persistent launch per solve.
//
// As for CG, the system is scaled on both sides by the diagonal: A = D^-1/2 K D^-1/2,
// x = D^1/2 phi, b' = D^-1/2 b (Jacobi preconditioning split between the two sides), and the
// stopping test is ||b' - A x||_2 <= rtol ||b'||_2 on the scaled residual of the free rows
// (Dirichlet rows are unit rows that hold their value from the start; counting their values
// in ||b'|| would loosen the test by the ratio of the boundary potentials to the free-row
// right-hand side, a factor of about 24 on the axisymmetric streamer gap).
//
// Van der Vorst's BiCGStab with both matrix products taken exactly (a variant that carries
// A p and A s by recurrences and needs only two synchronisations per iteration was tried: on
// the axisymmetric matrices its recurrence drift, |v - A p| / |v|, reached 1e-3 within a few
// hundred iterations and the residual stagnated near 1e-12).  Per iteration, four phases
// separated by grid-wide reductions, which double as the barriers that complete a vector
// before other rows gather it:
//
//   P1   v = A p (gather p);                 sum rh.v           -> alpha = rho / rh.v
//   P2   s = r - alpha v;                    sum s.s            (barrier: s complete)
//   P3   t = A s (gather s);                 sums t.s, t.t, rh.s, rh.t
//                                            -> omega = t.s / t.t, rho' = rh.s - omega rh.t,
//                                               beta = (rho' / rho)(alpha / omega)
//   P4   x += alpha p + omega s;  r = s - omega t;  p = r + beta (p - omega v);  sum r.r
//
// rh is the shadow residual (the residual at the last (re)start).  Convergence is tested on
// the recursive residual (or on s, which ends the iteration half way with x += alpha p) and
// confirmed on the true residual b' - A x; a breakdown (rh.v = 0, omega = 0 or rho' = 0) or a
// true residual still too large restarts from the true residual (bounded number of restarts).
#include <cuda_runtime.h>

#include <algorithm>

#include "avip_internal.h"
#include "grid_sync.cuh"
#include "sell.cuh"

namespace avip {

namespace {
constexpr int kBcgMaxRestarts = 8;
constexpr int kBcgTPB = 768;
}  // namespace

__global__ void __launch_bounds__(kBcgTPB, 1) bicgstab_fp64_kernel(PcgArgs a) {
  if (solve_skipped(a.sc)) return;  // an earlier stage of this run failed beyond repair
  __shared__ double smem[2 * 32 * 4];
  const int lane = threadIdx.x & 31;
  constexpr int wpb = kBcgTPB / 32;
  const int gwarp = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  const int N = a.A.N, nsl = a.A.nslices;
  const size_t Np = (size_t)a.Npad;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * Np;
  double* __restrict__ x = a.x;
  double* __restrict__ r = a.r;
  double* __restrict__ p = a.p;
  double* __restrict__ v = a.q_ap;
  double* __restrict__ sv = a.bcg;
  double* __restrict__ tv = a.bcg + Np;
  double* __restrict__ rh = a.bcg + 2 * Np;
  FlagSync fs{a.flags, a.parts, a.sync, 0u, a.spin_ns, (int)gridDim.x, (int)blockIdx.x};

  // ---- x = D^1/2 phi (warm start) and b'
  const double gain = dirichlet_gain(a);
  const int hist = history_length(a);
  double bb[1] = {0.0};
  for (int sl = gwarp; sl < nsl; sl += nwarps) {
    const int i = sl * kSlice + lane;
    if (i >= N) continue;
    x[i] = a.dsq[i] * predict_phi(a, i, hist);
    double b;
    if (a.use_density_rhs) {
      double rho = 0.0;
      if (a.rhs_src)
        rho = a.rhs_src[i];
      else
        for (int k = 0; k < a.ns; ++k) rho = fma(a.q[k], nb[(size_t)k * Np + i], rho);
      b = fma(a.rhs_scale[i], rho, gain * a.lift[i]);
      a.b[i] = b;
    } else {
      b = a.b[i];
    }
    if (a.rhs_scale[i] != 0.0) bb[0] = fma(b, b, bb[0]);  // free rows only: a Dirichlet row holds its value exactly
    else x[i] = b;  // a Dirichlet unit row takes its (possibly ramped) value exactly
  }
  if (!grid_allsum<1>(bb, fs, smem)) goto timeout;
  {
    const double thresh = a.rtol * a.rtol * bb[0];
    double rr_true = 0.0, rho = 0.0, alpha = 0.0;
    bool restart = true;
    int it = 0, restarts = 0, status = AVIP_OK;
    if (bb[0] == 0.0) {
      for (int sl = gwarp; sl < nsl; sl += nwarps) {
        const int i = sl * kSlice + lane;
        if (i < N) x[i] = a.b[i];  // free b == 0: x = b
      }
    } else {
      while (true) {
        if (restart) {
          // ---- true residual r = b' - A x (x complete: the last reduction is the barrier);
          //      rh = p = r
          double r2[1] = {0.0};
          for (int sl = gwarp; sl < nsl; sl += nwarps) {
            const int i = sl * kSlice + lane;
            if (i >= N) continue;
            const double ri = a.b[i] - sell_row_dot(a.A, sl, lane, i, x);
            r[i] = ri;
            rh[i] = ri;
            p[i] = ri;
            r2[0] = fma(ri, ri, r2[0]);
          }
          if (!grid_allsum<1>(r2, fs, smem)) goto timeout;
          rr_true = r2[0];
          if (rr_true <= thresh) break;
          if (!isfinite(rr_true)) {  // non-finite data: stop at once
            status = AVIP_ENAN;
            break;
          }
          if (it >= a.max_iter || (it > 0 && restarts >= kBcgMaxRestarts)) {
            status = AVIP_ENOTCONV;
            break;
          }
          if (it > 0) ++restarts;
          rho = rr_true;  // rh.r with rh = r
          restart = false;
        }
        // ---- P1: v = A p (p complete)
        double rv[1] = {0.0};
        for (int sl = gwarp; sl < nsl; sl += nwarps) {
          const int i = sl * kSlice + lane;
          if (i >= N) continue;
          const double w = sell_row_dot(a.A, sl, lane, i, p);
          v[i] = w;
          rv[0] = fma(rh[i], w, rv[0]);
        }
        double al[1];
        const double rho_now = rho;
        if (!grid_allsum<1, 1>(rv, al, fs, smem, [rho_now](const double* t, double* e) {
              e[0] = t[0] != 0.0 ? rho_now / t[0] : 0.0;
            }))
          goto timeout;
        if (rv[0] == 0.0) {  // breakdown: rh orthogonal to A p
          if (it == 0) {     // at the first (re)start nothing would change
            status = AVIP_ENOTCONV;
            break;
          }
          restart = true;    // the restart block bounds the number of restarts
          continue;
        }
        const double alpha = al[0];
        // ---- P2: s = r - alpha v (own rows)
        double ss[1] = {0.0};
        for (int sl = gwarp; sl < nsl; sl += nwarps) {
          const int i = sl * kSlice + lane;
          if (i >= N) continue;
          const double si = fma(-alpha, v[i], r[i]);
          sv[i] = si;
          ss[0] = fma(si, si, ss[0]);
        }
        if (!grid_allsum<1>(ss, fs, smem)) goto timeout;
        if (ss[0] <= thresh) {
          // s small enough: x += alpha p and confirm on the true residual
          for (int sl = gwarp; sl < nsl; sl += nwarps) {
            const int i = sl * kSlice + lane;
            if (i < N) x[i] = fma(alpha, p[i], x[i]);
          }
          ++it;
          restart = true;
          double dummy[1] = {0.0};
          if (!grid_allsum<1>(dummy, fs, smem)) goto timeout;  // x complete before it is gathered
          continue;
        }
        // ---- P3: t = A s (s complete)
        double d4[4] = {0.0, 0.0, 0.0, 0.0};  // t.s, t.t, rh.s, rh.t
        for (int sl = gwarp; sl < nsl; sl += nwarps) {
          const int i = sl * kSlice + lane;
          if (i >= N) continue;
          const double ti = sell_row_dot(a.A, sl, lane, i, sv);
          const double si = sv[i], rhi = rh[i];
          tv[i] = ti;
          d4[0] = fma(ti, si, d4[0]);
          d4[1] = fma(ti, ti, d4[1]);
          d4[2] = fma(rhi, si, d4[2]);
          d4[3] = fma(rhi, ti, d4[3]);
        }
        double e3[3];  // omega, rho', beta (0 after a breakdown)
        if (!grid_allsum<4, 3>(d4, e3, fs, smem, [rho_now, alpha](const double* t, double* e) {
              const double om = t[1] > 0.0 ? t[0] / t[1] : 0.0;
              const double rn = t[2] - om * t[3];
              e[0] = om;
              e[1] = rn;
              e[2] = (om != 0.0 && rn != 0.0) ? (rn / rho_now) * (alpha / om) : 0.0;
            }))
          goto timeout;
        const double omega = e3[0], rho_new = e3[1], beta = e3[2];
        // ---- P4: x, r, p (own rows; p was last gathered in P1, s in P3)
        double rn2[1] = {0.0};
        for (int sl = gwarp; sl < nsl; sl += nwarps) {
          const int i = sl * kSlice + lane;
          if (i >= N) continue;
          const double si = sv[i], ti = tv[i], pi = p[i];
          x[i] = fma(omega, si, fma(alpha, pi, x[i]));
          const double ri = fma(-omega, ti, si);
          r[i] = ri;
          p[i] = fma(beta, fma(-omega, v[i], pi), ri);
          rn2[0] = fma(ri, ri, rn2[0]);
        }
        if (!grid_allsum<1>(rn2, fs, smem)) goto timeout;
        ++it;
        rho = rho_new;
        if (rn2[0] <= thresh || !isfinite(rn2[0]) || omega == 0.0 || rho_new == 0.0 || it >= a.max_iter)
          restart = true;
      }
    }
    // ---- phi = D^-1/2 x
    for (int sl = gwarp; sl < nsl; sl += nwarps) {
      const int i = sl * kSlice + lane;
      if (i < N) a.phi[i] = a.dsqinv[i] * x[i];
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

// Grid: co-resident blocks, no more than there are slices to share.
PcgPlan bicgstab_plan(int nslices, int requested_tpb) {
  (void)requested_tpb;
  PcgPlan pl;
  pl.kind = 7;
  pl.tpb = kBcgTPB;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bicgstab_fp64_kernel, kBcgTPB, 0);
  const int wpb = kBcgTPB / kSlice;
  const int want = (nslices + wpb - 1) / wpb;
  pl.blocks = std::max(1, std::min(std::max(occ, 1) * std::max(sms, 1), want));
  return pl;
}

cudaError_t launch_bicgstab(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st) {
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
  return cudaLaunchKernelEx(&cfg, bicgstab_fp64_kernel, args);
}

}  // namespace avip
