// Jacobi-preconditioned conjugate gradients for K phi = b (the Poisson system of Eq.
// poisson_discretization_cartesian with Dirichlet unknowns eliminated), FP64.
//
// One cooperative, persistent launch runs the whole solve: assembly of b from the densities,
// the initial residual, every iteration and the final true-residual check.  Each warp owns
// SELL-32 slices (32 consecutive Morton-ordered rows), so every matrix load is coalesced and
// the gathered neighbour values are mostly cache hits.
//
// Iteration (two grid reductions):
//   phase A   w = K z (gather z),  q <- w + beta q,  p <- z + beta p,  sum p.q
//   phase B   alpha = rz / pq;  phi += alpha p;  r -= alpha q;  z = D^-1 r;  sum r.z, r.r
// q = K p is carried by the recurrence K(z + beta p) = K z + beta K p, so only z is gathered
// and p, q are updated in place by the thread that owns the row.  Convergence is tested on
// the recursive residual and confirmed on the true residual b - K phi; if the true residual
// is still too large the iteration restarts from it (bounded number of restarts).
#include <cuda_runtime.h>

#include "avip_internal.h"
#include "grid_sync.cuh"

namespace avip {

constexpr int kPcgThreads = 256;
constexpr int kMaxRestarts = 8;

// One row of y = K v over the SELL-32 structure (diagonal first, then ascending columns).
__device__ __forceinline__ double sell_row_dot(const SellView& A, int slice, int lane, int row,
                                               const double* __restrict__ v) {
  const int base = __ldg(A.sl_ptr + slice) + lane;
  const int w = __ldg(A.sl_w + slice);
  const int rl = __ldg(A.rlen + row);
  double acc = 0.0;
  for (int k = 0; k < w; ++k) {
    if (k < rl) {
      const int e = base + k * kSlice;
      acc = fma(__ldg(A.aval + e), __ldcg(v + __ldg(A.col + e)), acc);
    }
  }
  return acc;
}

__global__ void __launch_bounds__(kPcgThreads) pcg_fp64_kernel(PcgArgs a) {
  __shared__ double smem[32 * 4 + 4];
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int gwarp = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  const int N = a.A.N, nsl = a.A.nslices;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;

  // ---- b, r = b - K phi, z = D^-1 r, p = q = 0
  double red3[3] = {0.0, 0.0, 0.0};  // r.z, r.r, b.b
  for (int s = gwarp; s < nsl; s += nwarps) {
    const int i = s * kSlice + lane;
    if (i >= N) continue;
    double b;
    if (a.use_density_rhs) {
      double rho = 0.0;
      for (int k = 0; k < a.ns; ++k) rho = fma(a.q[k], nb[(size_t)k * a.Npad + i], rho);
      b = fma(a.rhs_scale[i], rho, a.lift[i]);
      a.b[i] = b;
    } else {
      b = a.b[i];
    }
    const double r = b - sell_row_dot(a.A, s, lane, i, a.x);
    const double z = a.dinv[i] * r;
    a.r[i] = r;
    a.z[i] = z;
    a.p[i] = 0.0;
    a.q_ap[i] = 0.0;
    red3[0] = fma(r, z, red3[0]);
    red3[1] = fma(r, r, red3[1]);
    red3[2] = fma(b, b, red3[2]);
  }
  if (!grid_sum<3>(red3, a.partials, a.sync, smem)) goto timeout;
  {
    double rz = red3[0], rr = red3[1];
    const double bb = red3[2];
    const double thresh = a.rtol * a.rtol * bb;
    double beta = 0.0;
    int it = 0, restarts = 0, status = AVIP_OK;
    double rr_true = rr;
    if (bb == 0.0) {
      // b == 0: the solution is phi = 0
      for (int s = gwarp; s < nsl; s += nwarps) {
        const int i = s * kSlice + lane;
        if (i < N) a.x[i] = 0.0;
      }
      rr_true = 0.0;
    } else {
      while (true) {
        if (rr <= thresh || it >= a.max_iter) {
          // ---- true residual; restart from it when the recursion drifted
          double red2[2] = {0.0, 0.0};
          for (int s = gwarp; s < nsl; s += nwarps) {
            const int i = s * kSlice + lane;
            if (i >= N) continue;
            const double r = a.b[i] - sell_row_dot(a.A, s, lane, i, a.x);
            const double z = a.dinv[i] * r;
            a.r[i] = r;
            a.z[i] = z;
            a.p[i] = 0.0;
            a.q_ap[i] = 0.0;
            red2[0] = fma(r, z, red2[0]);
            red2[1] = fma(r, r, red2[1]);
          }
          if (!grid_sum<2>(red2, a.partials, a.sync, smem)) goto timeout;
          rr_true = red2[1];
          if (rr_true <= thresh) break;
          if (it >= a.max_iter || restarts >= kMaxRestarts) {
            status = AVIP_ENOTCONV;
            break;
          }
          ++restarts;
          rz = red2[0];
          rr = red2[1];
          beta = 0.0;
        }
        // ---- phase A
        double pq[1] = {0.0};
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          const double w = sell_row_dot(a.A, s, lane, i, a.z);
          const double qn = fma(beta, a.q_ap[i], w);
          const double pn = fma(beta, a.p[i], a.z[i]);
          a.q_ap[i] = qn;
          a.p[i] = pn;
          pq[0] = fma(pn, qn, pq[0]);
        }
        if (!grid_sum<1>(pq, a.partials, a.sync, smem)) goto timeout;
        const double alpha = rz / pq[0];
        // ---- phase B
        double rzrr[2] = {0.0, 0.0};
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          a.x[i] = fma(alpha, a.p[i], a.x[i]);
          const double r = fma(-alpha, a.q_ap[i], a.r[i]);
          const double z = a.dinv[i] * r;
          a.r[i] = r;
          a.z[i] = z;
          rzrr[0] = fma(r, z, rzrr[0]);
          rzrr[1] = fma(r, r, rzrr[1]);
        }
        if (!grid_sum<2>(rzrr, a.partials, a.sync, smem)) goto timeout;
        beta = rzrr[0] / rz;
        rz = rzrr[0];
        rr = rzrr[1];
        ++it;
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.sc->pcg_iters = it;
      a.sc->pcg_status = status;
      a.sc->pcg_relres = bb > 0.0 ? sqrt(rr_true / bb) : 0.0;
      a.sc->pcg_bnorm = sqrt(bb);
      if (status != AVIP_OK && a.sc->status == AVIP_OK) a.sc->status = status;
    }
    return;
  }
timeout:
  if (threadIdx.x == 0) {
    atomicExch(&a.sync->abort, 1);
    a.sc->pcg_status = AVIP_ETIMEOUT;
    atomicCAS(&a.sc->status, AVIP_OK, AVIP_ETIMEOUT);
  }
}

// Launch helper (host).  `blocks` must not exceed the co-resident limit of the kernel.
cudaError_t launch_pcg_fp64(const PcgArgs& args, int blocks, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, pcg_fp64_kernel, args);
}

int pcg_fp64_max_blocks() {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_fp64_kernel, kPcgThreads, 0);
  return occ * sms;
}

int pcg_threads() { return kPcgThreads; }

}  // namespace avip
