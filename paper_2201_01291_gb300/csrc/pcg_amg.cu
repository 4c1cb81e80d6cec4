// Conjugate gradients preconditioned by one smoothed-aggregation AMG V-cycle (solver kind 8),
// BiCGStab preconditioned by it (kind 9, the non-symmetric axisymmetric matrix) and the
// mixed-precision form (kind 10): one cooperative persistent launch per solve.
//
// The system is the symmetrically scaled one of the Jacobi variant, A = D^-1/2 K D^-1/2,
// x = D^1/2 phi, b' = D^-1/2 b, with the same stopping test (true residual of the free rows,
// ||b' - A x|| <= rtol ||b'||).  The hierarchy (composite level operators, dense inverse of the
// coarsest matrix) is built once per mesh on the host (amg_setup.cpp); the preconditioner
// z = M r is one V-cycle of two grid-wide phases per level (amg_vcycle.cuh):
//
//   down, level l:  xp = Q b  (damped Jacobi pre-smoothing from zero, Q = omega D^-1),
//                   b' = Rf b = R (b - A xp)
//   coarsest:       x = A_c^-1 b  (dense product)
//   up, level l:    x = U xp + Pf x' = xp + P x' + Q (b - A (xp + P x'))  (post-smoothing)
//
// with omega = 1.7 / lambda_max(D^-1 A) (lambda_max from power iteration).  The pre- and
// post-smoother are the same step and R = P^T, so the V-cycle is a symmetric positive definite
// operator and plain CG applies.  Its values are FP32 by default
// (T = float) or FP64; the Krylov vectors, the products with A and the stopping test are FP64.
//
// Every phase gathers only vectors that other blocks completed in an earlier phase, so each
// ends with a grid-wide barrier (a reduction where CG needs a dot product).  Per CG iteration:
// 2 barriers per non-coarsest level, 1 for the coarsest, 1 for w = A z; the residual update of
// the iteration is folded into the finest down phase of the next (amg_cg_solve).
#include <cuda_runtime.h>

#include <algorithm>

#include "avip_internal.h"
#include "grid_sync.cuh"
#include "sell.cuh"
#include "amg_vcycle.cuh"

namespace avip {

namespace {
// Block sizes (one block per SM).  Default: 1024 threads for CG with the FP32 hierarchy (kind
// 8: 99.9 us per CG iteration on the pin-plane solve against 104.8 at 768), 768 otherwise
// (BiCGStab and the mixed form are 1 % faster at 768; the FP64 hierarchy spills at 1024)
constexpr int kAmgSizes[] = {768, 512, 1024};
int amg_default_threads(int kind, int fp64) { return kind == 8 && !fp64 ? 1024 : 768; }
constexpr int kAmgMaxRestarts = 8;

}  // namespace

// The hierarchy and the preconditioned residual of value type T.
template <typename T>
__device__ __forceinline__ const AmgDevT<T>* amg_of(const PcgArgs& a);
template <>
__device__ __forceinline__ const AmgDevT<float>* amg_of<float>(const PcgArgs& a) { return a.amg32; }
template <>
__device__ __forceinline__ const AmgDevT<double>* amg_of<double>(const PcgArgs& a) { return a.amg; }
// A wait was abandoned: make every other waiter of this solve leave, report the timeout.
__device__ __forceinline__ void report_timeout(const PcgArgs& a) {
  atomicExch(&a.sync->abort, 1);
  a.res->pcg_status = AVIP_ETIMEOUT;
  atomicCAS(&a.sc->status, AVIP_OK, AVIP_ETIMEOUT);
}

template <int TPB, typename T>
__global__ void __launch_bounds__(TPB, 1) pcg_amg_kernel(PcgArgs a) {
  if (solve_skipped(a.sc)) return;  // an earlier stage of this run failed beyond repair
  __shared__ double smem[2 * 32 * 4];
  constexpr int wpb = TPB / 32;
  FlagSync fs{a.flags, a.parts, a.sync, 0u, a.spin_ns, (int)gridDim.x, (int)blockIdx.x};
  GridOps ops{fs, smem};
  if (!amg_cg_solve<T>(a, amg_of<T>(a), a.z, ops, blockIdx.x * wpb + (threadIdx.x >> 5), gridDim.x * wpb,
                       threadIdx.x & 31, blockIdx.x == 0 && threadIdx.x == 0) &&
      threadIdx.x == 0)
    report_timeout(a);
}

// BiCGStab right-preconditioned by the same V-cycle, for the non-symmetric axisymmetric
// matrix (solver kind 9): with p^ = M p and s^ = M s,
//   P1  v = A p^, rh.v -> alpha;  P2  s = r - alpha v (barrier);  P3  t = A s^, t.s, t.t, rh.s,
//   rh.t -> omega, rho', beta;  P4  x += alpha p^ + omega s^, r = s - omega t,
//   p = r + beta (p - omega v), r.r -> stop test
// (van der Vorst's iteration with M^-1 applied on the right, so x is updated directly and the
// stopping test stays on the true scaled residual of the free rows).  Two V-cycles per
// iteration; breakdowns and a true residual still too large restart from the true residual.
// The products with A stream the matrix by contiguous slice shares (spmv_stream, each row's own
// operands fetched ahead), the elementwise phases take slices round-robin.
// The solve of one system by the blocks taking part in `fs` (gwarp / nwarps number their warps,
// `leader` is the one thread that writes the statistics); false if a wait was abandoned.
template <typename T>
__device__ bool amg_bicgstab_solve(const PcgArgs& a, const AmgDevT<T>* __restrict__ H, FlagSync& fs, double* smem,
                                   int gwarp, int nwarps, int lane, bool leader) {
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
  double* __restrict__ ph = a.bcg + 3 * Np;
  double* __restrict__ sh = a.bcg + 4 * Np;
  GridOps ops{fs, smem};
  double dummy = 0.0;
  // the matrix as a streamed operator (products by contiguous slice shares, see spmv_stream)
  const SellMatT<double> A0{a.A.sl_ptr, a.A.sl_w, a.A.rlen, a.A.col, a.A.aval, N, nsl, 1};
  int ma, mb;
  warp_slices(nsl, gwarp, nwarps, ma, mb);
  struct Two {
    double u, w;
  };

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
  if (!grid_allsum<1>(bb, fs, smem)) return false;
  {
    const double thresh = a.rtol * a.rtol * bb[0];
    double rr_true = 0.0, rho = 0.0;
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
          // ---- true residual; rh = p = r; first V-cycle direction of p
          double r2[1] = {0.0};
          {
            const double* __restrict__ bv = a.b;
            const double* __restrict__ xv = x;
            spmv_stream<double, GridOps::kStream64>(
                A0, ma, mb, lane, [xv](int c) { return __ldca(xv + c); }, [bv](int i) { return bv[i]; },
                [&](int i, double ax, double bi) {
                  const double ri = bi - ax;
                  r[i] = ri;
                  rh[i] = ri;
                  p[i] = ri;
                  r2[0] = fma(ri, ri, r2[0]);
                });
          }
          if (!grid_allsum<1>(r2, fs, smem)) return false;
          rr_true = r2[0];
          if (rr_true <= thresh) break;
          if (!isfinite(rr_true)) {
            status = AVIP_ENAN;
            break;
          }
          if (it >= a.max_iter || (it > 0 && restarts >= kAmgMaxRestarts)) {
            status = AVIP_ENOTCONV;
            break;
          }
          if (it > 0) ++restarts;
          rho = rr_true;
          restart = false;
        }
        // ---- p^ = M p, then P1: v = A p^
        if (!vcycle(H, (const double*)p, ph, ops, gwarp, nwarps, lane, false, dummy)) return false;
        double rv[1] = {0.0};
        {
          const double* __restrict__ phv = ph;
          const double* __restrict__ rhv = rh;
          spmv_stream<double, GridOps::kStream64>(
              A0, ma, mb, lane, [phv](int c) { return __ldca(phv + c); }, [rhv](int i) { return rhv[i]; },
              [&](int i, double w, double rhi) {
                v[i] = w;
                rv[0] = fma(rhi, w, rv[0]);
              });
        }
        double al[1];
        const double rho_now = rho;
        if (!grid_allsum<1, 1>(rv, al, fs, smem, [rho_now](const double* t, double* e) {
              e[0] = t[0] != 0.0 ? rho_now / t[0] : 0.0;
            }))
          return false;
        if (rv[0] == 0.0 || !isfinite(rv[0])) {  // breakdown
          if (it == 0) {
            status = AVIP_ENOTCONV;
            break;
          }
          restart = true;
          continue;
        }
        const double alpha = al[0];
        // ---- P2: s = r - alpha v; first V-cycle direction of s
        double ss[1] = {0.0};
        for (int sl = gwarp; sl < nsl; sl += nwarps) {
          const int i = sl * kSlice + lane;
          if (i >= N) continue;
          const double si = fma(-alpha, v[i], r[i]);
          sv[i] = si;
          ss[0] = fma(si, si, ss[0]);
        }
        if (!grid_allsum<1>(ss, fs, smem)) return false;
        if (ss[0] <= thresh) {  // s small enough: x += alpha p^, confirm on the true residual
          for (int sl = gwarp; sl < nsl; sl += nwarps) {
            const int i = sl * kSlice + lane;
            if (i < N) x[i] = fma(alpha, __ldcg(ph + i), x[i]);
          }
          ++it;
          restart = true;
          double z0[1] = {0.0};
          if (!grid_allsum<1>(z0, fs, smem)) return false;
          continue;
        }
        // ---- s^ = M s, then P3: t = A s^
        if (!vcycle(H, (const double*)sv, sh, ops, gwarp, nwarps, lane, false, dummy)) return false;
        double d4[4] = {0.0, 0.0, 0.0, 0.0};  // t.s, t.t, rh.s, rh.t
        {
          const double* __restrict__ shv = sh;
          const double* __restrict__ svv = sv;
          const double* __restrict__ rhv = rh;
          spmv_stream<double, GridOps::kStream64>(
              A0, ma, mb, lane, [shv](int c) { return __ldca(shv + c); },
              [svv, rhv](int i) { return Two{svv[i], rhv[i]}; },
              [&](int i, double ti, const Two& o) {
                const double si = o.u, rhi = o.w;
                tv[i] = ti;
                d4[0] = fma(ti, si, d4[0]);
                d4[1] = fma(ti, ti, d4[1]);
                d4[2] = fma(rhi, si, d4[2]);
                d4[3] = fma(rhi, ti, d4[3]);
              });
        }
        double e3[3];
        if (!grid_allsum<4, 3>(d4, e3, fs, smem, [rho_now, alpha](const double* t, double* e) {
              const double om = t[1] > 0.0 ? t[0] / t[1] : 0.0;
              const double rn = t[2] - om * t[3];
              e[0] = om;
              e[1] = rn;
              e[2] = (om != 0.0 && rn != 0.0) ? (rn / rho_now) * (alpha / om) : 0.0;
            }))
          return false;
        const double omega = e3[0], rho_new = e3[1], beta = e3[2];
        // ---- P4: x, r, p; first V-cycle direction of the new p
        double rn2[1] = {0.0};
        for (int sl = gwarp; sl < nsl; sl += nwarps) {
          const int i = sl * kSlice + lane;
          if (i >= N) continue;
          const double si = sv[i], ti = tv[i], pi = p[i];
          x[i] = fma(omega, __ldcg(sh + i), fma(alpha, __ldcg(ph + i), x[i]));
          const double ri = fma(-omega, ti, si);
          r[i] = ri;
          const double pn = fma(beta, fma(-omega, v[i], pi), ri);
          p[i] = pn;
          rn2[0] = fma(ri, ri, rn2[0]);
        }
        if (!grid_allsum<1>(rn2, fs, smem)) return false;
        ++it;
        rho = rho_new;
        if (rn2[0] <= thresh || !isfinite(rn2[0]) || omega == 0.0 || rho_new == 0.0 || it >= a.max_iter)
          restart = true;
      }
    }
    for (int sl = gwarp; sl < nsl; sl += nwarps) {
      const int i = sl * kSlice + lane;
      if (i < N) a.phi[i] = a.dsqinv[i] * x[i];
    }
    if (leader) {
      a.res->pcg_iters = it;
      advance_history(a);
      a.res->pcg_status = status;
      a.res->pcg_relres = bb[0] > 0.0 ? sqrt(rr_true / bb[0]) : 0.0;
      a.res->pcg_bnorm = sqrt(bb[0]);
      if (status != AVIP_OK && a.sc->status == AVIP_OK) a.sc->status = status;
    }
  }
  return true;
}

template <int TPB, typename T>
__global__ void __launch_bounds__(TPB, 1) bicgstab_amg_kernel(PcgArgs a) {
  if (solve_skipped(a.sc)) return;  // an earlier stage of this run failed beyond repair
  __shared__ double smem[2 * 32 * 4];
  constexpr int wpb = TPB / 32;
  FlagSync fs{a.flags, a.parts, a.sync, 0u, a.spin_ns, (int)gridDim.x, (int)blockIdx.x};
  if (!amg_bicgstab_solve<T>(a, amg_of<T>(a), fs, smem, blockIdx.x * wpb + (threadIdx.x >> 5), gridDim.x * wpb,
                             threadIdx.x & 31, blockIdx.x == 0 && threadIdx.x == 0) &&
      threadIdx.x == 0)
    report_timeout(a);
}

// Several systems solved side by side in one cooperative launch (the photoionisation terms):
// the grid is split into contiguous groups of blocks, start[j] .. start[j+1] - 1 solving
// system j with its own arguments, hierarchy, vectors and barrier state, so the systems share
// no barrier and each group stops when its own system has converged.  The blocks of a group
// first agree on whether an earlier stage failed (a group that has finished may already have
// reported a failure when another group's block starts).
template <int TPB, typename T, bool kBicg>
__global__ void __launch_bounds__(TPB, 1) amg_group_kernel(const __grid_constant__ AmgGroupArgs g) {
  int j = 0;
  while (j + 1 < g.n && (int)blockIdx.x >= g.start[j + 1]) ++j;
  // the group's arguments, copied to shared memory (a runtime index into the parameters would
  // keep every field the solve reads in registers)
  __shared__ PcgArgs s_args;
  {
    static_assert(sizeof(PcgArgs) % sizeof(unsigned long long) == 0, "PcgArgs: whole 8-byte words");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&g.a[j]);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_args);
    for (int k = threadIdx.x; k < (int)(sizeof(PcgArgs) / 8); k += TPB) dst[k] = src[k];
  }
  __syncthreads();
  const PcgArgs& a = s_args;
  __shared__ double smem[2 * 32 * 4];
  constexpr int wpb = TPB / 32;
  const int nb = g.start[j + 1] - g.start[j], rank = (int)blockIdx.x - g.start[j];
  FlagSync fs{a.flags, a.parts, a.sync, 0u, a.spin_ns, nb, rank};
  const int gwarp = rank * wpb + (int)(threadIdx.x >> 5), nwarps = nb * wpb, lane = threadIdx.x & 31;
  const bool leader = rank == 0 && threadIdx.x == 0;
  double skip[1] = {solve_skipped(a.sc) ? 1.0 : 0.0};
  bool ok = grid_allsum<1>(skip, fs, smem);
  if (ok && skip[0] > 0.0) return;
  if (ok) {
    if constexpr (kBicg) {
      ok = amg_bicgstab_solve<T>(a, amg_of<T>(a), fs, smem, gwarp, nwarps, lane, leader);
    } else {
      GridOps ops{fs, smem};
      ok = amg_cg_solve<T>(a, amg_of<T>(a), a.z, ops, gwarp, nwarps, lane, leader);
    }
  }
  if (!ok && threadIdx.x == 0) report_timeout(a);
}


// Mixed precision with the AMG preconditioner (solver kind 10): FP64 outer residual
// r = b' - A x and correction x += ||r|| e; the inner solve A e = r / ||r|| runs CG in FP32
// (FP32 matrix copies and vectors, compensated FP32 dot products per thread, FP64 grid sums)
// preconditioned by the FP32 V-cycle, to a relative reduction inner_rtol.  The stopping test
// is the FP64 one of the other kernels.
template <int TPB>
__global__ void __launch_bounds__(TPB, 1) pcg_amg_mixed_kernel(PcgArgs a) {
  if (solve_skipped(a.sc)) return;  // an earlier stage of this run failed beyond repair
  __shared__ double smem[2 * 32 * 4];
  constexpr int wpb = TPB / 32;
  FlagSync fs{a.flags, a.parts, a.sync, 0u, a.spin_ns, (int)gridDim.x, (int)blockIdx.x};
  GridOps ops{fs, smem};
  if (!amg_mixed_solve(a, ops, blockIdx.x * wpb + (threadIdx.x >> 5), gridDim.x * wpb, threadIdx.x & 31,
                       blockIdx.x == 0 && threadIdx.x == 0) &&
      threadIdx.x == 0)
    report_timeout(a);
}

template <typename T>
static const void* amg_kernel_ptr_t(int kind, int tpb) {
  if (kind == 9) {
    switch (tpb) {
      case 768: return (const void*)bicgstab_amg_kernel<768, T>;
      case 1024: return (const void*)bicgstab_amg_kernel<1024, T>;
      default: return (const void*)bicgstab_amg_kernel<512, T>;
    }
  }
  switch (tpb) {
    case 768: return (const void*)pcg_amg_kernel<768, T>;
    case 1024: return (const void*)pcg_amg_kernel<1024, T>;
    default: return (const void*)pcg_amg_kernel<512, T>;
  }
}

// Kernel of solver kind 8 (CG), 9 (BiCGStab) or 10 (mixed precision) with an FP32 (fp64 = 0)
// or FP64 hierarchy; kind 10 always takes the FP32 one.
static const void* amg_kernel_ptr(int kind, int tpb, int fp64) {
  if (kind == 10) {
    switch (tpb) {
      case 768: return (const void*)pcg_amg_mixed_kernel<768>;
      case 1024: return (const void*)pcg_amg_mixed_kernel<1024>;
      default: return (const void*)pcg_amg_mixed_kernel<512>;
    }
  }
  return fp64 ? amg_kernel_ptr_t<double>(kind, tpb) : amg_kernel_ptr_t<float>(kind, tpb);
}

// Grid: co-resident blocks (one per SM), no more than the finest level needs.
PcgPlan amg_plan(int nslices, int requested_tpb, int kind, int fp64) {
  PcgPlan pl;
  pl.kind = kind;
  pl.maxs = fp64;  // FP64 hierarchy (1) or FP32 (0)
  pl.tpb = amg_default_threads(kind, fp64);
  for (int t : kAmgSizes)
    if (t == requested_tpb) pl.tpb = t;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, amg_kernel_ptr(kind, pl.tpb, fp64), pl.tpb, 0);
  const int wpb = pl.tpb / kSlice;
  const int want = (nslices + wpb - 1) / wpb;
  pl.blocks = std::max(1, std::min(std::max(occ, 1) * std::max(sms, 1), want));
  return pl;
}

cudaError_t launch_pcg_amg(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st) {
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
  return cudaLaunchKernelExC(&cfg, amg_kernel_ptr(pl.kind, pl.tpb, pl.maxs), kargs);
}

template <typename T, bool kBicg>
static const void* amg_group_ptr_t(int tpb) {
  switch (tpb) {
    case 768: return (const void*)amg_group_kernel<768, T, kBicg>;
    case 1024: return (const void*)amg_group_kernel<1024, T, kBicg>;
    default: return (const void*)amg_group_kernel<512, T, kBicg>;
  }
}

// The side-by-side solves of g.n systems of solver kind pl.kind (8: CG, 9: BiCGStab) over the
// grid of pl (the grid of the single solve: one block per SM).
cudaError_t launch_amg_group(const AmgGroupArgs& g, const PcgPlan& pl, cudaStream_t st) {
  const bool bicg = pl.kind == 9;
  const void* fn = pl.maxs ? (bicg ? amg_group_ptr_t<double, true>(pl.tpb) : amg_group_ptr_t<double, false>(pl.tpb))
                           : (bicg ? amg_group_ptr_t<float, true>(pl.tpb) : amg_group_ptr_t<float, false>(pl.tpb));
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
  void* kargs[] = {const_cast<AmgGroupArgs*>(&g)};
  return cudaLaunchKernelExC(&cfg, fn, kargs);
}

}  // namespace avip
