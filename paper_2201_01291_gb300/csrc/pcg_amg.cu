// Conjugate gradients preconditioned by one smoothed-aggregation AMG V-cycle (solver kind 8),
// FP64, one cooperative persistent launch per solve.
//
// The system is the symmetrically scaled one of the Jacobi variant, A = D^-1/2 K D^-1/2,
// x = D^1/2 phi, b' = D^-1/2 b, with the same stopping test (true residual of the free rows,
// ||b' - A x|| <= rtol ||b'||).  The hierarchy (level matrices, prolongators, restrictions,
// diagonal inverses, largest-eigenvalue estimates, dense inverse of the coarsest matrix) is
// built once per mesh on the host (amg_setup.cpp); the preconditioner z = M r is one V-cycle:
//
//   down, level l:  x = Chebyshev(degree 2, from x = 0) of A_l x = b_l;
//                   r = b_l - A_l x;  b_{l+1} = R_l r
//   coarsest:       x = A_c^-1 b  (dense product)
//   up, level l:    x += P_l x_{l+1};  x = Chebyshev(degree 2, from x) of A_l x = b_l
//
// with the Chebyshev polynomial in D^-1 A on [lmax/30, lmax] (lmax from power iteration).
// The pre- and post-smoother are the same polynomial and R = P^T, so the V-cycle is a
// symmetric positive definite operator and plain CG applies.
//
// Every product gathers a vector that other blocks wrote in the previous phase, so each phase
// ends with a grid-wide barrier (a reduction that also carries the dot products CG needs).  No
// phase writes a vector that it also gathers: the Chebyshev steps gather the direction d and
// update x, and the first direction of each level is formed where its right-hand side is
// written (the restriction of the level above, or the CG residual update on the finest).
// Per CG iteration: 6 barriers per non-coarsest level, 1 for the coarsest, 2 for CG.
#include <cuda_runtime.h>

#include <algorithm>

#include "avip_internal.h"
#include "grid_sync.cuh"
#include "sell.cuh"

namespace avip {

namespace {
constexpr int kAmgSizes[] = {512, 768, 1024};  // block sizes; index 0 is the default
constexpr int kAmgMaxRestarts = 8;

// Degree-2 Chebyshev coefficients on [lmax/30, lmax]: d0 = D^-1 r / theta,
// d1 = c1 d0 + c2 D^-1 r1.
struct Cheb {
  double inv_theta, c1, c2;
};
__device__ __forceinline__ Cheb cheb_of(double lmax) {
  const double lmin = lmax / 30.0;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  const double rho0 = 1.0 / sigma, rho1 = 1.0 / (2.0 * sigma - rho0);
  return Cheb{1.0 / theta, rho1 * rho0, 2.0 * rho1 / delta};
}

__device__ __forceinline__ bool grid_barrier(FlagSync& fs, double* smem) {
  double d[1] = {0.0};
  return grid_allsum<1>(d, fs, smem);
}

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
template <typename T>
__device__ bool vcycle(const AmgDevT<T>* __restrict__ H, const T* __restrict__ b0, T* __restrict__ x0,
                       FlagSync& fs, double* smem, int gwarp, int nwarps, int lane, double& rz) {
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
      const Cheb ch = cheb_of(L->lmax);
      const T c1 = (T)ch.c1, c2 = (T)ch.c2;
      // second Chebyshev step from x = d0: r1 = b - A d0, x = d0 + c1 d0 + c2 D^-1 r1
      for (int sl = gwarp; sl < A.nslices; sl += nwarps) {
        const int i = sl * kSlice + lane;
        if (i >= n) continue;
        const T di = d[i];
        const T r1 = b[i] - sellmat_row_dot(A, sl, lane, i, (const T*)d);
        x[i] = di + fma_t(c1, di, c2 * dinv[i] * r1);
      }
    }
    if (!grid_barrier(fs, smem)) return false;
    // residual
    for (int sl = gwarp; sl < A.nslices; sl += nwarps) {
      const int i = sl * kSlice + lane;
      if (i >= n) continue;
      r[i] = b[i] - sellmat_row_dot(A, sl, lane, i, (const T*)x);
    }
    if (!grid_barrier(fs, smem)) return false;
    {  // restriction, and the first Chebyshev direction of the next level
      const AmgLevelT<T>* __restrict__ C = H->L + l + 1;
      const SellMatT<T> R = L->R;
      const int nc = C->n;
      const T c_inv_theta = (T)cheb_of(C->lmax).inv_theta;
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
    if (!grid_barrier(fs, smem)) return false;
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
    double av[1] = {acc.value()};
    if (!grid_allsum<1>(av, fs, smem)) return false;
    if (nl == 1) rz = av[0];
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
    if (!grid_barrier(fs, smem)) return false;
    const Cheb ch = cheb_of(L->lmax);
    const T inv_theta = (T)ch.inv_theta, c1 = (T)ch.c1, c2 = (T)ch.c2;
    // first post-smoothing step: r = b - A x, d = D^-1 r / theta (x updated in the next phase)
    for (int sl = gwarp; sl < A.nslices; sl += nwarps) {
      const int i = sl * kSlice + lane;
      if (i >= n) continue;
      const T ri = b[i] - sellmat_row_dot(A, sl, lane, i, (const T*)x);
      r[i] = ri;
      d[i] = dinv[i] * ri * inv_theta;
    }
    if (!grid_barrier(fs, smem)) return false;
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
    double av[1] = {acc.value()};
    if (!grid_allsum<1>(av, fs, smem)) return false;
    if (l == 0) rz = av[0];
  }
  return true;
}
}  // namespace

template <int TPB>
__global__ void __launch_bounds__(TPB, 1) pcg_amg_kernel(PcgArgs a) {
  if (solve_skipped(a.sc)) return;  // an earlier stage of this run failed beyond repair
  __shared__ double smem[2 * 32 * 4];
  const int lane = threadIdx.x & 31;
  constexpr int wpb = TPB / 32;
  const int gwarp = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  const int N = a.A.N, nsl = a.A.nslices;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
  const AmgDev* __restrict__ H = a.amg;
  const double* __restrict__ dinv0 = H->L[0].dinv;
  double* __restrict__ d0 = H->L[0].d;
  double* __restrict__ z = a.z;  // preconditioned residual (the V-cycle's finest solution)
  const double inv_theta0 = cheb_of(H->L[0].lmax).inv_theta;
  FlagSync fs{a.flags, a.parts, a.sync, 0u};
  double one[1];

  // ---- x = D^1/2 phi (warm start) and b'
  double bb[1] = {0.0};
  for (int s = gwarp; s < nsl; s += nwarps) {
    const int i = s * kSlice + lane;
    if (i >= N) continue;
    a.x[i] = a.dsq[i] * a.phi[i];
    double b;
    if (a.use_density_rhs) {
      double rho = 0.0;
      for (int k = 0; k < a.ns; ++k) rho = fma(a.q[k], nb[(size_t)k * a.Npad + i], rho);
      b = fma(a.rhs_scale[i], rho, a.lift[i]);
      a.b[i] = b;
    } else {
      b = a.b[i];
    }
    if (a.rhs_scale[i] != 0.0) bb[0] = fma(b, b, bb[0]);  // free rows only: a Dirichlet row holds its value exactly
  }
  if (!grid_allsum<1>(bb, fs, smem)) goto timeout;
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
          if (!grid_allsum<1>(r2, fs, smem)) goto timeout;
          rr_true = r2[0];
          if (rr_true <= thresh) break;
          if (!isfinite(rr_true)) {  // non-finite data: stop at once
            status = AVIP_ENAN;
            break;
          }
          if (it >= a.max_iter || (it > 0 && restarts >= kAmgMaxRestarts)) {
            status = AVIP_ENOTCONV;
            break;
          }
          if (it > 0) ++restarts;
          fresh = true;
          check = false;
        }
        // ---- z = M r (r and the level-0 direction complete)
        double rz_new = 0.0;
        if (!vcycle(H, a.r, z, fs, smem, gwarp, nwarps, lane, rz_new)) goto timeout;
        if (!(rz_new > 0.0) || !isfinite(rz_new)) {  // the preconditioned residual lost positivity
          if (it == 0 || restarts >= kAmgMaxRestarts) {
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
        const double rz_now = rz;
        if (!grid_allsum<1, 1>(pq, one, fs, smem, [rz_now](const double* t, double* e) { e[0] = rz_now / t[0]; }))
          goto timeout;
        const double alpha = one[0];
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
        double stop[1];
        if (!grid_allsum<1, 1>(rn, stop, fs, smem, [thresh](const double* t, double* e) {
              e[0] = (t[0] <= thresh || !isfinite(t[0])) ? 1.0 : 0.0;
            }))
          goto timeout;
        check = stop[0] != 0.0;
        ++it;
      }
    }
    // ---- phi = D^-1/2 x
    for (int s = gwarp; s < nsl; s += nwarps) {
      const int i = s * kSlice + lane;
      if (i < N) a.phi[i] = a.dsqinv[i] * a.x[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.sc->pcg_iters = it;
      a.sc->pcg_status = status;
      a.sc->pcg_relres = bb[0] > 0.0 ? sqrt(rr_true / bb[0]) : 0.0;
      a.sc->pcg_bnorm = sqrt(bb[0]);
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

// BiCGStab right-preconditioned by the same V-cycle, for the non-symmetric axisymmetric
// matrix (solver kind 9): with p^ = M p and s^ = M s,
//   P1  v = A p^, rh.v -> alpha;  P2  s = r - alpha v (barrier);  P3  t = A s^, t.s, t.t, rh.s,
//   rh.t -> omega, rho', beta;  P4  x += alpha p^ + omega s^, r = s - omega t,
//   p = r + beta (p - omega v), r.r -> stop test
// (van der Vorst's iteration with M^-1 applied on the right, so x is updated directly and the
// stopping test stays on the true scaled residual of the free rows).  Two V-cycles per
// iteration; breakdowns and a true residual still too large restart from the true residual.
template <int TPB>
__global__ void __launch_bounds__(TPB, 1) bicgstab_amg_kernel(PcgArgs a) {
  if (solve_skipped(a.sc)) return;  // an earlier stage of this run failed beyond repair
  __shared__ double smem[2 * 32 * 4];
  const int lane = threadIdx.x & 31;
  constexpr int wpb = TPB / 32;
  const int gwarp = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  const int N = a.A.N, nsl = a.A.nslices;
  const size_t Np = (size_t)a.Npad;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * Np;
  const AmgDev* __restrict__ H = a.amg;
  const double* __restrict__ dinv0 = H->L[0].dinv;
  double* __restrict__ d0 = H->L[0].d;
  const double inv_theta0 = cheb_of(H->L[0].lmax).inv_theta;
  double* __restrict__ x = a.x;
  double* __restrict__ r = a.r;
  double* __restrict__ p = a.p;
  double* __restrict__ v = a.q_ap;
  double* __restrict__ sv = a.bcg;
  double* __restrict__ tv = a.bcg + Np;
  double* __restrict__ rh = a.bcg + 2 * Np;
  double* __restrict__ ph = a.bcg + 3 * Np;
  double* __restrict__ sh = a.bcg + 4 * Np;
  FlagSync fs{a.flags, a.parts, a.sync, 0u};
  double dummy = 0.0;

  double bb[1] = {0.0};
  for (int sl = gwarp; sl < nsl; sl += nwarps) {
    const int i = sl * kSlice + lane;
    if (i >= N) continue;
    x[i] = a.dsq[i] * a.phi[i];
    double b;
    if (a.use_density_rhs) {
      double rho = 0.0;
      for (int k = 0; k < a.ns; ++k) rho = fma(a.q[k], nb[(size_t)k * Np + i], rho);
      b = fma(a.rhs_scale[i], rho, a.lift[i]);
      a.b[i] = b;
    } else {
      b = a.b[i];
    }
    if (a.rhs_scale[i] != 0.0) bb[0] = fma(b, b, bb[0]);  // free rows only: a Dirichlet row holds its value exactly
  }
  if (!grid_allsum<1>(bb, fs, smem)) goto timeout;
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
          for (int sl = gwarp; sl < nsl; sl += nwarps) {
            const int i = sl * kSlice + lane;
            if (i >= N) continue;
            const double ri = a.b[i] - sell_row_dot(a.A, sl, lane, i, x);
            r[i] = ri;
            rh[i] = ri;
            p[i] = ri;
            d0[i] = dinv0[i] * ri * inv_theta0;
            r2[0] = fma(ri, ri, r2[0]);
          }
          if (!grid_allsum<1>(r2, fs, smem)) goto timeout;
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
        if (!vcycle(H, p, ph, fs, smem, gwarp, nwarps, lane, dummy)) goto timeout;
        double rv[1] = {0.0};
        for (int sl = gwarp; sl < nsl; sl += nwarps) {
          const int i = sl * kSlice + lane;
          if (i >= N) continue;
          const double w = sell_row_dot(a.A, sl, lane, i, ph);
          v[i] = w;
          rv[0] = fma(rh[i], w, rv[0]);
        }
        double al[1];
        const double rho_now = rho;
        if (!grid_allsum<1, 1>(rv, al, fs, smem, [rho_now](const double* t, double* e) {
              e[0] = t[0] != 0.0 ? rho_now / t[0] : 0.0;
            }))
          goto timeout;
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
          d0[i] = dinv0[i] * si * inv_theta0;
          ss[0] = fma(si, si, ss[0]);
        }
        if (!grid_allsum<1>(ss, fs, smem)) goto timeout;
        if (ss[0] <= thresh) {  // s small enough: x += alpha p^, confirm on the true residual
          for (int sl = gwarp; sl < nsl; sl += nwarps) {
            const int i = sl * kSlice + lane;
            if (i < N) x[i] = fma(alpha, __ldcg(ph + i), x[i]);
          }
          ++it;
          restart = true;
          double z0[1] = {0.0};
          if (!grid_allsum<1>(z0, fs, smem)) goto timeout;
          continue;
        }
        // ---- s^ = M s, then P3: t = A s^
        if (!vcycle(H, sv, sh, fs, smem, gwarp, nwarps, lane, dummy)) goto timeout;
        double d4[4] = {0.0, 0.0, 0.0, 0.0};  // t.s, t.t, rh.s, rh.t
        for (int sl = gwarp; sl < nsl; sl += nwarps) {
          const int i = sl * kSlice + lane;
          if (i >= N) continue;
          const double ti = sell_row_dot(a.A, sl, lane, i, sh);
          const double si = sv[i], rhi = rh[i];
          tv[i] = ti;
          d4[0] = fma(ti, si, d4[0]);
          d4[1] = fma(ti, ti, d4[1]);
          d4[2] = fma(rhi, si, d4[2]);
          d4[3] = fma(rhi, ti, d4[3]);
        }
        double e3[3];
        if (!grid_allsum<4, 3>(d4, e3, fs, smem, [rho_now, alpha](const double* t, double* e) {
              const double om = t[1] > 0.0 ? t[0] / t[1] : 0.0;
              const double rn = t[2] - om * t[3];
              e[0] = om;
              e[1] = rn;
              e[2] = (om != 0.0 && rn != 0.0) ? (rn / rho_now) * (alpha / om) : 0.0;
            }))
          goto timeout;
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
          d0[i] = dinv0[i] * pn * inv_theta0;
          rn2[0] = fma(ri, ri, rn2[0]);
        }
        if (!grid_allsum<1>(rn2, fs, smem)) goto timeout;
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
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.sc->pcg_iters = it;
      a.sc->pcg_status = status;
      a.sc->pcg_relres = bb[0] > 0.0 ? sqrt(rr_true / bb[0]) : 0.0;
      a.sc->pcg_bnorm = sqrt(bb[0]);
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

// Mixed precision with the AMG preconditioner (solver kind 10): FP64 outer residual
// r = b' - A x and correction x += ||r|| e; the inner solve A e = r / ||r|| runs CG in FP32
// (FP32 matrix copies and vectors, compensated FP32 dot products per thread, FP64 grid sums)
// preconditioned by the FP32 V-cycle, to a relative reduction inner_rtol.  The stopping test
// is the FP64 one of the other kernels.
template <int TPB>
__global__ void __launch_bounds__(TPB, 1) pcg_amg_mixed_kernel(PcgArgs a) {
  if (solve_skipped(a.sc)) return;  // an earlier stage of this run failed beyond repair
  __shared__ double smem[2 * 32 * 4];
  const int lane = threadIdx.x & 31;
  constexpr int wpb = TPB / 32;
  const int gwarp = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  const int N = a.A.N, nsl = a.A.nslices;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
  const AmgDevT<float>* __restrict__ H = a.amg32;
  const SellMatT<float> A32 = H->L[0].A;
  const float* __restrict__ dinv0 = H->L[0].dinv;
  float* __restrict__ d0 = H->L[0].d;
  const float inv_theta0 = (float)cheb_of(H->L[0].lmax).inv_theta;
  float* __restrict__ r32 = a.r32;
  float* __restrict__ e32 = a.e32;
  float* __restrict__ p32 = a.p32;
  float* __restrict__ q32 = a.q32;
  float* __restrict__ z32 = a.z32;
  FlagSync fs{a.flags, a.parts, a.sync, 0u};
  double one[1];

  double bb[1] = {0.0};
  for (int s = gwarp; s < nsl; s += nwarps) {
    const int i = s * kSlice + lane;
    if (i >= N) continue;
    a.x[i] = a.dsq[i] * a.phi[i];
    double b;
    if (a.use_density_rhs) {
      double rho = 0.0;
      for (int k = 0; k < a.ns; ++k) rho = fma(a.q[k], nb[(size_t)k * a.Npad + i], rho);
      b = fma(a.rhs_scale[i], rho, a.lift[i]);
      a.b[i] = b;
    } else {
      b = a.b[i];
    }
    if (a.rhs_scale[i] != 0.0) bb[0] = fma(b, b, bb[0]);  // free rows only: a Dirichlet row holds its value exactly
  }
  if (!grid_allsum<1>(bb, fs, smem)) goto timeout;
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
      if (!grid_allsum<1>(r2, fs, smem)) goto timeout;
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
      if (!grid_allsum<1>(g0, fs, smem)) goto timeout;
      const double inner_thresh = a.inner_rtol * a.inner_rtol * g0[0];
      double rr = g0[0], rz = 0.0;
      bool fresh = true;
      while (rr > inner_thresh && it < a.max_iter) {
        double rz_new = 0.0;
        if (!vcycle(H, (const float*)r32, z32, fs, smem, gwarp, nwarps, lane, rz_new)) goto timeout;
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
        const double rz_now = rz;
        if (!grid_allsum<1, 1>(pq, one, fs, smem, [rz_now](const double* t, double* e) { e[0] = rz_now / t[0]; }))
          goto timeout;
        const float alpha = (float)one[0];
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
        if (!grid_allsum<1>(rn, fs, smem)) goto timeout;
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
      if (!grid_allsum<1>(z0, fs, smem)) goto timeout;  // x complete before the next residual
    }
    for (int s = gwarp; s < nsl; s += nwarps) {
      const int i = s * kSlice + lane;
      if (i < N) a.phi[i] = a.dsqinv[i] * (bb[0] == 0.0 ? a.b[i] : a.x[i]);  // free b == 0: x = b
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.sc->pcg_iters = it;
      a.sc->pcg_outer = outer;
      a.sc->pcg_status = status;
      a.sc->pcg_relres = bb[0] > 0.0 ? sqrt(rr64 / bb[0]) : 0.0;
      a.sc->pcg_bnorm = sqrt(bb[0]);
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

static const void* amg_kernel_ptr(int kind, int tpb) {
  if (kind == 10) {
    switch (tpb) {
      case 768: return (const void*)pcg_amg_mixed_kernel<768>;
      case 1024: return (const void*)pcg_amg_mixed_kernel<1024>;
      default: return (const void*)pcg_amg_mixed_kernel<512>;
    }
  }
  if (kind == 9) {
    switch (tpb) {
      case 768: return (const void*)bicgstab_amg_kernel<768>;
      case 1024: return (const void*)bicgstab_amg_kernel<1024>;
      default: return (const void*)bicgstab_amg_kernel<512>;
    }
  }
  switch (tpb) {
    case 768: return (const void*)pcg_amg_kernel<768>;
    case 1024: return (const void*)pcg_amg_kernel<1024>;
    default: return (const void*)pcg_amg_kernel<512>;
  }
}

// Grid: co-resident blocks (one per SM), no more than the finest level needs.
PcgPlan amg_plan(int nslices, int requested_tpb, int kind) {
  PcgPlan pl;
  pl.kind = kind;
  pl.tpb = kAmgSizes[0];
  for (int t : kAmgSizes)
    if (t == requested_tpb) pl.tpb = t;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, amg_kernel_ptr(kind, pl.tpb), pl.tpb, 0);
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
  return cudaLaunchKernelExC(&cfg, amg_kernel_ptr(pl.kind, pl.tpb), kargs);
}

}  // namespace avip
