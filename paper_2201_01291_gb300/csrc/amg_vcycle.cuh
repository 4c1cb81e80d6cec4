// Smoothed-aggregation AMG V-cycle shared by the whole-GPU cooperative solvers (grid-wide
// barriers) and the cluster solvers (one thread-block cluster per instance, cluster barriers).
//
// Each non-coarsest level takes two phases, through the composite operators built on the host
// (amg_setup.cpp): down, xp = Q b and b' = Rf b (the pre-smoothing, the residual and its
// restriction); up, x = U xp + Pf x' (the coarse correction and the post-smoothing).  It is the
// V-cycle of a damped Jacobi smoother (the same step before and after), R = P^T and a dense
// coarsest solve, written with fewer grid-wide phases: every phase gathers only vectors
// completed by an earlier one.  The values are FP32 by default (the preconditioner only shapes
// the search directions; the iterate, the residuals and the stopping test stay FP64) or FP64.
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

// Down phase of level l: xp = Q b on the rows of level l (Q = omega D^-1 is diagonal: an
// elementwise pass) and b' = Rf b on the rows of level l + 1 (a streamed product), b given by
// `src` (complete on entry).  `hook` takes part in every row i of level l: hook.begin(i) loads
// the row's own operands, hook.end(i, pre) runs with them (the CG update folded into the
// finest level's phase).  The elementwise pass takes one row per thread at a time (issuing the
// loads of several rows before their use kept more registers live than the 64 - 80 a thread has
// at 768 - 1024 threads per block: the spills cost more than the extra loads in flight saved);
// then every warp streams a contiguous share of Rf.
template <typename T, int U, class Src, class Hook>
__device__ __forceinline__ void amg_down(const AmgDevT<T>* __restrict__ H, int l, Src src, Hook hook, int gwarp,
                                         int nwarps, int lane) {
  const AmgLevelT<T>& L = H->L[l];
  T* __restrict__ bn = H->L[l + 1].b;
  T* __restrict__ xp = L.xp;
  const T* __restrict__ qd = L.qd;
  const int n = L.n;
  for (int i = gwarp * kSlice + lane; i < n; i += nwarps * kSlice) {
    const auto pre = hook.begin(i);
    const T bi = src(i);
    const T qi = __ldg(qd + i);
    hook.end(i, pre);
    xp[i] = qi * bi;
  }
  int sa, sb;
  warp_slices(L.Rf.nslices, gwarp, nwarps, sa, sb);
  spmv_stream<T, U>(L.Rf, sa, sb, lane, src, NoBegin(), [&](int j, T v, NoPre) { bn[j] = v; });
}

// Up phase of level l: x = U xp + Pf x' = [U | Pf] [xp; x'] on the rows of level l (x' = the
// next level's solution, complete on entry), each row handed to out.end(i, value, pre) with the
// operands out.begin(i) fetched ahead.
template <typename T, int U, class Out>
__device__ __forceinline__ void amg_up(const AmgDevT<T>* __restrict__ H, int l, Out out, int gwarp, int nwarps,
                                       int lane) {
  const AmgLevelT<T>& L = H->L[l];
  const T* __restrict__ xp = L.xp;
  const T* __restrict__ xn = H->L[l + 1].x;
  const int n = L.n;
  int sa, sb;
  warp_slices(L.UP.nslices, gwarp, nwarps, sa, sb);
  spmv_stream<T, U>(L.UP, sa, sb, lane, [xp, xn, n](int c) { return __ldca(c < n ? xp + c : xn + (c - n)); },
                    [&](int i) { return out.begin(i); },
                    [&](int i, T v, const decltype(out.begin(0))& pre) { out.end(i, v, pre); });
}

// Row hooks and outputs without prefetched operands.
struct NoHook {
  __device__ NoPre begin(int) const { return NoPre(); }
  __device__ void end(int, NoPre) const {}
};
template <typename T>
struct StoreOut {  // x_i = value
  T* x;
  __device__ NoPre begin(int) const { return NoPre(); }
  __device__ void end(int i, T v, NoPre) const { x[i] = v; }
};

// Coarsest level: x = A_c^-1 b as a dense product, one warp per row; b given by `src`
// (complete on entry), each row handed to out(row, value) by lane 0.
template <typename T, class Src, class Out>
__device__ __forceinline__ void amg_coarse(const AmgDevT<T>* __restrict__ H, Src src, Out out, int gwarp,
                                           int nwarps, int lane) {
  constexpr int K = 8;  // independent loads per lane in flight
  const int n = H->nc;
  const T* __restrict__ cinv = H->cinv;
  for (int row = gwarp; row < n; row += nwarps) {
    const T* __restrict__ crow = cinv + (size_t)row * n;
    T s = T(0);
    for (int k0 = lane; k0 < n; k0 += 32 * K) {
      T c[K], b[K];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int k = k0 + 32 * u;
        c[u] = k < n ? __ldg(crow + k) : T(0);
        b[u] = k < n ? src(k) : T(0);
      }
#pragma unroll
      for (int u = 0; u < K; ++u) s = fma_t(c[u], b[u], s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out(row, s);
  }
}

// The V-cycle below the finest level: down phases of levels 1 .. nlev-2, the coarsest solve,
// up phases of levels nlev-2 .. 1, one barrier after each.  Entered once the finest down phase
// is complete (nlev >= 2); on return the level-1 solution is complete.
template <typename T, class Ops>
__device__ bool amg_inner(const AmgDevT<T>* __restrict__ H, Ops& ops, int gwarp, int nwarps, int lane) {
  const int nl = H->nlev;
  for (int l = 1; l + 1 < nl; ++l) {
    const T* __restrict__ b = H->L[l].b;
    amg_down<T, Ops::kStream>(H, l, [b](int c) { return __ldca(b + c); }, NoHook(), gwarp, nwarps, lane);
    if (!ops.barrier()) return false;
  }
  {
    const T* __restrict__ cb = H->L[nl - 1].b;
    T* __restrict__ cx = H->L[nl - 1].x;
    amg_coarse(H, [cb](int k) { return __ldca(cb + k); }, [cx](int row, T v) { cx[row] = v; }, gwarp, nwarps, lane);
    if (!ops.barrier()) return false;
  }
  for (int l = nl - 2; l >= 1; --l) {
    amg_up<T, Ops::kStream>(H, l, StoreOut<T>{H->L[l].x}, gwarp, nwarps, lane);
    if (!ops.barrier()) return false;
  }
  return true;
}

// One V-cycle z = M b0, b0 complete on entry (TB: its type; TZ: the type z is stored in).  With
// want_dot the last barrier is a grid sum that returns dot = b0.z; otherwise a plain barrier.
// Returns false if a wait was abandoned.
template <typename T, typename TB, typename TZ, class Ops>
__device__ bool vcycle(const AmgDevT<T>* __restrict__ H, const TB* __restrict__ b0, TZ* __restrict__ z, Ops& ops,
                       int gwarp, int nwarps, int lane, bool want_dot, double& dot) {
  auto src = [b0](int c) { return (T)__ldca(b0 + c); };
  DotAcc<double> acc;
  struct Out {  // z_i = value, b0_i z_i into the dot product
    const TB* b0;
    TZ* z;
    DotAcc<double>* acc;
    __device__ double begin(int i) const { return (double)__ldca(b0 + i); }
    __device__ void end(int i, T v, double bi) const {
      z[i] = (TZ)v;
      acc->add(bi, (double)v);
    }
  } out{b0, z, &acc};
  if (H->nlev == 1) {
    amg_coarse(H, src, [&](int row, T v) { out.end(row, v, out.begin(row)); }, gwarp, nwarps, lane);
  } else {
    amg_down<T, Ops::kStream>(H, 0, src, NoHook(), gwarp, nwarps, lane);
    if (!ops.barrier()) return false;
    if (!amg_inner(H, ops, gwarp, nwarps, lane)) return false;
    amg_up<T, Ops::kStream>(H, 0, out, gwarp, nwarps, lane);
  }
  if (want_dot) {
    double v[1] = {acc.value()};
    if (!ops.sum(v)) return false;
    dot = v[0];
    return true;
  }
  return ops.barrier();
}

// CG preconditioned by the V-cycle on the scaled system (kinds 8, 11 and the batched FP64 form):
// warm start, b', true-residual checks and restarts, phi = D^-1/2 x.  The hierarchy H (values of
// type T) writes the preconditioned residual z in FP64 (only w = A z gathers it).  The residual update r - alpha q and
// x += alpha p of iteration k are folded into the finest down phase of iteration k + 1, whose
// products gather r - alpha q directly (the new residual goes to the other buffer, r2), so an
// iteration takes 2 nlev grid-wide phases: the finest down phase (sum of r.r: stop test), the
// levels below, the finest up phase (sum of r.z), and w = A z (sum of p.q).  `leader` is the
// one thread that writes the solve statistics.  Returns false if a wait was abandoned.
template <typename T, class Ops>
__device__ bool amg_cg_solve(const PcgArgs& a, const AmgDevT<T>* __restrict__ H, double* __restrict__ z, Ops& ops,
                             int gwarp, int nwarps, int lane, bool leader) {
  constexpr int kMaxRestarts = 8;
  const int N = a.A.N, nsl = a.A.nslices, nl = H->nlev;
  const double* nb = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;

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
    // the Poisson matrix as a streamed operator, and this warp's contiguous share of its slices
    const SellMatT<double> A0{a.A.sl_ptr, a.A.sl_w, a.A.rlen, a.A.col, a.A.aval, N, nsl, 1};
    int ma, mb;
    warp_slices(nsl, gwarp, nwarps, ma, mb);
    double* rc = a.r;   // current residual
    double* rn = a.r2;  // the other buffer
    // the vectors the finest down phase gathers, in the hierarchy's type: with T = float, FP32
    // copies of r (both buffers) and q, written beside them; with T = double, r and q themselves
    constexpr bool kCopies = sizeof(T) == 4;
    T* tc = kCopies ? (T*)a.rq32 : (T*)rc;
    T* tn = kCopies ? (T*)a.rq32 + a.Npad : (T*)rn;
    T* tq = kCopies ? (T*)a.rq32 + 2 * (size_t)a.Npad : (T*)a.q_ap;
    double rz = 0.0, rr_true = 0.0, alpha = 0.0;
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
          // ---- true residual r = b' - A x (x complete)
          double r2[1] = {0.0};
          {
            const double* __restrict__ xv = a.x;
            const double* __restrict__ bv = a.b;
            double* __restrict__ rw = rc;
            T* __restrict__ tw = tc;
            spmv_stream<double, Ops::kStream64>(
                A0, ma, mb, lane, [xv](int c) { return __ldca(xv + c); }, [bv](int i) { return bv[i]; },
                [&](int i, double ax, double bi) {
                  const double r = bi - ax;
                  rw[i] = r;
                  if (kCopies) tw[i] = (T)r;
                  r2[0] = fma(r, r, r2[0]);
                });
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
        // ---- finest down phase on the residual, updated by the last step unless fresh:
        //      r' = r - alpha q, x += alpha p (own rows), r'.r'; xp0 = Q r', b1 = Rf r'
        {
          const double al = fresh ? 0.0 : alpha;
          const bool upd = !fresh;
          const double* __restrict__ rv = rc;
          const double* __restrict__ qv = a.q_ap;
          const T* __restrict__ trv = tc;
          const T* __restrict__ tqv = tq;
          const T alT = (T)al;
          // the gathered residual r - alpha q in the hierarchy's type
          auto res = [trv, tqv, alT, upd](int c) {
            return upd ? fma_t(-alT, __ldca(tqv + c), __ldca(trv + c)) : __ldca(trv + c);
          };
          double rr = 0.0;
          struct Pre {
            double r, q, x, p;
          };
          struct Hook {  // r' = r - alpha q into the other buffer (and its copy), x += alpha p, r'.r'
            const double *rv, *qv, *pv;
            double *xv, *rnv, *rr;
            T* tnv;
            double al;
            bool upd;
            __device__ Pre begin(int i) const {
              if (!upd) return Pre{0.0, 0.0, 0.0, 0.0};
              return Pre{__ldca(rv + i), __ldca(qv + i), xv[i], pv[i]};
            }
            __device__ void end(int i, const Pre& p) const {
              if (!upd) return;
              const double v = fma(-al, p.q, p.r);
              rnv[i] = v;
              if (kCopies) tnv[i] = (T)v;
              xv[i] = fma(al, p.p, p.x);
              *rr = fma(v, v, *rr);
            }
          } hook{rv, qv, a.p, a.x, rn, &rr, tn, al, upd};
          if (nl == 1) {
            for (int s = gwarp; s < nsl; s += nwarps) {
              const int i = s * kSlice + lane;
              if (i < N) hook.end(i, hook.begin(i));
            }
          } else {
            amg_down<T, Ops::kStream>(H, 0, [res](int c) { return (T)res(c); }, hook, gwarp, nwarps, lane);
          }
          if (upd) {
            double v[1] = {rr};
            if (!ops.sum(v)) return false;
            ++it;
            double* t = rc;
            rc = rn;
            rn = t;
            T* tt = tc;
            tc = tn;
            tn = tt;
            check = v[0] <= thresh || !isfinite(v[0]);
            if (check) continue;  // confirm on the true residual
          } else if (!ops.barrier()) {
            return false;
          }
        }
        // ---- the levels below, then the finest up phase: z = U0 xp0 + Pf0 x1, r.z
        double rzv[1];
        {
          DotAcc<double> acc;
          const double* __restrict__ rv = rc;
          struct Out {  // z_i = value (widened once here: w = A z gathers it in FP64), r_i z_i into r.z
            const double* rv;
            double* z;
            DotAcc<double>* acc;
            __device__ double begin(int i) const { return __ldca(rv + i); }
            __device__ void end(int i, T v, double ri) const {
              const double zi = (double)v;
              z[i] = zi;
              acc->add(ri, zi);
            }
          } out{rv, z, &acc};
          if (nl == 1) {
            amg_coarse(H, [rv](int k) { return (T)__ldca(rv + k); },
                       [&](int row, T v) { out.end(row, v, out.begin(row)); }, gwarp, nwarps, lane);
          } else {
            if (!amg_inner(H, ops, gwarp, nwarps, lane)) return false;
            amg_up<T, Ops::kStream>(H, 0, out, gwarp, nwarps, lane);
          }
          rzv[0] = acc.value();
          if (!ops.sum(rzv)) return false;
        }
        const double rz_new = rzv[0];
        if (!(rz_new > 0.0) || !isfinite(rz_new)) {  // the preconditioned residual lost positivity
          if (it == 0 || restarts >= kMaxRestarts) {
            status = AVIP_ENOTCONV;
            break;
          }
          check = true;
          continue;
        }
        const double beta = fresh ? 0.0 : rz_new / rz;
        rz = rz_new;
        fresh = false;
        // ---- w = A z, q = w + beta q, p = z + beta p, p.q -> alpha
        double pq[1] = {0.0};
        {
          const double* __restrict__ zc = z;
          double* __restrict__ qv = a.q_ap;
          double* __restrict__ pv = a.p;
          T* __restrict__ tqw = tq;
          struct PreA {
            double z, q, p;
          };
          spmv_stream<double, Ops::kStream64>(
              A0, ma, mb, lane, [zc](int c) { return __ldca(zc + c); },
              [=](int i) { return PreA{__ldca(zc + i), qv[i], pv[i]}; },
              [&](int i, double w, const PreA& o) {
                const double qn = beta == 0.0 ? w : fma(beta, o.q, w);
                const double pn = beta == 0.0 ? o.z : fma(beta, o.p, o.z);
                qv[i] = qn;
                if (kCopies) tqw[i] = (T)qn;
                pv[i] = pn;
                pq[0] = fma(pn, qn, pq[0]);
              });
        }
        if (!ops.sum(pq)) return false;
        alpha = rz / pq[0];
      }
    }
    // ---- phi = D^-1/2 x
    for (int s = gwarp; s < nsl; s += nwarps) {
      const int i = s * kSlice + lane;
      if (i < N) a.phi[i] = a.dsqinv[i] * a.x[i];
    }
    if (leader) {
      a.res->pcg_iters = it;
      advance_history(a);
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
  const SellMatT<float> A32{a.A.sl_ptr, a.A.sl_w, a.A.rlen, a.A.col, a.aval32, N, nsl, 1};
  int ma, mb;
  warp_slices(nsl, gwarp, nwarps, ma, mb);
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
      // ---- FP32 right-hand side r / ||r||, e = 0
      double g0[1];
      {
        DotAcc<float> k;
        for (int s = gwarp; s < nsl; s += nwarps) {
          const int i = s * kSlice + lane;
          if (i >= N) continue;
          const float r = (float)(a.r[i] * rscale);
          r32[i] = r;
          e32[i] = 0.f;
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
        if (!vcycle(H, (const float*)r32, z32, ops, gwarp, nwarps, lane, true, rz_new)) return false;
        if (!(rz_new > 0.0) || !isfinite(rz_new)) break;  // refine with what the inner solve has
        const float beta = fresh ? 0.f : (float)(rz_new / rz);
        rz = rz_new;
        fresh = false;
        DotAcc<float> kpq;
        struct PreA {
          float z, q, p;
        };
        spmv_stream<float, Ops::kStream>(
            A32, ma, mb, lane, [z32](int c) { return __ldca(z32 + c); },
            [=](int i) { return PreA{__ldca(z32 + i), q32[i], p32[i]}; },
            [&](int i, float w, const PreA& o) {
              const float qn = beta == 0.f ? w : fmaf(beta, o.q, w);  // (restart: old p, q unused)
              const float pn = beta == 0.f ? o.z : fmaf(beta, o.p, o.z);
              q32[i] = qn;
              p32[i] = pn;
              kpq.add(pn, qn);
            });
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
      advance_history(a);
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
// kStream / kStream64: steps per batch of the streamed products with FP32 / FP64 values (8 and 8
// for the whole-GPU kernels, measured fastest with their 24 warps per SM, and for the cluster
// solves).
struct GridOps {
  // steps of 32 elements loaded ahead by the streamed products: FP32 operators, FP64 matrix.
  // Measured on the pin-plane solve (500k rows, 1024 threads): 6 / 4 gave 99.9 us per CG
  // iteration, 8 / 4 101.2, 4 / 4 104.9, 12 / 4 139 (register spills), 8 / 8 (with row batches
  // of 4 in the down phase) 127
  static constexpr int kStream = 6, kStream64 = 4;
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
// S, S64: steps loaded ahead by the streamed FP32 / FP64 products (8 / 8 at 512 threads per CTA,
// 6 / 4 at 768, where fewer registers are left per thread).
template <int S, int S64>
struct ClusterOpsT {
  static constexpr int kStream = S, kStream64 = S64;
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
using ClusterOps = ClusterOpsT<8, 8>;

}  // namespace avip
