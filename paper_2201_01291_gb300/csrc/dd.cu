// Drift-diffusion part of the explicit step, FP64, node-centric and atomic-free.
//
//   node_fields_kernel  E = -grad(phi), grad(n_s), nodal velocities V_s = sign(q_s) mu_s E,
//                       n_s mu_s, source rates, chemical time-step candidates
//   dt_cells_kernel     cell-based CFL / Fourier / dielectric candidates (section "Time step
//                       computation"); global minimum by an integer atomicMin on the bits of
//                       the positive doubles (exact and order independent)
//   flux_update_kernel  for each node, every incident edge flux (limited Lax-Wendroff +
//                       central diffusion) and the node-flux boundary closure, then source
//                       and explicit update into the other density buffer; per-block charge
//   finalize_kernel     charge sum in fixed order, time, parity flip, run statistics
//   *32 forms           the same in FP32 arithmetic for the mixed-precision path
//
// The residual of Eq. vertex_centered_flux is a sum over the edges of each dual cell.  Here
// every node gathers its own edges (each flux is evaluated at both ends), so no scatter and
// no atomics are needed and the result is deterministic.  Each edge flux is evaluated from the
// (lower index, higher index) ordered pair, so both ends compute bit-identical values and the
// scheme stays exactly conservative.
#include <cuda_runtime.h>

#include <cfloat>

#include "avip_internal.h"
#include "fp64_math.cuh"

namespace avip {

constexpr int kDDThreads = 256;
constexpr int kDDMinThreads = 128;  // smallest block of the batched stages (autotuned)

// Local-field mobility and the Townsend exponential with the library's FP64 exp / log
// (fp64_math.cuh: a few ulp, a fraction of the FP64 instructions of the general routines).
// mu0 (max(|E|, E_floor) / E_ref)^p = mu0 exp(p (log max(|E|, E_floor) - log E_ref)), log E_ref
// from the host: no FP64 division.
__device__ __forceinline__ double mobility(const SpeciesParams& sp, double Emag) {
  if (sp.mob_model == AVIP_MOB_POWER)
    return sp.mob[0] * exp_fp64(sp.mob[2] * (log_fp64(fmax(Emag, sp.mob[3])) - sp.mob_log_ref));
  return sp.mob[0];
}

__device__ __forceinline__ double limiter(double r, double beta, int kind) {
  if (kind == AVIP_LIM_VANLEER) return (r + fabs(r)) / (1.0 + fabs(r));
  return fmax(0.0, fmax(fmin(beta * r, 1.0), fmin(r, beta)));
}

__device__ __forceinline__ void block_min_to_global(double v, unsigned long long* dst) {
  __shared__ double sm[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? sm[lane] : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0 && t < INFINITY && t > 0.0)
      atomicMin(dst, (unsigned long long)__double_as_longlong(t));
  }
}

// ------------------------------------------------------------------------ nodal fields
__device__ __forceinline__ void node_fields_body(const DDArgs& a, int with_dt, int bid) {
  const int i = bid * blockDim.x + threadIdx.x;
  const int N = a.A.N;
  const int ns = a.ph.ns;
  double chem = INFINITY;
  if (i < N) {
    const int slice = i / kSlice, lane = i % kSlice;
    const double* n = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
    const int base = __ldg(a.A.sl_ptr + slice) + lane;
    const int rl = __ldg(a.A.rlen + i);
    double gpx = 0.0, gpy = 0.0;
    double gnx[AVIP_MAX_SPECIES], gny[AVIP_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) gnx[s] = gny[s] = 0.0;
    // neighbours in groups of kG: the column and weight loads of a group are issued together,
    // then its potential and density gathers, then the sums (in slot order, as one at a time)
    constexpr int kG = 4;
    for (int k0 = 0; k0 < rl; k0 += kG) {
      int c[kG];
      double wx[kG], wy[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int e = base + (k0 + u) * kSlice;
        const bool in = k0 + u < rl;
        c[u] = in ? __ldg(a.A.col + e) : i;
        wx[u] = in ? __ldg(a.A.gx + e) : 0.0;
        wy[u] = in ? __ldg(a.A.gy + e) : 0.0;
      }
      double pj[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) pj[u] = a.phi[c[u]];
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        if (k0 + u < rl) {
          gpx = fma(wx[u], pj[u], gpx);
          gpy = fma(wy[u], pj[u], gpy);
        }
      }
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
        if (s < ns) {
          double uj[kG];
#pragma unroll
          for (int u = 0; u < kG; ++u) uj[u] = n[(size_t)s * a.Npad + c[u]];
#pragma unroll
          for (int u = 0; u < kG; ++u) {
            if (k0 + u < rl) {
              gnx[s] = fma(wx[u], uj[u], gnx[s]);
              gny[s] = fma(wy[u], uj[u], gny[s]);
            }
          }
        }
      }
    }
    const double Ex = -gpx, Ey = -gpy;
    // |E| and 1/|E| from one reciprocal square root (the Townsend and attachment exponents take
    // -B/|E| as a product)
    const double E2 = Ex * Ex + Ey * Ey;
    const double invE = E2 > 0.0 ? rsqrt(E2) : 0.0;
    const double Emag = E2 * invE;
    a.Ex[i] = Ex;
    a.Ey[i] = Ey;
    double mu[AVIP_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
      if (s < ns) {
        const SpeciesParams& sp = a.ph.sp[s];
        mu[s] = mobility(sp, Emag);
        const double sg = sp.q > 0 ? 1.0 : -1.0;
        const double vx = sg * mu[s] * Ex, vy = sg * mu[s] * Ey;
        double2* d = reinterpret_cast<double2*>(a.ndat + ((size_t)s * a.Npad + i) * 4);
        d[0] = make_double2(gnx[s], gny[s]);
        d[1] = make_double2(vx, vy);
        a.nm[(size_t)s * a.Npad + i] = n[(size_t)s * a.Npad + i] * mu[s];
      }
    }
    double src[AVIP_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) src[s] = 0.0;
    if (a.ph.src_model != AVIP_SRC_NONE) {
      const int ie = a.ph.src_idx[0], ip = a.ph.src_idx[1], ineg = a.ph.src_idx[2];
      const double ne = n[(size_t)ie * a.Npad + i];
      const double alpha = Emag > 0.0 ? a.ph.src_params[0] * exp_fp64(-a.ph.src_params[1] * invE) : 0.0;
      double mue = 0.0;
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s)
        if (s == ie) mue = mu[s];
      const double ion = alpha * mue * Emag * ne;
      if (a.ph.photo_terms > 0) a.photo_I[i] = ion;
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
        if (s == ie) src[s] += ion;
        if (s == ip) src[s] += ion;
      }
      if (a.ph.src_model == AVIP_SRC_TOWNSEND_ATTACH) {
        const double att = a.ph.src_params[2] * ne;
#pragma unroll
        for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
          if (s == ie) src[s] -= att;
          if (s == ineg) src[s] += att;
        }
      } else if (a.ph.src_model == AVIP_SRC_MORROW_LOWKE) {
        // attachment eta(|E|) w n_e, recombination beta_r n_e n_p and beta_r n_n n_p
        double npos = 0.0, nneg = 0.0;
#pragma unroll
        for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
          if (s == ip) npos = n[(size_t)s * a.Npad + i];
          if (s == ineg) nneg = n[(size_t)s * a.Npad + i];
        }
        const double eta = Emag > 0.0 ? a.ph.src_params[2] * exp_fp64(-a.ph.src_params[3] * invE) : 0.0;
        const double att = eta * mue * Emag * ne;
        const double rep = a.ph.src_params[4] * ne * npos;
        const double rnp = a.ph.src_params[4] * nneg * npos;
#pragma unroll
        for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
          if (s == ie) src[s] = src[s] - att - rep;
          if (s == ip) src[s] = src[s] - rep - rnp;
          if (s == ineg) src[s] = src[s] + att - rnp;
        }
      }
      double se = 0.0;
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s)
        if (s == ie) se = src[s];
      if (se != 0.0) chem = a.ph.a_chem * fabs(ne) * recip_nr(fabs(se));
    }
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s)
      if (s < ns) a.src[(size_t)s * a.Npad + i] = src[s];
  }
  if (with_dt) block_min_to_global(chem, &a.sc->dt_bits);
}

__global__ void __launch_bounds__(kDDThreads, 3) node_fields_kernel(DDArgs a, int with_dt) {
  node_fields_body(a, with_dt, blockIdx.x);
}

// ------------------------------------------------------------------------ time step
// Convective and dielectric limits over cells (section "Time step computation"), with the cell
// velocity and conductivity the means of the n_v nodal values.  Each thread carries the largest
// |V_cell| / dx (the sum of the nodal velocities times the per-cell weight 1/(n_v dx)) and the
// largest conductivity over its cells and species, and divides once at the end:
// min_c cfl dx / |V| = cfl / max_c |V| / dx, likewise for the dielectric limit.  The Fourier
// limit, fourier dx^2 / D over cells and species, depends on the mesh only (ph.dt_fourier).
__device__ __forceinline__ void dt_cells_body(const DDArgs& a, int bid, int nblocks) {
  // the largest (|V_cell| / dx)^2 is carried instead of |V_cell| / dx, so that each thread
  // takes one square root at the end rather than one per cell and species (FP64 square roots
  // dominated this kernel's FP64 issue)
  double v2max = 0.0, smax = 0.0;
  const int ns = a.ph.ns;
  for (int c = bid * blockDim.x + threadIdx.x; c < a.T; c += nblocks * blockDim.x) {
    const int n0 = a.cell[c], n1 = a.cell[a.T + c], n2 = a.cell[2 * a.T + c];
    const int n3 = a.nvmax == 4 ? a.cell[3 * a.T + c] : -1;  // -1: triangle
    const bool quad = n3 >= 0;
    const double w = a.cw[c];
    const double w2 = w * w;
    const double inv_nv = quad ? 0.25 : (1.0 / 3.0);
    double sigma = 0.0;
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
      if (s < ns) {
        double vx, vy;
        if (a.ph.dd_fp32) {  // FP32 velocities, FP64 candidate and reduction
          const float* d = a.ndat32 + (size_t)s * a.Npad * 4;
          vx = (double)d[4 * n0 + 2] + (double)d[4 * n1 + 2] + (double)d[4 * n2 + 2];
          vy = (double)d[4 * n0 + 3] + (double)d[4 * n1 + 3] + (double)d[4 * n2 + 3];
          if (quad) {
            vx += (double)d[4 * n3 + 2];
            vy += (double)d[4 * n3 + 3];
          }
        } else {
          const double* d = a.ndat + (size_t)s * a.Npad * 4;
          vx = d[4 * n0 + 2] + d[4 * n1 + 2] + d[4 * n2 + 2];
          vy = d[4 * n0 + 3] + d[4 * n1 + 3] + d[4 * n2 + 3];
          if (quad) {
            vx += d[4 * n3 + 2];
            vy += d[4 * n3 + 3];
          }
        }
        v2max = fmax(v2max, (vx * vx + vy * vy) * w2);
        const double* nm = a.nm + (size_t)s * a.Npad;
        double cell = nm[n0] + nm[n1] + nm[n2];
        if (quad) cell += nm[n3];
        sigma += fabs(a.ph.sp[s].q * kECharge * cell);
      }
    }
    smax = fmax(smax, sigma * inv_nv);
  }
  double cand = a.ph.dt_fourier;
  if (v2max > 0.0) cand = fmin(cand, a.ph.cfl / sqrt(v2max));
  if (smax > 0.0) cand = fmin(cand, a.ph.a_diel * kEps0 / smax);
  block_min_to_global(cand, &a.sc->dt_bits);
}

__global__ void __launch_bounds__(kDDThreads) dt_cells_kernel(DDArgs a) { dt_cells_body(a, blockIdx.x, gridDim.x); }

// ------------------------------------------------------------------------ fluxes + update
struct EdgeEnd {
  double u, gx, gy, vx, vy, x, y;
};

// Bernoulli function B(x) = x / (e^x - 1) for x >= 0 (B(0) = 1; 0 once e^x overflows).
// B(-x) = x + B(x), so one expm1 gives both values without cancellation.
__device__ __forceinline__ double bernoulli_pos(double x) { return x != 0.0 ? x / expm1(x) : 1.0; }

// Geometry of one edge for the Scharfetter-Gummel split (species independent), canonical
// orientation lo -> hi: unit direction e, length h, s = S.e and S_perp = S - s e.
struct SgGeo {
  double ex, ey, h, rh, s, spx, spy;
};
__device__ __forceinline__ SgGeo sg_geometry(double dx, double dy, double Sx, double Sy) {
  SgGeo g;
  g.h = sqrt(dx * dx + dy * dy);
  g.rh = 1.0 / g.h;
  g.ex = dx * g.rh;
  g.ey = dy * g.rh;
  g.s = Sx * g.ex + Sy * g.ey;
  g.spx = Sx - g.s * g.ex;
  g.spy = Sy - g.s * g.ey;
  return g;
}

// Scharfetter-Gummel flux (section "Scharfetter Gummel scheme"): S is split along the edge
// direction e into S_par = (S.e) e and S_perp; the tangential part is the exponentially fitted
// V.S_par (u_hi - e^a u_lo)/(1 - e^a), a = h V.e / D, evaluated as
// (D (S.e)/h)(B(-a) u_lo - B(a) u_hi) (no overflow for large |a|, no 0/0 at a = 0; D = 0 is
// the upwind limit); the normal part is centred: V.S_perp (u_lo + u_hi)/2 - D g.S_perp.
__device__ __forceinline__ double sg_flux(double ulo, double uhi, const SgGeo& G, double Vx, double Vy, double gx,
                                          double gy, double D) {
  const double Vt = Vx * G.ex + Vy * G.ey;
  double fpar;
  if (D > 0.0) {
    const double a = G.h * Vt / D;
    const double aa = fabs(a);
    const double Bp = bernoulli_pos(aa), Bm = aa + Bp;  // B(|a|), B(-|a|)
    const double B_neg_a = a >= 0.0 ? Bm : Bp, B_a = a >= 0.0 ? Bp : Bm;
    fpar = (D * G.s * G.rh) * (B_neg_a * ulo - B_a * uhi);
  } else {
    fpar = G.s * (fmax(Vt, 0.0) * ulo + fmin(Vt, 0.0) * uhi);
  }
  const double fperp = (Vx * G.spx + Vy * G.spy) * (0.5 * (ulo + uhi)) - D * (gx * G.spx + gy * G.spy);
  return fpar + fperp;
}

// Flux from `lo` to `hi` through the dual face with normal (Sx, Sy) oriented lo -> hi:
// limited Lax-Wendroff convective part with a virtual upwind node plus central diffusion, or
// (sg != nullptr) the Scharfetter-Gummel flux.
//
// The edge means V_ij = (V_i + V_j)/2 and grad_ij = (grad_i + grad_j)/2 are kept as sums and the
// halves folded into the products that use them: scaling by a power of two is exact in floating
// point, so this adds no rounding, for four FP64 multiplications fewer per edge and species (the
// FP64 issue rate bounds this kernel on GB300).
__device__ __forceinline__ double edge_flux(const EdgeEnd& lo, const EdgeEnd& hi, double Sx, double Sy,
                                            double D, double dt, double beta, int lim, const SgGeo* sg) {
  if (sg)
    return sg_flux(lo.u, hi.u, *sg, 0.5 * (lo.vx + hi.vx), 0.5 * (lo.vy + hi.vy), 0.5 * (lo.gx + hi.gx),
                   0.5 * (lo.gy + hi.gy), D);
  const double sVx = lo.vx + hi.vx, sVy = lo.vy + hi.vy;  // 2 V_ij
  const double sgx = lo.gx + hi.gx, sgy = lo.gy + hi.gy;  // 2 grad_ij
  const double av = 0.5 * (sVx * Sx + sVy * Sy);          // V_ij . S
  const bool up_lo = av >= 0.0;
  const EdgeEnd& U = up_lo ? lo : hi;
  const EdgeEnd& W = up_lo ? hi : lo;
  const double delta = W.u - U.u;
  double psi = 0.0;
  if (delta != 0.0) {
    const double dx = W.x - U.x, dy = W.y - U.y;
    // the ratio of the upwind to the local difference
    const double r = (2.0 * (U.gx * dx + U.gy * dy) - delta) * recip_nr(delta);
    psi = (lim == AVIP_LIM_SWEBY && beta == 1.0) ? fmax(0.0, fmin(r, 1.0))  // min-mod: the same value
                                                 : limiter(r, beta, lim);
  }
  const double lw = 0.5 * delta - (0.125 * dt) * (sgx * sVx + sgy * sVy);  // delta/2 - dt/2 grad_ij.V_ij
  const double fc = (U.u + lw * psi) * av;
  const double fd = -(0.5 * D) * (sgx * Sx + sgy * Sy);                    // -D grad_ij.S
  return fc + fd;
}

// kGather: the edge fluxes were evaluated once per edge (edge_flux_kernel) and are gathered;
// otherwise every row evaluates its own edges (batches).  Specialised so that the single-instance
// kernel carries none of the per-row evaluation's registers.
template <bool kGather>
__device__ __forceinline__ void flux_update_body_t(const DDArgs& a, int bid) {
  const int i = bid * blockDim.x + threadIdx.x;
  const int N = a.A.N;
  const int ns = a.ph.ns;
  const double dt = a.ph.dt_fixed > 0.0 ? a.ph.dt_fixed : __longlong_as_double((long long)a.sc->dt_bits);
  double qsum = 0.0;
  if (i < N) {
    const int par = a.sc->parity;
    const double* n = a.nbuf + (size_t)par * AVIP_MAX_SPECIES * a.Npad;
    double* nn = a.nbuf + (size_t)(par ^ 1) * AVIP_MAX_SPECIES * a.Npad;
    const int slice = i / kSlice, lane = i % kSlice;
    const int base = __ldg(a.A.sl_ptr + slice) + lane;
    const int rl = __ldg(a.flen + i);  // edge slots only
    const double xi = a.x[i], yi = a.y[i];
    double R[AVIP_MAX_SPECIES];
    EdgeEnd me[AVIP_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
      R[s] = 0.0;
      if (s < ns) {
        const double2* d = reinterpret_cast<const double2*>(a.ndat + ((size_t)s * a.Npad + i) * 4);
        const double2 g = d[0], v = d[1];
        me[s] = EdgeEnd{n[(size_t)s * a.Npad + i], g.x, g.y, v.x, v.y, xi, yi};
      }
    }
    if (kGather) {
      // fluxes already evaluated once per edge (lo -> hi), gathered in the same slot order: the
      // edge ids of kG slots are loaded together, then their fluxes, then summed in slot order
      constexpr int kG = 4;
      for (int k0 = 1; k0 < rl; k0 += kG) {
        int32_t v[kG];
#pragma unroll
        for (int u = 0; u < kG; ++u) v[u] = k0 + u < rl ? __ldg(a.slot_eid + base + (k0 + u) * kSlice) : 0;
#pragma unroll
        for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
          if (s < ns) {
            double F[kG];
#pragma unroll
            for (int u = 0; u < kG; ++u) F[u] = k0 + u < rl ? a.eflux[(size_t)s * a.E + (v[u] & 0x7fffffff)] : 0.0;
#pragma unroll
            for (int u = 0; u < kG; ++u)
              if (k0 + u < rl) R[s] = v[u] >= 0 ? R[s] - F[u] : R[s] + F[u];
          }
        }
      }
    }
    for (int k = 1; k < (kGather ? 0 : rl); ++k) {
      const int e = base + k * kSlice;
      const int j = __ldg(a.A.col + e);
      const double Sx = __ldg(a.A.sx + e), Sy = __ldg(a.A.sy + e);
      const bool lo_is_me = i < j;
      const double xj = a.x[j], yj = a.y[j];
      SgGeo geo;
      const bool use_sg = a.ph.scheme == AVIP_FLUX_SG;
      if (use_sg)  // canonical lo -> hi, like the flux itself
        geo = lo_is_me ? sg_geometry(xj - xi, yj - yi, Sx, Sy) : sg_geometry(xi - xj, yi - yj, -Sx, -Sy);
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
        if (s < ns) {
          const double2* d = reinterpret_cast<const double2*>(a.ndat + ((size_t)s * a.Npad + j) * 4);
          const double2 g = d[0], v = d[1];
          const EdgeEnd other{n[(size_t)s * a.Npad + j], g.x, g.y, v.x, v.y, xj, yj};
          const EdgeEnd& lo = lo_is_me ? me[s] : other;
          const EdgeEnd& hi = lo_is_me ? other : me[s];
          // the stored normal is oriented i -> j; the canonical one lo -> hi
          const double sgn = lo_is_me ? 1.0 : -1.0;
          const double F = edge_flux(lo, hi, sgn * Sx, sgn * Sy, a.ph.sp[s].D, dt, a.ph.beta, a.ph.limiter,
                                     use_sg ? &geo : nullptr);
          R[s] = lo_is_me ? R[s] - F : R[s] + F;
        }
      }
    }
    // boundary closure through the boundary nodal normal kept in the diagonal slot
    const double Sbx = __ldg(a.A.sx + base), Sby = __ldg(a.A.sy + base);
    const double Vi = a.vol[i], iVi = a.ivol[i];
    bool bad = false;
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
      if (s < ns) {
        const SpeciesParams& sp = a.ph.sp[s];
        double Fx = me[s].u * me[s].vx, Fy = me[s].u * me[s].vy;
        if (sp.bnd_mode == AVIP_BND_OUTFLOW) {
          Fx -= sp.D * me[s].gx;
          Fy -= sp.D * me[s].gy;
        }
        const double rs = R[s] - (Fx * Sbx + Fy * Sby);
        const double un = me[s].u + dt * fma(rs, iVi, a.src[(size_t)s * a.Npad + i]);
        nn[(size_t)s * a.Npad + i] = un;
        bad |= !isfinite(un);
        qsum += sp.q * (Vi * un);
      }
    }
    if (bad) atomicCAS(&a.sc->status, AVIP_OK, AVIP_ENAN);
  }
  // per-block charge partial (fixed order)
  __shared__ double sm[32];
  const int ln = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qsum += __shfl_xor_sync(0xffffffffu, qsum, o);
  if (ln == 0) sm[warp] = qsum;
  __syncthreads();
  if (warp == 0) {
    double t = ln < nw ? sm[ln] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (ln == 0) a.partials[bid] = t;
  }
  if (bid == 0 && threadIdx.x == 0) a.sc->dt = dt;
}

template <bool kGather>
__global__ void __launch_bounds__(kDDThreads, kGather ? 3 : 2) flux_update_kernel(DDArgs a) {
  flux_update_body_t<kGather>(a, blockIdx.x);
}

// One thread per edge (lo, hi): the flux of every species from lo to hi through the edge's dual
// face, the same function of the same operands as in flux_update_body's per-row evaluation, so
// both ends receive identical values.
__global__ void __launch_bounds__(kDDThreads) edge_flux_kernel(DDArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.E) return;
  const int ns = a.ph.ns;
  const double dt = a.ph.dt_fixed > 0.0 ? a.ph.dt_fixed : __longlong_as_double((long long)a.sc->dt_bits);
  const double* n = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
  const int lo = __ldg(a.e_lo + e), hi = __ldg(a.e_hi + e);
  const double Sx = __ldg(a.e_sx + e), Sy = __ldg(a.e_sy + e);
  const double xl = a.x[lo], yl = a.y[lo], xh = a.x[hi], yh = a.y[hi];
  const bool use_sg = a.ph.scheme == AVIP_FLUX_SG;
  SgGeo geo;
  if (use_sg) geo = sg_geometry(xh - xl, yh - yl, Sx, Sy);
#pragma unroll
  for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
    if (s < ns) {
      const double2* dl = reinterpret_cast<const double2*>(a.ndat + ((size_t)s * a.Npad + lo) * 4);
      const double2* dh = reinterpret_cast<const double2*>(a.ndat + ((size_t)s * a.Npad + hi) * 4);
      const double2 gl = dl[0], vl = dl[1], gh = dh[0], vh = dh[1];
      const EdgeEnd L{n[(size_t)s * a.Npad + lo], gl.x, gl.y, vl.x, vl.y, xl, yl};
      const EdgeEnd H{n[(size_t)s * a.Npad + hi], gh.x, gh.y, vh.x, vh.y, xh, yh};
      a.eflux[(size_t)s * a.E + e] =
          edge_flux(L, H, Sx, Sy, a.ph.sp[s].D, dt, a.ph.beta, a.ph.limiter, use_sg ? &geo : nullptr);
    }
  }
}

// Single block: charge in block order, time, parity, statistics; re-arm the dt minimum.
__device__ __forceinline__ void finalize_body(DevScalars* sc, const double* partials, int nparts) {
  __shared__ double sm[32];
  double t = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) t += partials[b];
  const int ln = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (ln == 0) sm[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double q = 0.0;
    for (int w = 0; w < nw; ++w) q += sm[w];
    sc->charge = kECharge * q;
    const double dt = sc->dt;
    if (!(dt > 0.0) || !isfinite(dt)) {
      if (sc->status == AVIP_OK) sc->status = AVIP_ENAN;
    }
    sc->t += dt;
    sc->parity ^= 1;
    sc->run_steps += 1;
    sc->run_iters_total += sc->pcg_iters;
    sc->run_iters_max = max(sc->run_iters_max, sc->pcg_iters);
    sc->run_dt_min = fmin(sc->run_dt_min, dt);
    sc->run_dt_max = fmax(sc->run_dt_max, dt);
    sc->run_relres_max = fmax(sc->run_relres_max, sc->pcg_relres);
    sc->dt_bits = (unsigned long long)__double_as_longlong(INFINITY);
  }
}

// Photoionisation (after the Helmholtz solves): S_ph = sum_j S_ph,j added to the electron and
// positive-ion sources, and the chemical time-step limit with the complete electron source.
__global__ void __launch_bounds__(kDDThreads) photo_add_kernel(DDArgs a, int with_dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double chem = INFINITY;
  if (i < a.A.N) {
    double S = 0.0;
    for (int j = 0; j < a.ph.photo_terms; ++j) S += a.photo_psi[(size_t)j * a.Npad + i];
    a.photo_S[i] = S;
    const int ie = a.ph.src_idx[0], ip = a.ph.src_idx[1];
    const double se = a.src[(size_t)ie * a.Npad + i] + S;
    a.src[(size_t)ie * a.Npad + i] = se;
    a.src[(size_t)ip * a.Npad + i] += S;
    if (with_dt && se != 0.0) {
      const double* n = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
      chem = a.ph.a_chem * fabs(n[(size_t)ie * a.Npad + i]) * recip_nr(fabs(se));
    }
  }
  if (with_dt) block_min_to_global(chem, &a.sc->dt_bits);
}

__global__ void finalize_kernel(DevScalars* sc, const double* partials, int nparts) {
  finalize_body(sc, partials, nparts);
}

__global__ void run_reset_kernel(DevScalars* sc) {
  sc->run_steps = 0;
  sc->run_iters_total = 0;
  sc->run_iters_max = 0;
  sc->run_dt_min = INFINITY;
  sc->run_dt_max = 0.0;
  sc->run_relres_max = 0.0;
  sc->status = AVIP_OK;
}


// ------------------------------------------------------------------------ FP32 forms
// Mixed precision (ph.dd_fp32): gradients, velocities, sources and fluxes in FP32 with FP32
// accumulation; the density state, the explicit update n += dt (R/V + S), the time-step
// candidates and reduction and the charge sum stay FP64.  Two differences are formed in FP64
// before rounding, because FP32 cannot resolve them from the absolute values: the potential
// differences phi_k - phi_i of the gradient (phi ~ 1e4 V varies by ~10 V between neighbours,
// so E from absolute values would lose 4 digits), using sum_k G_ik = 0 (each cell's nodal
// normals sum to zero), and the edge vectors x_j - x_i (coordinates ~1e-2 m, edges ~1e-5 m).
__device__ __forceinline__ float mobility32(const SpeciesParams& sp, float Emag) {
  if (sp.mob_model == AVIP_MOB_POWER)
    return (float)sp.mob[0] * powf(fmaxf(Emag, (float)sp.mob[3]) / (float)sp.mob[1], (float)sp.mob[2]);
  return (float)sp.mob[0];
}

__device__ __forceinline__ float limiter32(float r, float beta, int kind) {
  if (kind == AVIP_LIM_VANLEER) return (r + fabsf(r)) / (1.0f + fabsf(r));
  return fmaxf(0.0f, fmaxf(fminf(beta * r, 1.0f), fminf(r, beta)));
}

__device__ __forceinline__ void node_fields32_body(const DDArgs& a, int with_dt, int bid) {
  const int i = bid * blockDim.x + threadIdx.x;
  const int N = a.A.N;
  const int ns = a.ph.ns;
  double chem = INFINITY;
  if (i < N) {
    const int slice = i / kSlice, lane = i % kSlice;
    const double* n = a.nbuf + (size_t)a.sc->parity * AVIP_MAX_SPECIES * a.Npad;
    const int base = __ldg(a.A.sl_ptr + slice) + lane;
    const int rl = __ldg(a.A.rlen + i);
    const double phii = a.phi[i];
    float ui[AVIP_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) ui[s] = s < ns ? (float)n[(size_t)s * a.Npad + i] : 0.0f;
    float gpx = 0.0f, gpy = 0.0f;
    float gnx[AVIP_MAX_SPECIES], gny[AVIP_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) gnx[s] = gny[s] = 0.0f;
    for (int k = 1; k < rl; ++k) {  // slot 0 is the row itself: zero difference
      const int e = base + k * kSlice;
      const int j = __ldg(a.A.col + e);
      const float wx = __ldg(a.gx32 + e), wy = __ldg(a.gy32 + e);
      const float dp = (float)(a.phi[j] - phii);
      gpx = fmaf(wx, dp, gpx);
      gpy = fmaf(wy, dp, gpy);
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
        if (s < ns) {
          const float du = (float)n[(size_t)s * a.Npad + j] - ui[s];
          gnx[s] = fmaf(wx, du, gnx[s]);
          gny[s] = fmaf(wy, du, gny[s]);
        }
      }
    }
    const float Ex = -gpx, Ey = -gpy;
    const float Emag = sqrtf(Ex * Ex + Ey * Ey);
    a.Ex[i] = Ex;
    a.Ey[i] = Ey;
    float mu[AVIP_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
      if (s < ns) {
        const SpeciesParams& sp = a.ph.sp[s];
        mu[s] = mobility32(sp, Emag);
        const float sg = sp.q > 0 ? 1.0f : -1.0f;
        reinterpret_cast<float4*>(a.ndat32)[(size_t)s * a.Npad + i] =
            make_float4(gnx[s], gny[s], sg * mu[s] * Ex, sg * mu[s] * Ey);
        a.nm[(size_t)s * a.Npad + i] = n[(size_t)s * a.Npad + i] * (double)mu[s];
      } else {
        mu[s] = 0.0f;
      }
    }
    float src[AVIP_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) src[s] = 0.0f;
    if (a.ph.src_model != AVIP_SRC_NONE) {
      const int ie = a.ph.src_idx[0], ip = a.ph.src_idx[1], ineg = a.ph.src_idx[2];
      const float ne = (float)n[(size_t)ie * a.Npad + i];
      const float alpha = Emag > 0.0f ? (float)a.ph.src_params[0] * expf(-(float)a.ph.src_params[1] / Emag) : 0.0f;
      float mue = 0.0f;
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s)
        if (s == ie) mue = mu[s];
      const float ion = alpha * mue * Emag * ne;
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
        if (s == ie) src[s] += ion;
        if (s == ip) src[s] += ion;
      }
      if (a.ph.src_model == AVIP_SRC_TOWNSEND_ATTACH) {
        const float att = (float)a.ph.src_params[2] * ne;
#pragma unroll
        for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
          if (s == ie) src[s] -= att;
          if (s == ineg) src[s] += att;
        }
      } else if (a.ph.src_model == AVIP_SRC_MORROW_LOWKE) {
        float npos = 0.0f, nneg = 0.0f;
#pragma unroll
        for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
          if (s == ip) npos = (float)n[(size_t)s * a.Npad + i];
          if (s == ineg) nneg = (float)n[(size_t)s * a.Npad + i];
        }
        const float eta =
            Emag > 0.0f ? (float)a.ph.src_params[2] * expf(-(float)a.ph.src_params[3] / Emag) : 0.0f;
        const float att = eta * mue * Emag * ne;
        const float br = (float)a.ph.src_params[4];
        const float rep = br * ne * npos;
        const float rnp = br * nneg * npos;
#pragma unroll
        for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
          if (s == ie) src[s] = src[s] - att - rep;
          if (s == ip) src[s] = src[s] - rep - rnp;
          if (s == ineg) src[s] = src[s] + att - rnp;
        }
      }
      float se = 0.0f;
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s)
        if (s == ie) se = src[s];
      // chemical time-step candidate in FP64 (part of the time-step reduction)
      if (se != 0.0f) chem = a.ph.a_chem * fabs(n[(size_t)ie * a.Npad + i]) / fabs((double)se);
    }
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s)
      if (s < ns) a.src[(size_t)s * a.Npad + i] = src[s];
  }
  if (with_dt) block_min_to_global(chem, &a.sc->dt_bits);
}

__global__ void __launch_bounds__(kDDThreads) node_fields32_kernel(DDArgs a, int with_dt) {
  node_fields32_body(a, with_dt, blockIdx.x);
}

struct EdgeEnd32 {
  float u, gx, gy, vx, vy;
};

// FP32 edge flux lo -> hi through (Sx, Sy) oriented lo -> hi; (dx, dy) = x_hi - x_lo.
__device__ __forceinline__ float edge_flux32(const EdgeEnd32& lo, const EdgeEnd32& hi, float dx, float dy, float Sx,
                                             float Sy, float D, float dt, float beta, int lim, int scheme) {
  const float Vx = 0.5f * (lo.vx + hi.vx), Vy = 0.5f * (lo.vy + hi.vy);
  const float gx = 0.5f * (lo.gx + hi.gx), gy = 0.5f * (lo.gy + hi.gy);
  if (scheme == AVIP_FLUX_SG) {
    const float h = sqrtf(dx * dx + dy * dy);
    const float rh = 1.0f / h;
    const float ex = dx * rh, ey = dy * rh;
    const float s = Sx * ex + Sy * ey;
    const float spx = Sx - s * ex, spy = Sy - s * ey;
    const float Vt = Vx * ex + Vy * ey;
    float fpar;
    if (D > 0.0f) {
      const float aa = h * Vt / D, ab = fabsf(aa);
      const float Bp = ab != 0.0f ? ab / expm1f(ab) : 1.0f, Bm = ab + Bp;  // B(|a|), B(-|a|)
      fpar = (D * s * rh) * ((aa >= 0.0f ? Bm : Bp) * lo.u - (aa >= 0.0f ? Bp : Bm) * hi.u);
    } else {
      fpar = s * (fmaxf(Vt, 0.0f) * lo.u + fminf(Vt, 0.0f) * hi.u);
    }
    return fpar + (Vx * spx + Vy * spy) * (0.5f * (lo.u + hi.u)) - D * (gx * spx + gy * spy);
  }
  const float av = Vx * Sx + Vy * Sy;
  const bool up_lo = av >= 0.0f;
  const EdgeEnd32& U = up_lo ? lo : hi;
  const float delta = (up_lo ? hi.u : lo.u) - U.u;
  float psi = 0.0f;
  if (delta != 0.0f) {
    const float ux = up_lo ? dx : -dx, uy = up_lo ? dy : -dy;  // x_W - x_U
    const float r = (2.0f * (U.gx * ux + U.gy * uy) - delta) / delta;
    psi = limiter32(r, beta, lim);
  }
  const float lw = 0.5f * delta - 0.5f * dt * (gx * Vx + gy * Vy);
  return (U.u + lw * psi) * av - D * (gx * Sx + gy * Sy);
}

__device__ __forceinline__ void flux_update32_body(const DDArgs& a, int bid) {
  const int i = bid * blockDim.x + threadIdx.x;
  const int N = a.A.N;
  const int ns = a.ph.ns;
  const double dt = a.ph.dt_fixed > 0.0 ? a.ph.dt_fixed : __longlong_as_double((long long)a.sc->dt_bits);
  const float dtf = (float)dt, betaf = (float)a.ph.beta;
  double qsum = 0.0;
  if (i < N) {
    const int par = a.sc->parity;
    const double* n = a.nbuf + (size_t)par * AVIP_MAX_SPECIES * a.Npad;
    double* nn = a.nbuf + (size_t)(par ^ 1) * AVIP_MAX_SPECIES * a.Npad;
    const float4* nd = reinterpret_cast<const float4*>(a.ndat32);
    const int slice = i / kSlice, lane = i % kSlice;
    const int base = __ldg(a.A.sl_ptr + slice) + lane;
    const int rl = __ldg(a.flen + i);  // edge slots only
    const double xi = a.x[i], yi = a.y[i];
    float R[AVIP_MAX_SPECIES];
    EdgeEnd32 me[AVIP_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
      R[s] = 0.0f;
      if (s < ns) {
        const float4 d = nd[(size_t)s * a.Npad + i];
        me[s] = EdgeEnd32{(float)n[(size_t)s * a.Npad + i], d.x, d.y, d.z, d.w};
      }
    }
    for (int k = 1; k < rl; ++k) {
      const int e = base + k * kSlice;
      const int j = __ldg(a.A.col + e);
      const float Sx = __ldg(a.sx32 + e), Sy = __ldg(a.sy32 + e);
      const bool lo_is_me = i < j;
      // canonical lo -> hi edge vector, formed in FP64 so that both ends round the same value
      const float dx = lo_is_me ? (float)(a.x[j] - xi) : (float)(xi - a.x[j]);
      const float dy = lo_is_me ? (float)(a.y[j] - yi) : (float)(yi - a.y[j]);
      const float cSx = lo_is_me ? Sx : -Sx, cSy = lo_is_me ? Sy : -Sy;
#pragma unroll
      for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
        if (s < ns) {
          const float4 d = nd[(size_t)s * a.Npad + j];
          const EdgeEnd32 other{(float)n[(size_t)s * a.Npad + j], d.x, d.y, d.z, d.w};
          const EdgeEnd32& lo = lo_is_me ? me[s] : other;
          const EdgeEnd32& hi = lo_is_me ? other : me[s];
          const float F = edge_flux32(lo, hi, dx, dy, cSx, cSy, (float)a.ph.sp[s].D, dtf, betaf, a.ph.limiter,
                                      a.ph.scheme);
          R[s] = lo_is_me ? R[s] - F : R[s] + F;
        }
      }
    }
    const float Sbx = __ldg(a.sx32 + base), Sby = __ldg(a.sy32 + base);
    const double Vi = a.vol[i];
    bool bad = false;
#pragma unroll
    for (int s = 0; s < AVIP_MAX_SPECIES; ++s) {
      if (s < ns) {
        const SpeciesParams& sp = a.ph.sp[s];
        float Fx = me[s].u * me[s].vx, Fy = me[s].u * me[s].vy;
        if (sp.bnd_mode == AVIP_BND_OUTFLOW) {
          Fx -= (float)sp.D * me[s].gx;
          Fy -= (float)sp.D * me[s].gy;
        }
        const float rs = R[s] - (Fx * Sbx + Fy * Sby);
        // FP64 update of the FP64 state
        const double un = n[(size_t)s * a.Npad + i] + dt * ((double)rs / Vi + a.src[(size_t)s * a.Npad + i]);
        nn[(size_t)s * a.Npad + i] = un;
        bad |= !isfinite(un);
        qsum += sp.q * (Vi * un);
      }
    }
    if (bad) atomicCAS(&a.sc->status, AVIP_OK, AVIP_ENAN);
  }
  __shared__ double sm[32];
  const int ln = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qsum += __shfl_xor_sync(0xffffffffu, qsum, o);
  if (ln == 0) sm[warp] = qsum;
  __syncthreads();
  if (warp == 0) {
    double t = ln < nw ? sm[ln] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (ln == 0) a.partials[bid] = t;
  }
  if (bid == 0 && threadIdx.x == 0) a.sc->dt = dt;
}

__global__ void __launch_bounds__(kDDThreads, 3) flux_update32_kernel(DDArgs a) { flux_update32_body(a, blockIdx.x); }

// ------------------------------------------------------------------------ batched forms
// One launch covers every instance of a batch: block b belongs to the instance k with
// bpref[k] <= b < bpref[k + 1] and runs that instance's block b - bpref[k].
__device__ __forceinline__ int batch_instance(const int32_t* __restrict__ bpref, int count, int b) {
  int lo = 0, hi = count;  // largest k with bpref[k] <= b
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(bpref + mid) <= b) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kDDThreads) node_fields_batch_kernel(const DDArgs* __restrict__ args,
                                                                        const int32_t* __restrict__ bpref, int count) {
  const int k = batch_instance(bpref, count, blockIdx.x);
  const DDArgs& a = args[k];
  if (a.ph.dd_fp32)
    node_fields32_body(a, a.ph.dt_fixed > 0.0 ? 0 : 1, blockIdx.x - __ldg(bpref + k));
  else
    node_fields_body(a, a.ph.dt_fixed > 0.0 ? 0 : 1, blockIdx.x - __ldg(bpref + k));
}
__global__ void __launch_bounds__(kDDThreads) dt_cells_batch_kernel(const DDArgs* __restrict__ args,
                                                                     const int32_t* __restrict__ bpref, int count) {
  const int k = batch_instance(bpref, count, blockIdx.x);
  const DDArgs& a = args[k];
  if (a.ph.dt_fixed > 0.0) return;
  dt_cells_body(a, blockIdx.x - __ldg(bpref + k), __ldg(bpref + k + 1) - __ldg(bpref + k));
}
// (one resident block per SM guaranteed: the per-row evaluation of every edge needs ~140
// registers, and a cap of 128 made it spill)
__global__ void __launch_bounds__(kDDThreads, 1) flux_update_batch_kernel(const DDArgs* __restrict__ args,
                                                                        const int32_t* __restrict__ bpref, int count) {
  const int k = batch_instance(bpref, count, blockIdx.x);
  if (args[k].ph.dd_fp32)
    flux_update32_body(args[k], blockIdx.x - __ldg(bpref + k));
  else
    flux_update_body_t<false>(args[k], blockIdx.x - __ldg(bpref + k));  // batches evaluate each edge per row
}
__global__ void finalize_batch_kernel(const DDArgs* __restrict__ args, int count, int threads) {
  const DDArgs& a = args[blockIdx.x];
  finalize_body(a.sc, a.partials, (a.A.N + threads - 1) / threads);
}
__global__ void run_reset_batch_kernel(const DDArgs* __restrict__ args, int count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  DevScalars* sc = args[k].sc;
  sc->run_steps = 0;
  sc->run_iters_total = 0;
  sc->run_iters_max = 0;
  sc->run_dt_min = INFINITY;
  sc->run_dt_max = 0.0;
  sc->run_relres_max = 0.0;
  sc->status = AVIP_OK;
}

// ------------------------------------------------------------------------ host launchers
static inline int nblk(int n) { return (n + kDDThreads - 1) / kDDThreads; }

cudaError_t launch_node_fields(const DDArgs& a, int with_dt, cudaStream_t st) {
  if (a.ph.dd_fp32)
    node_fields32_kernel<<<nblk(a.A.N), kDDThreads, 0, st>>>(a, with_dt);
  else
    node_fields_kernel<<<nblk(a.A.N), kDDThreads, 0, st>>>(a, with_dt);
  return cudaGetLastError();
}
cudaError_t launch_photo_add(const DDArgs& a, int with_dt, cudaStream_t st) {
  photo_add_kernel<<<nblk(a.A.N), kDDThreads, 0, st>>>(a, with_dt);
  return cudaGetLastError();
}

cudaError_t launch_dt_cells(const DDArgs& a, cudaStream_t st) {
  // a few cells per thread: 8 resident blocks on each of the 152 SMs
  const int blocks = nblk(a.T) < 152 * 8 ? nblk(a.T) : 152 * 8;
  dt_cells_kernel<<<blocks, kDDThreads, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_flux_update(const DDArgs& a, cudaStream_t st) {
  if (a.ph.dd_fp32) {
    flux_update32_kernel<<<nblk(a.A.N), kDDThreads, 0, st>>>(a);
  } else {
    if (a.eflux && a.E > 0) {
      edge_flux_kernel<<<nblk(a.E), kDDThreads, 0, st>>>(a);
      flux_update_kernel<true><<<nblk(a.A.N), kDDThreads, 0, st>>>(a);
    } else {
      flux_update_kernel<false><<<nblk(a.A.N), kDDThreads, 0, st>>>(a);
    }
  }
  return cudaGetLastError();
}
cudaError_t launch_finalize(DevScalars* sc, const double* partials, int nparts, cudaStream_t st) {
  finalize_kernel<<<1, 256, 0, st>>>(sc, partials, nparts);
  return cudaGetLastError();
}
cudaError_t launch_run_reset(DevScalars* sc, cudaStream_t st) {
  run_reset_kernel<<<1, 1, 0, st>>>(sc);
  return cudaGetLastError();
}
// ------------------------------------------------------------------ checkpoint copies
// state_get: the device state in the caller's layout (one coalesced read per field, a scattered
// write to the caller positions); state_put: the reverse, after state_check has found every
// entry finite.  Values are copied, never recomputed, so a checkpoint round trip is exact.
__global__ void state_take_kernel(StateArgs s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t N = (size_t)s.N;
  const size_t hb = (size_t)(s.ns + 1) * N + 1;  // first predictor-history entry
  if (i == 0) {
    s.stage[(size_t)(s.ns + 1) * N] = s.sc->t;
    s.stage[hb + 3 * N] = (double)s.sc->phi_hist;
  }
  if (i >= s.N) return;
  const size_t c = (size_t)__ldg(s.perm + i);
  const double* n = s.nbuf + (size_t)s.sc->parity * AVIP_MAX_SPECIES * s.Npad;
  for (int k = 0; k < s.ns; ++k) s.stage[k * N + c] = n[(size_t)k * s.Npad + i];
  s.stage[s.ns * N + c] = s.phi[i];
  s.stage[hb + c] = s.phi1[i];
  s.stage[hb + N + c] = s.phi2[i];
  s.stage[hb + 2 * N + c] = s.phi3[i];
}
__global__ void state_check_kernel(StateArgs s) {
  const size_t total = (size_t)(s.ns + 4) * s.N + 2;
  bool bad = false;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(s.stage[k]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(s.flag, 1);
}
__global__ void state_put_kernel(StateArgs s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t N = (size_t)s.N;
  const size_t hb = (size_t)(s.ns + 1) * N + 1;
  if (i == 0) {
    s.sc->t = s.t;
    s.sc->phi_hist = s.hist;
  }
  if (i >= s.N) return;
  const size_t c = (size_t)__ldg(s.perm + i);
  double* n = s.nbuf + (size_t)s.sc->parity * AVIP_MAX_SPECIES * s.Npad;
  for (int k = 0; k < s.ns; ++k) n[(size_t)k * s.Npad + i] = s.stage[k * N + c];
  s.phi[i] = s.stage[s.ns * N + c];
  s.phi1[i] = s.stage[hb + c];
  s.phi2[i] = s.stage[hb + N + c];
  s.phi3[i] = s.stage[hb + 2 * N + c];
}
cudaError_t launch_state_take(const StateArgs& s, cudaStream_t st) {
  state_take_kernel<<<nblk(s.N), kDDThreads, 0, st>>>(s);
  return cudaGetLastError();
}
cudaError_t launch_state_check(const StateArgs& s, cudaStream_t st) {
  state_check_kernel<<<nblk(s.N), kDDThreads, 0, st>>>(s);
  return cudaGetLastError();
}
cudaError_t launch_state_put(const StateArgs& s, cudaStream_t st) {
  state_put_kernel<<<nblk(s.N), kDDThreads, 0, st>>>(s);
  return cudaGetLastError();
}

int flux_blocks(int N) { return nblk(N); }
// Charge partials a handle must hold: one per block at the smallest batched block size.
int flux_partials_max(int N) { return (N + kDDMinThreads - 1) / kDDMinThreads; }

// The drift-diffusion stages of a batch with `threads` threads per block (kDDMinThreads ..
// kDDThreads, a multiple of 32; the block prefix sums node_pref / cell_pref were made for it).
cudaError_t launch_dd_batch(const DDArgs* args, const int32_t* node_pref, const int32_t* cell_pref, int count,
                            int node_blocks, int cell_blocks, int threads, cudaStream_t st) {
  if (threads < kDDMinThreads || threads > kDDThreads || threads % 32) return cudaErrorInvalidValue;
  node_fields_batch_kernel<<<node_blocks, threads, 0, st>>>(args, node_pref, count);
  dt_cells_batch_kernel<<<cell_blocks, threads, 0, st>>>(args, cell_pref, count);
  flux_update_batch_kernel<<<node_blocks, threads, 0, st>>>(args, node_pref, count);
  finalize_batch_kernel<<<count, 256, 0, st>>>(args, count, threads);
  return cudaGetLastError();
}
cudaError_t launch_run_reset_batch(const DDArgs* args, int count, cudaStream_t st) {
  run_reset_batch_kernel<<<(count + 127) / 128, 128, 0, st>>>(args, count);
  return cudaGetLastError();
}
int dd_threads() { return kDDThreads; }

}  // namespace avip
