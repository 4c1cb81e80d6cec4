// Host set-up of a smoothed-aggregation algebraic multigrid (SA-AMG) hierarchy for the
// Poisson system, used as the preconditioner of the conjugate-gradient solve (solver kind 8).
//
// The matrix of a mesh never changes (only the right-hand side does, step after step), so the
// hierarchy is built once when the mesh is created and every step reuses it; the V-cycle runs
// on the device.  The paper does not name its linear solver; this is one more preconditioner
// for the same conjugate-gradient iteration on the same matrix (Eq. coeff_matriceA with the
// Dirichlet rows eliminated and the symmetric diagonal scaling of the Jacobi variant).
//
// Construction (smoothed aggregation of Vanek, Mandel and Brezina, written from its published
// description):
//   * strength of connection: |a_ij| >= theta sqrt(|a_ii a_jj|), theta = 0.08 (0, i.e. the matrix graph,
//     when no connection is strong: strongly diagonally dominant Helmholtz operators);
//   * aggregation in node order (Morton order keeps aggregates compact): a node whose strong
//     neighbours are all free starts an aggregate with them; remaining nodes join the
//     aggregate of their strongest aggregated neighbour; what is left forms aggregates with
//     its free strong neighbours.  Rows without strong connections (the decoupled Dirichlet
//     unit rows) get no coarse unknown: the smoother solves them exactly;
//   * tentative prolongator T from the near-null-space vector B (the scaled system maps the
//     constant potential to zero away from the boundary, so B = D^1/2 1 on the finest
//     level): T_ij = B_i / ||B restricted to aggregate j||, and B_coarse,j = that norm;
//   * smoothed prolongator P = (I - omega D^-1 A) T, omega = 4 / (3 lambda_max(D^-1 A)),
//     lambda_max from 30 power iterations (times 1.05);
//   * restriction R = P^T and Galerkin coarse matrix A_c = R A P (rounding symmetrised);
//   * smoother: one damped Jacobi step, from zero x = Q b and from a given x
//     x <- x + Q (b - A x), with Q = omega D^-1, omega = 1.7 / lambda_max(D^-1 A) (the same step
//     before and after the coarse correction, so the V-cycle stays symmetric; omega lambda_max
//     stays below the stability limit 2 with a margin for the estimate).  On the pin-plane
//     hierarchy it needs about as many CG iterations (24 to 1e-12 from zero, CPU emulation) as
//     a degree-2 Chebyshev smoother (22) with composite operators 2.4 times smaller (below);
//   * composite operators, so that the V-cycle needs two grid-wide phases per level instead of
//     six: with xp = Q b,
//         b' = R (b - A xp)                 = Rf b,   Rf = R (I - A Q)
//         x  = xp + P x' + Q (b - A (xp + P x'))
//            = (2 I - Q A) xp + (I - Q A) P x' = U xp + Pf x'
//     (the same V-cycle in exact arithmetic; for a symmetric A, Rf = Pf^T exactly; U has the
//     sparsity of A, Pf that of P widened by one ring);
//   * levels until at most N/64 unknowns remain (clamped to [256, 1500]: a larger dense coarse
//     level saves barriers per V-cycle on big meshes, a smaller one keeps the O(n^3) set-up of
//     small meshes cheap), where the coarse matrix is inverted
//     densely (Cholesky; Gauss-Jordan with partial pivoting for the non-symmetric matrix of
//     the axisymmetric configuration) and applied as a dense product.
// The same construction serves the axisymmetric matrix (mildly non-symmetric; it also maps the
// constant potential to zero), preconditioning BiCGStab there (solver kind 9).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <thread>
#include <utility>

#include "avip_internal.h"

namespace avip {

namespace {

constexpr double kTheta = 0.08;
constexpr double kJacobiOmega = 1.7;  // omega = kJacobiOmega / lambda_max(D^-1 A)
constexpr int kCoarseMin = 256, kCoarseMax = 1500;

// y = A x (CSR)
void csr_mv(const Csr& A, const std::vector<double>& x, std::vector<double>& y) {
  y.assign(A.n, 0.0);
  for (int32_t i = 0; i < A.n; ++i) {
    double s = 0.0;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) s += A.v[e] * x[A.ci[e]];
    y[i] = s;
  }
}

Csr transpose(const Csr& A) {
  Csr T;
  T.n = A.m;
  T.m = A.n;
  T.rp.assign(T.n + 1, 0);
  for (int32_t e = 0; e < A.rp[A.n]; ++e) T.rp[A.ci[e] + 1]++;
  for (int32_t i = 0; i < T.n; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.rp[A.n]);
  T.v.resize(A.rp[A.n]);
  std::vector<int32_t> fill(T.rp.begin(), T.rp.end() - 1);
  for (int32_t i = 0; i < A.n; ++i)
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
      const int32_t k = fill[A.ci[e]]++;
      T.ci[k] = i;  // rows visited in order: each row of T comes out sorted
      T.v[k] = A.v[e];
    }
  return T;
}

// C = A B (row by row with a dense accumulator); columns of each row sorted
Csr spgemm(const Csr& A, const Csr& B) {
  Csr C;
  C.n = A.n;
  C.m = B.m;
  C.rp.assign(C.n + 1, 0);
  std::vector<double> acc(B.m, 0.0);
  std::vector<int32_t> mark(B.m, -1), cols;
  for (int32_t i = 0; i < A.n; ++i) {
    cols.clear();
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
      const int32_t k = A.ci[e];
      const double a = A.v[e];
      for (int32_t f = B.rp[k]; f < B.rp[k + 1]; ++f) {
        const int32_t j = B.ci[f];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] += a * B.v[f];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t j : cols) {
      C.ci.push_back(j);
      C.v.push_back(acc[j]);
    }
    C.rp[i + 1] = (int32_t)C.ci.size();
  }
  return C;
}

double diag_of(const Csr& A, int32_t i) {
  for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
    if (A.ci[e] == i) return A.v[e];
  return 0.0;
}

// largest eigenvalue of D^-1 A by power iteration (deterministic start vector)
double lambda_max(const Csr& A, const std::vector<double>& dinv) {
  std::vector<double> x(A.n), y;
  for (int32_t i = 0; i < A.n; ++i) x[i] = 1.0 + 0.37 * std::sin(1.7 * i + 0.3);
  double lam = 1.0;
  for (int it = 0; it < 30; ++it) {
    csr_mv(A, x, y);
    double nrm = 0.0, dot = 0.0, xx = 0.0;
    for (int32_t i = 0; i < A.n; ++i) {
      y[i] *= dinv[i];
      nrm += y[i] * y[i];
      dot += y[i] * x[i];
      xx += x[i] * x[i];
    }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0) || !(xx > 0)) break;
    lam = dot / xx;
    for (int32_t i = 0; i < A.n; ++i) x[i] = y[i] / nrm;
  }
  return std::max(lam, 1e-300) * 1.05;
}

// aggregate index per row (-1: no coarse unknown); returns the number of aggregates
int32_t aggregate(const Csr& A, std::vector<int32_t>& agg, double theta) {
  const int32_t n = A.n;
  std::vector<double> d(n);
  for (int32_t i = 0; i < n; ++i) d[i] = std::fabs(diag_of(A, i));
  auto strong = [&](int32_t i, int32_t e) {
    const int32_t j = A.ci[e];
    return j != i && A.v[e] != 0.0 && std::fabs(A.v[e]) >= theta * std::sqrt(d[i] * d[j]);
  };
  agg.assign(n, -2);  // -2 free, -1 isolated
  int32_t na = 0;
  for (int32_t i = 0; i < n; ++i) {
    bool any = false;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) any |= strong(i, e);
    if (!any) agg[i] = -1;
  }
  // pass 1: roots whose strong neighbourhood is entirely free
  for (int32_t i = 0; i < n; ++i) {
    if (agg[i] != -2) continue;
    bool free_nb = true;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1] && free_nb; ++e)
      if (strong(i, e) && agg[A.ci[e]] != -2) free_nb = false;
    if (!free_nb) continue;
    agg[i] = na;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
      if (strong(i, e)) agg[A.ci[e]] = na;
    ++na;
  }
  // pass 2: join the aggregate of the strongest aggregated neighbour
  std::vector<int32_t> join(n, -1);
  for (int32_t i = 0; i < n; ++i) {
    if (agg[i] != -2) continue;
    double best = 0.0;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
      if (strong(i, e) && agg[A.ci[e]] >= 0 && std::fabs(A.v[e]) > best) {
        best = std::fabs(A.v[e]);
        join[i] = agg[A.ci[e]];
      }
  }
  for (int32_t i = 0; i < n; ++i)
    if (agg[i] == -2 && join[i] >= 0) agg[i] = join[i];
  // pass 3: leftovers aggregate with their free strong neighbours
  for (int32_t i = 0; i < n; ++i) {
    if (agg[i] != -2) continue;
    agg[i] = na;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
      if (strong(i, e) && agg[A.ci[e]] == -2) agg[A.ci[e]] = na;
    ++na;
  }
  return na;
}

// Host threads for a dense set-up step of order n: one below 256 rows, else up to 16 (the
// hardware concurrency when it is known).
int host_threads(int n) {
  if (n < 256) return 1;
  const unsigned hc = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(16u, hc == 0 ? 1u : hc));
}

// dense inverse of an SPD matrix (row-major n x n) through its Cholesky factor
bool dense_spd_inverse(std::vector<double>& a, int n) {
  for (int j = 0; j < n; ++j) {  // a = L L^T, L in the lower triangle
    double s = a[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
    if (!(s > 0)) return false;
    const double ljj = std::sqrt(s);
    a[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = a[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= a[(size_t)i * n + k] * a[(size_t)j * n + k];
      a[(size_t)i * n + j] = t / ljj;
    }
  }
  // U = L^T stored by rows, so that both triangular solves walk memory contiguously
  std::vector<double> U((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k <= i; ++k) U[(size_t)k * n + i] = a[(size_t)i * n + k];
  std::vector<double> inv((size_t)n * n);
  // the columns are independent: spread them over the host cores (each column's arithmetic
  // does not depend on the thread that computes it)
  auto columns = [&](int first, int stride) {
    std::vector<double> y(n), x(n);
    for (int c = first; c < n; c += stride) {  // column c of the inverse: L y = e_c, L^T x = y
      // y_i = 0 for i < c exactly, so the forward solve starts at row c
      for (int i = 0; i < c; ++i) y[i] = 0.0;
      for (int i = c; i < n; ++i) {
        double t = (i == c) ? 1.0 : 0.0;
        const double* li = &a[(size_t)i * n];
        for (int k = c; k < i; ++k) t -= li[k] * y[k];
        y[i] = t / li[i];
      }
      for (int i = n - 1; i >= 0; --i) {
        double t = y[i];
        const double* ui = &U[(size_t)i * n];
        for (int k = i + 1; k < n; ++k) t -= ui[k] * x[k];
        x[i] = t / ui[i];
      }
      for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = x[i];
    }
  };
  const int nt = host_threads(n);
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(columns, t, nt);
  columns(0, nt);
  for (auto& th : pool) th.join();
  a.swap(inv);
  return true;
}

// dense inverse of a general matrix (row-major n x n) by Gauss-Jordan elimination with
// partial pivoting; false if singular
bool dense_inverse(std::vector<double>& a, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(a[(size_t)i * n + c]) > std::fabs(a[(size_t)piv * n + c])) piv = i;
    if (!(std::fabs(a[(size_t)piv * n + c]) > 0)) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)c * n + k], a[(size_t)piv * n + k]);
        std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
      }
    const double dinv = 1.0 / a[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      a[(size_t)c * n + k] *= dinv;
      inv[(size_t)c * n + k] *= dinv;
    }
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = a[(size_t)i * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)i * n + k] -= f * a[(size_t)c * n + k];
        inv[(size_t)i * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

// alpha I + beta M (M square; the diagonal entry is created where M has none)
Csr identity_plus(double alpha, double beta, const Csr& M) {
  Csr C;
  C.n = M.n;
  C.m = M.m;
  C.rp.assign(M.n + 1, 0);
  for (int32_t i = 0; i < M.n; ++i) {
    bool diag = false;
    for (int32_t e = M.rp[i]; e < M.rp[i + 1]; ++e) {
      const int32_t j = M.ci[e];
      if (!diag && j > i) {  // columns are sorted: insert the missing diagonal in place
        C.ci.push_back(i);
        C.v.push_back(alpha);
        diag = true;
      }
      double v = beta * M.v[e];
      if (j == i) {
        v += alpha;
        diag = true;
      }
      C.ci.push_back(j);
      C.v.push_back(v);
    }
    if (!diag) {
      C.ci.push_back(i);
      C.v.push_back(alpha);
    }
    C.rp[i + 1] = (int32_t)C.ci.size();
  }
  return C;
}

// Q = omega D^-1 (diagonal)
Csr smoother_matrix(const std::vector<double>& dinv, double omega) {
  Csr Q;
  Q.n = Q.m = (int32_t)dinv.size();
  Q.rp.resize(Q.n + 1);
  Q.ci.resize(Q.n);
  Q.v.resize(Q.n);
  for (int32_t i = 0; i < Q.n; ++i) {
    Q.rp[i] = i;
    Q.ci[i] = i;
    Q.v[i] = omega * dinv[i];
  }
  Q.rp[Q.n] = Q.n;
  return Q;
}

// Composite operators of level L (Q, Rf, U, Pf; see the header comment)
void composite_operators(AmgHostLevel& L, bool symmetric) {
  L.omega = kJacobiOmega / L.lmax;
  // the level matrix with sorted rows (the finest level keeps its diagonal first)
  Csr A = L.A;
  for (int32_t i = 0; i < A.n; ++i) {
    std::vector<std::pair<int32_t, double>> row;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) row.emplace_back(A.ci[e], A.v[e]);
    std::sort(row.begin(), row.end());
    for (size_t k = 0; k < row.size(); ++k) {
      A.ci[A.rp[i] + k] = row[k].first;
      A.v[A.rp[i] + k] = row[k].second;
    }
  }
  L.Q = smoother_matrix(L.dinv, L.omega);
  const Csr QA = spgemm(L.Q, A);
  L.U = identity_plus(2.0, -1.0, QA);
  L.Pf = spgemm(identity_plus(1.0, -1.0, QA), L.P);
  if (symmetric) {
    L.Rf = transpose(L.Pf);  // R (I - A Q) = ((I - Q A) P)^T when A and Q are symmetric
  } else {
    L.Rf = spgemm(L.R, identity_plus(1.0, -1.0, spgemm(A, L.Q)));
  }
}

}  // namespace

void sell_from_csr(const Csr& A, SellHost& S, int lpr) {
  const int rps = kSlice / lpr;  // rows per slice
  S.n = A.n;
  S.lpr = lpr;
  S.nslices = (A.n + rps - 1) / rps;
  S.rlen.assign((size_t)S.nslices * rps, 0);
  for (int32_t i = 0; i < A.n; ++i) S.rlen[i] = A.rp[i + 1] - A.rp[i];
  S.sl_ptr.assign(S.nslices + 1, 0);
  S.sl_w.assign(S.nslices, 0);
  int64_t off = 0;
  for (int32_t s = 0; s < S.nslices; ++s) {
    int32_t w = 0;
    for (int r = 0; r < rps; ++r) w = std::max(w, (S.rlen[(size_t)s * rps + r] + lpr - 1) / lpr);
    S.sl_w[s] = w;
    S.sl_ptr[s] = (int32_t)off;
    off += (int64_t)w * kSlice;
  }
  S.sl_ptr[S.nslices] = (int32_t)off;
  S.col.assign(off, 0);
  S.val.assign(off, 0.0);
  for (int32_t s = 0; s < S.nslices; ++s)
    for (int r = 0; r < rps; ++r) {
      const int32_t i = s * rps + r;
      if (i >= A.n) continue;
      for (int32_t k = 0; k < S.rlen[i]; ++k) {  // padding slots keep column 0 and value 0
        const int64_t e = (int64_t)S.sl_ptr[s] + (int64_t)(k / lpr) * kSlice + r * lpr + (k % lpr);
        S.col[e] = A.ci[A.rp[i] + k];
        S.val[e] = A.v[A.rp[i] + k];
      }
    }
}

int lanes_per_row(const Csr& A) {
  const double avg = A.n > 0 ? (double)A.rp[A.n] / A.n : 0.0;
  int lpr = 1;
  while (lpr < kSlice && avg > 8.0 * lpr) lpr *= 2;
  return lpr;
}

int amg_setup(const HostMesh& m, AmgHost& H, char* err, size_t errlen) {
  // the axisymmetric matrix is not symmetric: no symmetrisation, LU instead of Cholesky
  const bool symmetric = m.geometry != AVIP_GEOM_AXISYMMETRIC;
  const int32_t coarse_max = std::min(kCoarseMax, std::max(kCoarseMin, m.N / 64));
  auto fail = [&](const char* msg) {
    if (err && errlen) std::snprintf(err, errlen, "%s", msg);
    return AVIP_EINVAL;
  };
  H.lv.clear();
  // finest level: the scaled matrix, read back from its SELL form (explicit zeros dropped;
  // diagonal first, then the other columns ascending)
  Csr A;
  A.n = A.m = m.N;
  A.rp.assign(m.N + 1, 0);
  std::vector<std::pair<int32_t, double>> row;
  for (int32_t i = 0; i < m.N; ++i) {
    const int32_t s = i / kSlice, l = i % kSlice;
    row.clear();
    for (int32_t k = 0; k < m.rlen[i]; ++k) {
      const int64_t e = (int64_t)m.sl_ptr[s] + (int64_t)k * kSlice + l;
      if (k == 0 || m.aval[e] != 0.0) row.emplace_back(m.col[e], m.aval[e]);
    }
    std::sort(row.begin() + 1, row.end());
    for (const auto& cv : row) {
      A.ci.push_back(cv.first);
      A.v.push_back(cv.second);
    }
    A.rp[i + 1] = (int32_t)A.ci.size();
  }
  std::vector<double> B(m.N);
  for (int32_t i = 0; i < m.N; ++i) B[i] = m.bc[i] == 1 ? 0.0 : m.dsq[i];
  while (true) {
    AmgHostLevel L;
    L.dinv.resize(A.n);
    for (int32_t i = 0; i < A.n; ++i) {
      const double d = diag_of(A, i);
      if (!(d > 0)) return fail("AMG set-up: non-positive diagonal");
      L.dinv[i] = 1.0 / d;
    }
    L.lmax = lambda_max(A, L.dinv);
    if (A.n <= coarse_max || H.lv.size() + 1 >= (size_t)kAmgMaxLevels) {
      std::vector<double> dense((size_t)A.n * A.n, 0.0);
      for (int32_t i = 0; i < A.n; ++i)
        for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) dense[(size_t)i * A.n + A.ci[e]] += A.v[e];
      if (symmetric ? !dense_spd_inverse(dense, A.n) : !dense_inverse(dense, A.n))
        return fail("AMG set-up: coarse matrix is singular");
      H.nc = A.n;
      H.cinv.swap(dense);
      L.A = std::move(A);
      H.lv.push_back(std::move(L));
      break;
    }
    std::vector<int32_t> agg;
    int32_t na = aggregate(A, agg, kTheta);
    // a strongly diagonally dominant matrix (a Helmholtz operator with a large shift on a
    // coarse mesh) may have no strong connection at all: aggregate its graph instead
    if (na <= 0 || na >= A.n) na = aggregate(A, agg, 0.0);
    if (na <= 0 || na >= A.n) return fail("AMG set-up: aggregation made no progress");
    std::vector<double> norm2(na, 0.0);
    for (int32_t i = 0; i < A.n; ++i)
      if (agg[i] >= 0) norm2[agg[i]] += B[i] * B[i];
    Csr T;
    T.n = A.n;
    T.m = na;
    T.rp.assign(A.n + 1, 0);
    for (int32_t i = 0; i < A.n; ++i) {
      if (agg[i] >= 0 && norm2[agg[i]] > 0) {
        T.ci.push_back(agg[i]);
        T.v.push_back(B[i] / std::sqrt(norm2[agg[i]]));
      }
      T.rp[i + 1] = (int32_t)T.ci.size();
    }
    std::vector<double> Bc(na);
    for (int32_t j = 0; j < na; ++j) Bc[j] = std::sqrt(norm2[j]);
    // smoothed prolongator P = T - omega D^-1 A T
    const double omega = 4.0 / (3.0 * L.lmax);
    const Csr AT = spgemm(A, T);
    Csr P;
    P.n = A.n;
    P.m = na;
    P.rp.assign(A.n + 1, 0);
    {
      std::vector<double> acc(na, 0.0);
      std::vector<int32_t> mark(na, -1), cols;
      for (int32_t i = 0; i < A.n; ++i) {
        cols.clear();
        auto add = [&](int32_t j, double v) {
          if (mark[j] != i) {
            mark[j] = i;
            acc[j] = 0.0;
            cols.push_back(j);
          }
          acc[j] += v;
        };
        for (int32_t e = T.rp[i]; e < T.rp[i + 1]; ++e) add(T.ci[e], T.v[e]);
        for (int32_t e = AT.rp[i]; e < AT.rp[i + 1]; ++e) add(AT.ci[e], -omega * L.dinv[i] * AT.v[e]);
        std::sort(cols.begin(), cols.end());
        for (int32_t j : cols)
          if (acc[j] != 0.0) {
            P.ci.push_back(j);
            P.v.push_back(acc[j]);
          }
        P.rp[i + 1] = (int32_t)P.ci.size();
      }
    }
    Csr R = transpose(P);
    Csr Ac = spgemm(R, spgemm(A, P));
    // (the composite operators of this level are formed below, once P and R are final)
    if (symmetric) {  // symmetrise the rounding of the Galerkin product (its pattern is symmetric)
      const Csr AcT = transpose(Ac);
      for (int32_t i = 0; i < Ac.n; ++i)
        for (int32_t e = Ac.rp[i], f = AcT.rp[i]; e < Ac.rp[i + 1]; ++e, ++f) Ac.v[e] = 0.5 * (Ac.v[e] + AcT.v[f]);
    }
    L.A = std::move(A);
    L.P = std::move(P);
    L.R = std::move(R);
    composite_operators(L, symmetric);
    H.lv.push_back(std::move(L));
    A = std::move(Ac);
    B.swap(Bc);
  }
  return AVIP_OK;
}

}  // namespace avip
