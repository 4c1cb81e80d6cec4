// Host-side mesh preparation: validation, Morton renumbering, vertex-centred metrics and the
// SELL-32 sparse structures consumed by the kernels.
//
// Metrics (section "Nomenclature and notations" and "Cartesian geometry"):
//   * V_tau = signed area of the counter-clockwise triangle;
//   * nodal normal S_k^tau (Eq. node_normal) = minus the sum of the two faces adjacent to k,
//     which for a triangle is the outward length-normal of the face opposite k;
//   * median-dual volume V_i = sum over E(i) of V_tau / 3;
//   * edge normal S_ij^tau = (S_i^tau - S_j^tau) / 6, oriented i -> j (the relation quoted in
//     the axisymmetric section; it satisfies sum_j S_ij^tau = S_i^tau / n_d), summed over the
//     cells sharing the edge;
//   * boundary nodal normal S_i^b = 1/2 sum of the outward normals of the boundary faces at
//     i (Fig. bcs_normal);
//   * Poisson matrix K_ik = sum_tau S_i.S_k / (n_d^2 V_tau) (Eq. coeff_matriceA with the sign
//     of -lap phi = rho/eps0), Dirichlet unknowns eliminated symmetrically, then scaled
//     symmetrically by its diagonal (D^-1/2 K D^-1/2) for Jacobi-preconditioned CG;
//   * nodal gradient weights: grad u_i = (1/V_i) sum_tau (V_tau/3) grad u_tau with
//     grad u_tau = -1/(n_d V_tau) sum_k u_k S_k, i.e. grad u_i = sum_k G_ik u_k with
//     G_ik = -(1 / (6 V_i)) sum_{tau containing i and k} S_k^tau.
//
// Quadrangles (hybrid meshes, planar geometry; n_v = 4 vertices, n_v^f = n_d = 2):
//   * V_tau = shoelace area of the counter-clockwise quadrangle, dual share V_tau / 4;
//   * nodal normal S_k = -(S_f(k-1,k) + S_f(k,k+1)), the two faces adjacent to k;
//   * edge normal of side (k, k+1): length-normal of the dual face from the side midpoint to
//     the cell centre (vertex mean), oriented k -> k+1; the diagonals carry no edge;
//   * K_ik = S_i.S_k / (4 V_tau) couples all four vertices (diagonals included), and
//     G_ik = -(1 / (2 n_v A_i)) sum S_k likewise.
//
// Axisymmetric geometry (second coordinate = radius r; every integral per radian):
//   * Poisson row i: K_ik = sum_tau S_k . I_i^tau / (n_d V_tau), with I_i^tau the integral of
//     r n dl over the dual contour of i inside tau in the closed form of the axisymmetric
//     Poisson section, 1/24 [(4 r_tau + 2 r_i + r_j + r_l) S_i - (2 r_tau + r_i + r_j) S_j
//     - (2 r_tau + r_i + r_l) S_l]; the radius makes K non-symmetric;
//   * dual volume = integral of r over the median-dual cell, per triangle
//     V_tau (22 r_i + 7 r_j + 7 r_l) / 108 (the centroid radius of the dual cell in the
//     second Pappus theorem; the node radius would give nodes on the axis no volume);
//   * edge normal S_ij^tau times the radius at the middle of its dual face,
//     ((r_i + r_j)/2 + r_tau)/2 (first Pappus theorem, axisymmetric flux form);
//   * boundary normal: each half face times the radius at its middle, (3 r_p + r_q)/4;
//   * the gradient is two-dimensional: G_ik keeps the planar dual areas.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "avip_internal.h"

namespace avip {

namespace {

uint64_t spread_bits(uint64_t v) {  // 21 bits -> every other bit
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

void morton_order(const double* xy, int32_t n, std::vector<int32_t>& perm) {
  double xmin = xy[0], xmax = xy[0], ymin = xy[1], ymax = xy[1];
  for (int32_t i = 0; i < n; ++i) {
    xmin = std::min(xmin, xy[2 * i]);
    xmax = std::max(xmax, xy[2 * i]);
    ymin = std::min(ymin, xy[2 * i + 1]);
    ymax = std::max(ymax, xy[2 * i + 1]);
  }
  double ext = std::max(xmax - xmin, ymax - ymin);
  if (!(ext > 0)) ext = 1.0;
  const double scale = double((1u << 21) - 1) / ext;
  std::vector<uint64_t> key(n);
  for (int32_t i = 0; i < n; ++i) {
    uint64_t qx = (uint64_t)std::llround((xy[2 * i] - xmin) * scale);
    uint64_t qy = (uint64_t)std::llround((xy[2 * i + 1] - ymin) * scale);
    key[i] = spread_bits(qx) | (spread_bits(qy) << 1);
  }
  perm.resize(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
}

}  // namespace

int prepare_mesh(const double* xy, int32_t n_nodes, const int32_t* tris, int32_t n_tris, const int32_t* quads,
                 int32_t n_quads, const int32_t* node_bc, const double* phi_D, int reorder, int geometry,
                 HostMesh& m, char* err, size_t errlen) {
  auto fail = [&](const char* msg) {
    if (err && errlen) std::snprintf(err, errlen, "%s", msg);
    return AVIP_EINVAL;
  };
  if (!xy || !node_bc || !phi_D || (n_tris > 0 && !tris) || (n_quads > 0 && !quads)) return fail("null input array");
  if (n_tris < 0 || n_quads < 0) return fail("negative cell count");
  if (n_nodes < 3 || (int64_t)n_tris + n_quads < 1) return fail("mesh needs at least 3 nodes and 1 cell");
  if ((int64_t)n_tris + n_quads > INT32_MAX / 4) return fail("too many cells");
  const int32_t N = n_nodes, T = n_tris + n_quads, Q = n_quads;
  for (int64_t k = 0; k < 3LL * n_tris; ++k)
    if (tris[k] < 0 || tris[k] >= N) return fail("triangle index out of range");
  for (int64_t k = 0; k < 4LL * n_quads; ++k)
    if (quads[k] < 0 || quads[k] >= N) return fail("quadrangle index out of range");
  int ndir = 0;
  for (int32_t i = 0; i < N; ++i) {
    if (node_bc[i] < 0 || node_bc[i] > 2) return fail("node_bc must be 0, 1 or 2");
    if (!std::isfinite(xy[2 * i]) || !std::isfinite(xy[2 * i + 1])) return fail("non-finite coordinate");
    if (node_bc[i] == 1) {
      ++ndir;
      if (!std::isfinite(phi_D[i])) return fail("non-finite Dirichlet value");
    }
  }
  if (ndir == 0) return fail("at least one Dirichlet node is required (pure Neumann problem is singular)");
  if (geometry != AVIP_GEOM_PLANAR && geometry != AVIP_GEOM_AXISYMMETRIC) return fail("unknown geometry");
  const bool axi = geometry == AVIP_GEOM_AXISYMMETRIC;
  if (axi && Q > 0) return fail("quadrangles are supported in the planar geometry only");
  if (axi)
    for (int32_t i = 0; i < N; ++i)
      if (xy[2 * i + 1] < 0) return fail("axisymmetric mesh with a negative radius (y < 0)");
  m.geometry = geometry;

  // ---- renumbering
  if (reorder) {
    morton_order(xy, N, m.perm);
  } else {
    m.perm.resize(N);
    std::iota(m.perm.begin(), m.perm.end(), 0);
  }
  m.iperm.assign(N, 0);
  for (int32_t i = 0; i < N; ++i) m.iperm[m.perm[i]] = i;
  m.N = N;
  m.T = T;
  m.Q = Q;
  m.nvmax = Q > 0 ? 4 : 3;
  m.x.resize(N);
  m.y.resize(N);
  m.bc.resize(N);
  for (int32_t i = 0; i < N; ++i) {
    m.x[i] = xy[2 * m.perm[i]];
    m.y[i] = xy[2 * m.perm[i] + 1];
    m.bc[i] = node_bc[m.perm[i]] == 1 ? 1 : 0;  // 2 (Neumann side) is the natural condition, as 0
  }

  // ---- cells: orientation, volume, nodal normals, side normals of the dual faces, shortest side
  // Cells 0..n_tris-1 are the triangles, then the quadrangles; per cell up to 4 vertices.
  std::vector<int32_t> nv(T), tv(4 * (size_t)T, -1);
  std::vector<double> Vt(T), Sn(8 * (size_t)T), Sd(8 * (size_t)T);  // Sn[8c + 2k + {0,1}], Sd likewise
  m.dxmin.resize(T);
  for (int32_t c = 0; c < T; ++c) {
    int32_t* v = tv.data() + 4 * (size_t)c;
    double* S = Sn.data() + 8 * (size_t)c;
    double* D = Sd.data() + 8 * (size_t)c;
    if (c < n_tris) {
      nv[c] = 3;
      int32_t a = m.iperm[tris[3 * c]], b = m.iperm[tris[3 * c + 1]], d = m.iperm[tris[3 * c + 2]];
      double cr = (m.x[b] - m.x[a]) * (m.y[d] - m.y[a]) - (m.y[b] - m.y[a]) * (m.x[d] - m.x[a]);
      if (cr < 0) {
        std::swap(b, d);
        cr = -cr;
      }
      if (!(cr > 0)) return fail("degenerate (zero-area) triangle");
      v[0] = a;
      v[1] = b;
      v[2] = d;
      Vt[c] = 0.5 * cr;
      for (int k = 0; k < 3; ++k) {
        int32_t p = v[(k + 1) % 3], q = v[(k + 2) % 3];
        // outward length-normal of the opposite face p -> q (right-hand side of travel)
        S[2 * k] = m.y[q] - m.y[p];
        S[2 * k + 1] = -(m.x[q] - m.x[p]);
      }
      // dual face of side (k, k+1): (S_k - S_k+1) / 6, oriented k -> k+1
      for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3;
        D[2 * k] = (S[2 * k] - S[2 * k1]) / 6.0;
        D[2 * k + 1] = (S[2 * k + 1] - S[2 * k1 + 1]) / 6.0;
      }
    } else {
      nv[c] = 4;
      const int32_t* qc = quads + 4 * (size_t)(c - n_tris);
      for (int k = 0; k < 4; ++k) v[k] = m.iperm[qc[k]];
      double a2 = 0.0;  // twice the signed shoelace area
      for (int k = 0; k < 4; ++k) {
        const int32_t p = v[k], q = v[(k + 1) % 4];
        a2 += m.x[p] * m.y[q] - m.x[q] * m.y[p];
      }
      if (a2 < 0) {
        std::swap(v[0], v[3]);
        std::swap(v[1], v[2]);
        a2 = 0.0;
        for (int k = 0; k < 4; ++k) {
          const int32_t p = v[k], q = v[(k + 1) % 4];
          a2 += m.x[p] * m.y[q] - m.x[q] * m.y[p];
        }
      }
      if (!(a2 > 0)) return fail("degenerate (zero-area) quadrangle");
      Vt[c] = 0.5 * a2;
      // nodal normal (Eq. node_normal, n_d = n_v^f = 2): minus the two faces adjacent to k
      double Fx[4], Fy[4];
      for (int k = 0; k < 4; ++k) {
        const int32_t p = v[k], q = v[(k + 1) % 4];
        Fx[k] = m.y[q] - m.y[p];
        Fy[k] = -(m.x[q] - m.x[p]);
      }
      for (int k = 0; k < 4; ++k) {
        S[2 * k] = -(Fx[k] + Fx[(k + 3) % 4]);
        S[2 * k + 1] = -(Fy[k] + Fy[(k + 3) % 4]);
      }
      // dual face of side (k, k+1): from the side midpoint to the cell centre (vertex mean),
      // length-normal oriented k -> k+1
      const double cx = (((m.x[v[0]] + m.x[v[1]]) + m.x[v[2]]) + m.x[v[3]]) / 4.0;
      const double cy = (((m.y[v[0]] + m.y[v[1]]) + m.y[v[2]]) + m.y[v[3]]) / 4.0;
      for (int k = 0; k < 4; ++k) {
        const int32_t p = v[k], q = v[(k + 1) % 4];
        const double wx = cx - 0.5 * (m.x[p] + m.x[q]), wy = cy - 0.5 * (m.y[p] + m.y[q]);
        double nx = wy, ny = -wx;
        const double dot = nx * (m.x[q] - m.x[p]) + ny * (m.y[q] - m.y[p]);
        const double sg = dot > 0 ? 1.0 : (dot < 0 ? -1.0 : 0.0);
        D[2 * k] = nx * sg;
        D[2 * k + 1] = ny * sg;
      }
    }
    double l = INFINITY;
    for (int k = 0; k < nv[c]; ++k) {
      const int32_t p = v[k], q = v[(k + 1) % nv[c]];
      l = std::min(l, std::hypot(m.x[q] - m.x[p], m.y[q] - m.y[p]));
    }
    m.dxmin[c] = l;
  }
  m.cw.resize(T);
  m.dxmin_all = INFINITY;
  for (int32_t c = 0; c < T; ++c) {
    m.cw[c] = 1.0 / ((double)nv[c] * m.dxmin[c]);
    m.dxmin_all = std::min(m.dxmin_all, m.dxmin[c]);
  }
  m.cell.assign((size_t)m.nvmax * T, -1);
  for (int32_t c = 0; c < T; ++c)
    for (int k = 0; k < nv[c]; ++k) m.cell[(size_t)k * T + c] = tv[4 * (size_t)c + k];

  // ---- node -> cells
  std::vector<int32_t> ncell(N + 1, 0);
  for (int32_t c = 0; c < T; ++c)
    for (int k = 0; k < nv[c]; ++k) ncell[tv[4 * (size_t)c + k] + 1]++;
  for (int32_t i = 0; i < N; ++i) ncell[i + 1] += ncell[i];
  std::vector<int32_t> cells(ncell[N]);
  {
    std::vector<int32_t> fillp(ncell.begin(), ncell.end() - 1);
    for (int32_t c = 0; c < T; ++c)
      for (int k = 0; k < nv[c]; ++k) cells[fillp[tv[4 * (size_t)c + k]]++] = c;
  }
  // planar dual areas (gradient weights) and the dual volumes of the transport update
  std::vector<double> area(N, 0.0);
  for (int32_t i = 0; i < N; ++i)
    for (int32_t e = ncell[i]; e < ncell[i + 1]; ++e) area[i] += Vt[cells[e]] / (double)nv[cells[e]];
  for (int32_t i = 0; i < N; ++i)
    if (!(area[i] > 0)) return fail("node not used by any cell");
  if (axi) {
    m.vol.assign(N, 0.0);
    for (int32_t c = 0; c < T; ++c)
      for (int k = 0; k < 3; ++k) {
        const int32_t i = tv[4 * c + k], j = tv[4 * c + (k + 1) % 3], l = tv[4 * c + (k + 2) % 3];
        m.vol[i] += Vt[c] * (22.0 * m.y[i] + 7.0 * m.y[j] + 7.0 * m.y[l]) / 108.0;
      }
    for (int32_t i = 0; i < N; ++i)
      if (!(m.vol[i] > 0)) return fail("axisymmetric dual volume is not positive");
  } else {
    m.vol = area;
  }

  // ---- rows: diagonal, then the edge neighbours ascending, then the other cell vertices
  std::vector<int32_t> rowptr(N + 1, 0), fl(N, 1);
  std::vector<int32_t> cols;
  cols.reserve((size_t)N * 8);
  {
    std::vector<int32_t> nb, other;
    for (int32_t i = 0; i < N; ++i) {
      nb.clear();
      other.clear();
      for (int32_t e = ncell[i]; e < ncell[i + 1]; ++e) {
        const int32_t c = cells[e];
        const int32_t* v = tv.data() + 4 * (size_t)c;
        const int n = nv[c];
        int li = 0;
        while (v[li] != i) ++li;
        nb.push_back(v[(li + 1) % n]);
        nb.push_back(v[(li + n - 1) % n]);
        for (int k = 0; k < n; ++k)
          if (v[k] != i) other.push_back(v[k]);
      }
      std::sort(nb.begin(), nb.end());
      nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
      std::sort(other.begin(), other.end());
      other.erase(std::unique(other.begin(), other.end()), other.end());
      cols.push_back(i);
      cols.insert(cols.end(), nb.begin(), nb.end());
      fl[i] = 1 + (int32_t)nb.size();
      for (int32_t k : other)
        if (!std::binary_search(nb.begin(), nb.end(), k)) cols.push_back(k);
      rowptr[i + 1] = (int32_t)cols.size();
    }
  }
  const int64_t nnz = (int64_t)cols.size();
  m.nnz = nnz;
  {
    int64_t se = 0;
    for (int32_t i = 0; i < N; ++i) se += fl[i] - 1;
    m.E = (int32_t)(se / 2);
  }
  std::vector<double> K(nnz, 0.0), Gx(nnz, 0.0), Gy(nnz, 0.0), Sx(nnz, 0.0), Sy(nnz, 0.0);
  std::vector<int32_t> shared(nnz, 0);
  auto slot = [&](int32_t i, int32_t k) -> int64_t {
    if (k == i) return rowptr[i];
    const int32_t* b = cols.data() + rowptr[i] + 1;
    const int32_t* f = cols.data() + rowptr[i] + fl[i];
    const int32_t* p = std::lower_bound(b, f, k);
    if (p != f && *p == k) return (int64_t)(p - cols.data());
    const int32_t* e = cols.data() + rowptr[i + 1];
    return (int64_t)(std::lower_bound(f, e, k) - cols.data());
  };
  for (int32_t i = 0; i < N; ++i) {
    for (int32_t e = ncell[i]; e < ncell[i + 1]; ++e) {
      const int32_t c = cells[e];
      const int32_t* v = tv.data() + 4 * (size_t)c;
      const double* S = Sn.data() + 8 * (size_t)c;
      const double* D = Sd.data() + 8 * (size_t)c;
      const int n = nv[c];
      int li = 0;
      while (v[li] != i) ++li;
      const double six = S[2 * li], siy = S[2 * li + 1];
      // axisymmetric (triangles only): integral of r n dl over the dual contour of i inside c
      double Ix = 0.0, Iy = 0.0, rc = 0.0;
      if (axi) {
        const int lj = (li + 1) % 3, ll = (li + 2) % 3;
        const double ri = m.y[i], rj = m.y[v[lj]], rl = m.y[v[ll]];
        rc = (ri + rj + rl) / 3.0;
        const double wi = 4.0 * rc + 2.0 * ri + rj + rl, wj = 2.0 * rc + ri + rj, wl = 2.0 * rc + ri + rl;
        Ix = (wi * six - wj * S[2 * lj] - wl * S[2 * ll]) / 24.0;
        Iy = (wi * siy - wj * S[2 * lj + 1] - wl * S[2 * ll + 1]) / 24.0;
      }
      for (int k = 0; k < n; ++k) {
        const int32_t j = v[k];
        const int64_t s = slot(i, j);
        const double skx = S[2 * k], sky = S[2 * k + 1];
        if (axi)
          K[s] += (Ix * skx + Iy * sky) / (2.0 * Vt[c]);
        else
          K[s] += (six * skx + siy * sky) / (4.0 * Vt[c]);
        // grad u_i = (1/A_i) sum_c (V_c/n_v) grad u_c, grad u_c = -1/(n_d V_c) sum_k u_k S_k
        Gx[s] += -skx / (2.0 * n * area[i]);
        Gy[s] += -sky / (2.0 * n * area[i]);
      }
      // the two sides of c at i: (li, li+1) leaves i forward, (li-1, li) arrives at i
      for (int side = 0; side < 2; ++side) {
        const int m0 = side == 0 ? li : (li + n - 1) % n;
        const int32_t j = side == 0 ? v[(li + 1) % n] : v[m0];
        const double sg = side == 0 ? 1.0 : -1.0;  // D is oriented m0 -> m0+1
        const int64_t s = slot(i, j);
        const double rf = axi ? 0.5 * (0.5 * (m.y[i] + m.y[j]) + rc) : 1.0;
        Sx[s] += rf * (sg * D[2 * m0]);
        Sy[s] += rf * (sg * D[2 * m0 + 1]);
        shared[s] += 1;
      }
    }
  }
  // boundary faces: sides with a single adjacent cell; their outward normal is split between
  // the two end nodes (stored in the diagonal slot)
  for (int32_t c = 0; c < T; ++c) {
    const int n = nv[c];
    for (int k = 0; k < n; ++k) {
      int32_t p = tv[4 * (size_t)c + k], q = tv[4 * (size_t)c + (k + 1) % n];
      if (shared[slot(p, q)] == 1) {
        double nx = m.y[q] - m.y[p], ny = -(m.x[q] - m.x[p]);
        // axisymmetric: each half face weighted by the radius at its middle
        const double wp = axi ? 0.25 * (3.0 * m.y[p] + m.y[q]) : 1.0;
        const double wq = axi ? 0.25 * (3.0 * m.y[q] + m.y[p]) : 1.0;
        Sx[rowptr[p]] += 0.5 * nx * wp;
        Sy[rowptr[p]] += 0.5 * ny * wp;
        Sx[rowptr[q]] += 0.5 * nx * wq;
        Sy[rowptr[q]] += 0.5 * ny * wq;
      }
    }
  }

  // ---- Dirichlet elimination
  m.lift.assign(N, 0.0);
  m.rhs_scale.assign(N, 0.0);
  std::vector<double> Ael(K);
  for (int32_t i = 0; i < N; ++i) {
    if (m.bc[i] == 1) {
      for (int32_t s = rowptr[i]; s < rowptr[i + 1]; ++s) Ael[s] = 0.0;
      Ael[rowptr[i]] = 1.0;
      m.lift[i] = phi_D[m.perm[i]];
      m.rhs_scale[i] = 0.0;
    } else {
      double l = 0.0;
      for (int32_t s = rowptr[i] + 1; s < rowptr[i + 1]; ++s) {
        int32_t k = cols[s];
        if (m.bc[k] == 1) {
          l -= K[s] * phi_D[m.perm[k]];
          Ael[s] = 0.0;
        }
      }
      m.lift[i] = l;
      m.rhs_scale[i] = kECharge * m.vol[i] / kEps0;
    }
    if (!(Ael[rowptr[i]] > 0)) return fail("non-positive Poisson diagonal");
  }
  // symmetric Jacobi scaling: Jacobi-PCG on K is plain CG on D^-1/2 K D^-1/2
  m.dsq.assign(N, 1.0);
  m.dsqinv.assign(N, 1.0);
  for (int32_t i = 0; i < N; ++i) {
    m.dsq[i] = std::sqrt(Ael[rowptr[i]]);
    m.dsqinv[i] = 1.0 / m.dsq[i];
  }
  for (int32_t i = 0; i < N; ++i) {
    for (int32_t s = rowptr[i]; s < rowptr[i + 1]; ++s) Ael[s] = Ael[s] / (m.dsq[i] * m.dsq[cols[s]]);
    m.lift[i] *= m.dsqinv[i];
    m.rhs_scale[i] *= m.dsqinv[i];
  }

  // ---- SELL-32 layout
  m.nslices = (N + kSlice - 1) / kSlice;
  const int32_t Npad = m.nslices * kSlice;
  m.rlen.assign(Npad, 0);
  m.flen.assign(Npad, 0);
  for (int32_t i = 0; i < N; ++i) {
    m.rlen[i] = rowptr[i + 1] - rowptr[i];
    m.flen[i] = fl[i];
  }
  m.sl_ptr.resize(m.nslices + 1);
  m.sl_w.resize(m.nslices);
  int64_t off = 0;
  for (int32_t s = 0; s < m.nslices; ++s) {
    int32_t w = 0;
    for (int l = 0; l < kSlice; ++l) w = std::max(w, m.rlen[s * kSlice + l]);
    m.sl_w[s] = w;
    m.sl_ptr[s] = (int32_t)off;
    off += (int64_t)w * kSlice;
    if (off > INT32_MAX) return fail("mesh too large for 32-bit sparse offsets");
  }
  m.sl_ptr[m.nslices] = (int32_t)off;
  m.nelem = off;
  m.col.assign(off, 0);
  m.aval.assign(off, 0.0);
  m.gx.assign(off, 0.0);
  m.gy.assign(off, 0.0);
  m.sx.assign(off, 0.0);
  m.sy.assign(off, 0.0);
  for (int32_t s = 0; s < m.nslices; ++s) {
    for (int l = 0; l < kSlice; ++l) {
      int32_t i = s * kSlice + l;
      for (int32_t k = 0; k < m.sl_w[s]; ++k) {
        int64_t e = (int64_t)m.sl_ptr[s] + (int64_t)k * kSlice + l;
        if (i < N && k < m.rlen[i]) {
          int64_t src = rowptr[i] + k;
          m.col[e] = cols[src];
          m.aval[e] = Ael[src];
          m.gx[e] = Gx[src];
          m.gy[e] = Gy[src];
          m.sx[e] = Sx[src];
          m.sy[e] = Sy[src];
        } else {
          m.col[e] = (i < N) ? i : 0;
        }
      }
    }
  }
  // ---- edge list for the flux-per-edge kernel: each edge once, from its lo row
  {
    std::vector<int32_t> first(N + 1, 0);
    for (int32_t i = 0; i < N; ++i) {
      int32_t c = 0;
      for (int32_t k = 1; k < fl[i]; ++k)
        if (cols[rowptr[i] + k] > i) ++c;
      first[i + 1] = first[i] + c;
    }
    const int32_t E = first[N];
    m.e_lo.resize(E);
    m.e_hi.resize(E);
    m.e_sx.resize(E);
    m.e_sy.resize(E);
    m.slot_eid.assign(off, 0);
    for (int32_t i = 0; i < N; ++i) {
      int32_t e = first[i];
      for (int32_t k = 1; k < fl[i]; ++k) {
        const int32_t j = cols[rowptr[i] + k];
        if (j > i) {
          m.e_lo[e] = i;
          m.e_hi[e] = j;
          m.e_sx[e] = Sx[rowptr[i] + k];
          m.e_sy[e] = Sy[rowptr[i] + k];
          ++e;
        }
      }
    }
    // slot -> edge: the lo row's edges are found by position, the hi row's by search in the
    // lo row's (ascending) edge range
    for (int32_t i = 0; i < N; ++i) {
      const int32_t s = i / kSlice, l = i % kSlice;
      int32_t e = first[i];
      for (int32_t k = 1; k < fl[i]; ++k) {
        const int32_t j = cols[rowptr[i] + k];
        int32_t id;
        if (j > i) {
          id = e++;
        } else {
          const int32_t* b = m.e_hi.data() + first[j];
          const int32_t* f = m.e_hi.data() + first[j + 1];
          const int32_t* p = std::lower_bound(b, f, i);
          if (p == f || *p != i) return fail("internal: edge list inconsistent");
          id = (int32_t)(p - m.e_hi.data()) | (int32_t)0x80000000u;
        }
        m.slot_eid[(int64_t)m.sl_ptr[s] + (int64_t)k * kSlice + l] = id;
      }
    }
  }
  return AVIP_OK;
}

}  // namespace avip
