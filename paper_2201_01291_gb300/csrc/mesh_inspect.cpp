// Host-only inspection of the prepared mesh (mesh_inspect in include/avip.h): the same
// preparation as mesh_create, without a device, reported in the caller's numbering.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "avip_internal.h"

using namespace avip;

namespace {
thread_local char g_inspect_err[256];
}

extern "C" const char* avip_inspect_error(void) { return g_inspect_err; }

extern "C" int mesh_inspect(const double* xy, int32_t n_nodes, const int32_t* tris, int32_t n_tris,
                            const int32_t* quads, int32_t n_quads, const int32_t* node_bc, const double* phi_D,
                            int32_t geometry, int64_t* counts, double* vol, int32_t* edges, double* S_edge,
                            double* S_b) {
  if (!counts) return AVIP_EINVAL;
  HostMesh m;
  g_inspect_err[0] = 0;
  const int rc = prepare_mesh(xy, n_nodes, tris, n_tris, quads, n_quads, node_bc, phi_D, 1, geometry, m,
                              g_inspect_err, sizeof(g_inspect_err));
  if (rc != AVIP_OK) return rc;
  const int32_t E = (int32_t)m.e_lo.size();
  counts[0] = E;
  counts[1] = m.nnz;
  counts[2] = m.T;
  // edges in caller numbering, (i < j), sorted; S oriented i -> j
  if (edges || S_edge) {
    std::vector<int64_t> order(E);
    std::vector<int32_t> a(E), b(E);
    std::vector<double> sx(E), sy(E);
    for (int32_t e = 0; e < E; ++e) {
      int32_t p = m.perm[m.e_lo[e]], q = m.perm[m.e_hi[e]];
      double x = m.e_sx[e], y = m.e_sy[e];
      if (p > q) {
        std::swap(p, q);
        x = -x;
        y = -y;
      }
      a[e] = p;
      b[e] = q;
      sx[e] = x;
      sy[e] = y;
      order[e] = e;
    }
    std::sort(order.begin(), order.end(), [&](int64_t u, int64_t v) {
      return a[u] != a[v] ? a[u] < a[v] : b[u] < b[v];
    });
    for (int32_t k = 0; k < E; ++k) {
      const int64_t e = order[k];
      if (edges) {
        edges[2 * (size_t)k] = a[e];
        edges[2 * (size_t)k + 1] = b[e];
      }
      if (S_edge) {
        S_edge[2 * (size_t)k] = sx[e];
        S_edge[2 * (size_t)k + 1] = sy[e];
      }
    }
  }
  for (int32_t i = 0; i < m.N; ++i) {
    const int32_t c = m.perm[i];
    if (vol) vol[c] = m.vol[i];
    if (S_b) {
      const int32_t s = i / kSlice, l = i % kSlice;
      const int64_t d = m.sl_ptr[s] + l;  // diagonal slot: the boundary nodal normal
      S_b[2 * (size_t)c] = m.sx[d];
      S_b[2 * (size_t)c + 1] = m.sy[d];
    }
  }
  return AVIP_OK;
}
