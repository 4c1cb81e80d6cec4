// C ABI entry points (include/avip.h): handle life cycle, device memory, launch sequencing
// of one explicit step, CUDA-graph replay of the time loop, host <-> device field copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "avip_internal.h"

namespace avip {
// NVTX range around the host code that queues one stage (kernel) or one step, so that a
// timeline tool shows the library's work by name; free when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

cudaError_t launch_pcg_fp64(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st);
cudaError_t launch_pcg_mixed(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st);
cudaError_t launch_bicgstab(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st);
cudaError_t launch_pcg_amg(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st);
cudaError_t launch_amg_group(const AmgGroupArgs& g, const PcgPlan& pl, cudaStream_t st);
cudaError_t launch_pcg_amg_cluster(const PcgArgs& args, const PcgPlan& pl, cudaStream_t st);
cudaError_t launch_pcg_cluster(const PcgArgs& args, const PcgPlan& pl, const ClusterLayout& L, cudaStream_t st);
cudaError_t launch_node_fields(const DDArgs& a, int with_dt, cudaStream_t st);
cudaError_t launch_dt_cells(const DDArgs& a, cudaStream_t st);
cudaError_t launch_photo_add(const DDArgs& a, int with_dt, cudaStream_t st);
cudaError_t launch_flux_update(const DDArgs& a, cudaStream_t st);
cudaError_t launch_finalize(DevScalars* sc, const double* partials, int nparts, cudaStream_t st);
cudaError_t launch_run_reset(DevScalars* sc, cudaStream_t st);
int flux_blocks(int N);
cudaError_t launch_state_take(const StateArgs& s, cudaStream_t st);
cudaError_t launch_state_check(const StateArgs& s, cudaStream_t st);
cudaError_t launch_state_put(const StateArgs& s, cudaStream_t st);
int flux_partials_max(int N);
}  // namespace avip

using namespace avip;

struct avip_mesh {
  avip_opts opts;
  HostMesh hm;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  size_t bytes = 0;  // device bytes held
  // device arrays
  int32_t *sl_ptr = nullptr, *sl_w = nullptr, *rlen = nullptr, *col = nullptr, *cell = nullptr, *flen = nullptr;
  double *aval = nullptr, *gx = nullptr, *gy = nullptr, *sx = nullptr, *sy = nullptr;
  double *ivol = nullptr;  // 1 / V_i (the update multiplies; an FP64 division costs ~10 FP64 instructions)
  double *x = nullptr, *y = nullptr, *vol = nullptr, *dsq = nullptr, *dsqinv = nullptr, *lift = nullptr,
         *rhs_scale = nullptr;
  double* cw = nullptr;
  int32_t *e_lo = nullptr, *e_hi = nullptr, *slot_eid = nullptr;  // edge list (flux once per edge)
  double *e_sx = nullptr, *e_sy = nullptr, *eflux = nullptr;
  double *phi1 = nullptr, *phi2 = nullptr, *phi3 = nullptr;  // the three previous potentials (predictor)
  double *phi = nullptr, *xs = nullptr, *b = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
  double *nbuf = nullptr, *ndat = nullptr, *nm = nullptr, *src = nullptr, *Ex = nullptr, *Ey = nullptr;
  double* qpart = nullptr;      // per-block charge partials of the flux kernel
  double* bcg = nullptr;        // BiCGStab vectors (kind 7 only)
  AmgDev* amg = nullptr;            // AMG hierarchy with FP64 values (opts.precond_fp64)
  AmgDevT<float>* amg32 = nullptr;  // AMG hierarchy with FP32 values (default; kind 10 always)
  float* z32 = nullptr;             // preconditioned residual of the mixed-precision solve
  double* amg_z = nullptr;          // preconditioned residual of the FP64 CG (either hierarchy)
  double* r2 = nullptr;             // second buffer of the AMG-CG residual
  float* rq32 = nullptr;            // FP32 copies of both residual buffers and of q (FP32 hierarchy)
  int32_t amg_levels = 0;
  std::vector<int64_t> amg_stats;  // per level: rows, nnz(A), nnz(P)
  float *aval32 = nullptr, *e32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;  // mixed precision
  float *gx32 = nullptr, *gy32 = nullptr, *sx32 = nullptr, *sy32 = nullptr, *ndat32 = nullptr;  // FP32 DD
  GridSync* sync = nullptr;     // followed in the same allocation by the barrier flags
  unsigned* flags = nullptr;
  double* parts = nullptr;
  size_t sync_bytes = 0;
  DevScalars* sc = nullptr;
  // photoionisation: per Helmholtz term its scaled matrix values, scaling, right-hand-side
  // factors, AMG hierarchy (AMG solver kinds) and solution; the ionisation rate, the summed
  // source, a zero lift and the result block of those solves
  struct PhotoTerm {
    double *aval = nullptr, *dsq = nullptr, *dsqinv = nullptr, *rhs = nullptr;
    AmgDev* amg = nullptr;
    AmgDevT<float>* amg32 = nullptr;
  };
  std::vector<PhotoTerm> photo;
  double *photo_psi = nullptr, *photo_I = nullptr, *photo_S = nullptr, *photo_zero = nullptr;
  int32_t* photo_hist = nullptr;  // per term: earlier solutions kept for the predictor
  DevScalars* sc_aux = nullptr;   // per term: the solve's statistics
  // whole-GPU AMG solvers (kinds 8, 9): the terms are solved side by side in one launch, each on
  // its own group of blocks, with per term its own Krylov vectors (kPhotoWork x Npad doubles),
  // FP32 residual copies (3 x Npad floats, FP32 hierarchy) and barrier state
  // checkpoint copies (allocated at the first state_get / state_set): the node permutation and
  // the state in the caller's layout on the device, and a validation flag
  int32_t* d_perm = nullptr;
  double* d_stage = nullptr;
  int32_t* d_state_flag = nullptr;
  bool photo_group = false;
  double* photo_work = nullptr;
  float* photo_rq32 = nullptr;
  GridSync* photo_gs = nullptr;
  int32_t Npad = 0;
  PcgPlan plan;
  ClusterLayout clay{};
  int nparts = 0;
  Physics ph;
  int species_declared = 0;
  // graph of one step
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
};

namespace {

thread_local char g_err[256];
constexpr int kClusterAutoRows = 20000;  // one-cluster solvers up to this many nodes
constexpr int kClusterAmgMinRows = 500;  // AMG on one cluster above this many nodes (Jacobi below)

void* dev_alloc(avip_mesh* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (h->opts.alloc) {
    p = h->opts.alloc(bytes, h->opts.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    h->allocs.push_back(p);
    h->bytes += bytes;
  }
  return p;
}

void dev_free_all(avip_mesh* h) {
  for (void* p : h->allocs) {
    if (h->opts.free)
      h->opts.free(p, h->opts.alloc_ctx);
    else
      cudaFree(p);
  }
  h->allocs.clear();
}

template <typename T>
bool upload(avip_mesh* h, T*& dst, const std::vector<T>& src, size_t min_count = 0) {
  size_t n = std::max(src.size(), min_count);
  dst = static_cast<T*>(dev_alloc(h, n * sizeof(T)));
  if (!dst) return false;
  if (cudaMemsetAsync(dst, 0, n * sizeof(T), h->stream) != cudaSuccess) return false;
  if (!src.empty() && cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice,
                                      h->stream) != cudaSuccess)
    return false;
  return true;
}

template <typename T>
bool zalloc(avip_mesh* h, T*& dst, size_t count) {
  dst = static_cast<T*>(dev_alloc(h, count * sizeof(T)));
  if (!dst) return false;
  return cudaMemsetAsync(dst, 0, count * sizeof(T), h->stream) == cudaSuccess;
}

SellView sell_view(const avip_mesh* h) {
  SellView v;
  v.sl_ptr = h->sl_ptr;
  v.sl_w = h->sl_w;
  v.rlen = h->rlen;
  v.col = h->col;
  v.aval = h->aval;
  v.gx = h->gx;
  v.gy = h->gy;
  v.sx = h->sx;
  v.sy = h->sy;
  v.N = h->hm.N;
  v.nslices = h->hm.nslices;
  return v;
}

PcgArgs pcg_args(const avip_mesh* h) {
  PcgArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = sell_view(h);
  a.dsq = h->dsq;
  a.dsqinv = h->dsqinv;
  a.rhs_scale = h->rhs_scale;
  a.lift = h->lift;
  a.nbuf = h->nbuf;
  a.Npad = h->Npad;
  a.ns = h->ph.ns;
  for (int s = 0; s < AVIP_MAX_SPECIES; ++s) a.q[s] = h->ph.sp[s].q;
  a.phi = h->phi;
  a.phi1 = h->phi1;
  a.phi2 = h->phi2;
  a.phi3 = h->phi3;
  a.hist = &h->sc->phi_hist;
  a.x = h->xs;
  a.b = h->b;
  a.r = h->r;
  a.p = h->p;
  a.q_ap = h->q;
  a.flags = h->flags;
  a.parts = h->parts;
  a.sync = h->sync;
  a.sc = h->sc;
  a.res = h->sc;
  a.rtol = h->opts.rtol;
  a.v_rise = h->opts.v_rise;
  a.spin_ns = (unsigned long long)(h->opts.wait_timeout * 1e9);
  a.max_iter = h->opts.max_iter;
  a.use_density_rhs = 1;
  a.aval32 = h->aval32;
  a.e32 = h->e32;
  a.r32 = h->r32;
  a.p32 = h->p32;
  a.q32 = h->q32;
  a.inner_rtol = h->opts.inner_rtol;
  a.bcg = h->bcg;
  a.amg = h->amg;
  a.z = h->amg_z;
  a.amg32 = h->amg32;
  a.z32 = h->z32;
  a.r2 = h->r2;
  a.rq32 = h->rq32;
  a.amg_mixed = h->opts.precision == AVIP_PREC_MIXED ? 1 : 0;
  return a;
}

DDArgs dd_args(const avip_mesh* h) {
  DDArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = sell_view(h);
  a.ph = h->ph;
  // Fourier limit: fourier dx^2 / D is smallest at the shortest side and the largest D
  a.ph.dt_fourier = INFINITY;
  for (int sp = 0; sp < h->ph.ns; ++sp)
    if (h->ph.sp[sp].D > 0.0)
      a.ph.dt_fourier = std::fmin(a.ph.dt_fourier, h->ph.fourier * (h->hm.dxmin_all * h->hm.dxmin_all) / h->ph.sp[sp].D);
  a.x = h->x;
  a.y = h->y;
  a.vol = h->vol;
  a.ivol = h->ivol;
  a.phi = h->phi;
  a.nbuf = h->nbuf;
  a.ndat = h->ndat;
  a.nm = h->nm;
  a.src = h->src;
  a.Ex = h->Ex;
  a.Ey = h->Ey;
  a.photo_I = h->photo_I;
  a.photo_psi = h->photo_psi;
  a.photo_S = h->photo_S;
  a.cell = h->cell;
  a.cw = h->cw;
  a.e_lo = h->e_lo;
  a.e_hi = h->e_hi;
  a.e_sx = h->e_sx;
  a.e_sy = h->e_sy;
  a.slot_eid = h->slot_eid;
  a.eflux = h->eflux;
  a.E = (int32_t)h->hm.e_lo.size();
  a.flen = h->flen;
  a.T = h->hm.T;
  a.nvmax = h->hm.nvmax;
  a.Npad = h->Npad;
  a.partials = h->qpart;
  a.sc = h->sc;
  a.gx32 = h->gx32;
  a.gy32 = h->gy32;
  a.sx32 = h->sx32;
  a.sy32 = h->sy32;
  a.ndat32 = h->ndat32;
  return a;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return AVIP_OK;
  std::snprintf(g_err, sizeof(g_err), "CUDA: %s", cudaGetErrorString(e));
  cudaGetLastError();
  return AVIP_ECUDA;
}

cudaError_t enqueue_solver(avip_mesh* h, const PcgArgs& a) {
  if (h->plan.kind == 4) return launch_pcg_mixed(a, h->plan, h->stream);
  if (h->plan.kind == 7) return launch_bicgstab(a, h->plan, h->stream);
  if (h->plan.kind >= 8 && h->plan.kind <= 10) return launch_pcg_amg(a, h->plan, h->stream);
  if (h->plan.kind == 11) return launch_pcg_amg_cluster(a, h->plan, h->stream);
  if (h->plan.kind == 5 || h->plan.kind == 6) return launch_pcg_cluster(a, h->plan, h->clay, h->stream);
  return launch_pcg_fp64(a, h->plan, h->stream);
}

cudaError_t enqueue_pcg_only(avip_mesh* h) { return enqueue_solver(h, pcg_args(h)); }

// Queue one Poisson solve (cooperative PCG launch).
cudaError_t enqueue_poisson(avip_mesh* h) {
  cudaError_t e = cudaMemsetAsync(h->sync, 0, h->sync_bytes, h->stream);
  if (e != cudaSuccess) return e;
  return enqueue_pcg_only(h);
}

// Per photoionisation term, the Krylov vectors of a side-by-side solve: x, b, r, p, q, r2, z
// and the five of BiCGStab.
constexpr int kPhotoWork = 12;

// First block of term j's group in the side-by-side solve (the grid split as evenly as possible).
// 1 / V_i per node (V_i > 0 for every node of a valid mesh).
std::vector<double> inverse_volumes(const std::vector<double>& vol) {
  std::vector<double> r(vol.size());
  for (size_t i = 0; i < vol.size(); ++i) r[i] = 1.0 / vol[i];
  return r;
}

int photo_group_start(const avip_mesh* h, int j) {
  return (int)((int64_t)j * h->plan.blocks / h->ph.photo_terms);
}

// Arguments of the solve of photoionisation term j: the same solver and sparsity as the
// Poisson problem, the term's scaled Helmholtz values, b = rhs_j * (ionisation rate), zero
// Dirichlet values, results reported to the auxiliary block.
PcgArgs photo_args(const avip_mesh* h, int j) {
  PcgArgs a = pcg_args(h);
  const avip_mesh::PhotoTerm& t = h->photo[j];
  a.A.aval = t.aval;
  a.dsq = t.dsq;
  a.dsqinv = t.dsqinv;
  a.rhs_scale = t.rhs;
  a.lift = h->photo_zero;
  a.rhs_src = h->photo_I;
  a.phi = h->photo_psi + (size_t)j * h->Npad;
  a.phi1 = h->photo_psi + (size_t)(h->ph.photo_terms + kPredictorHistory * j) * h->Npad;  // own history
  a.phi2 = a.phi1 + h->Npad;
  a.phi3 = a.phi2 + h->Npad;
  a.hist = h->photo_hist + j;
  a.res = h->sc_aux + j;
  a.v_rise = 0.0;
  a.amg = t.amg;
  a.amg32 = t.amg32;
  if (h->photo_group) {  // own vectors and barrier state: the terms run at the same time
    const size_t Np = (size_t)h->Npad;
    double* w = h->photo_work + (size_t)j * kPhotoWork * Np;
    a.x = w;
    a.b = w + Np;
    a.r = w + 2 * Np;
    a.p = w + 3 * Np;
    a.q_ap = w + 4 * Np;
    a.r2 = w + 5 * Np;
    a.z = w + 6 * Np;
    a.bcg = w + 7 * Np;  // 5 vectors
    a.rq32 = h->photo_rq32 ? h->photo_rq32 + (size_t)j * 3 * Np : nullptr;
    a.sync = h->photo_gs + j;
    a.flags = &h->photo_gs[j].count;
    a.parts = h->parts + (size_t)8 * photo_group_start(h, j);
  }
  return a;
}

// The photoionisation solves and the source update that follows them: side by side in one
// launch (whole-GPU AMG solvers), else one after another.
cudaError_t enqueue_photo(avip_mesh* h, const DDArgs& a, bool auto_dt) {
  cudaError_t e = cudaSuccess;
  const int n = h->ph.photo_terms;
  if (h->photo_group) {
    AmgGroupArgs g;
    std::memset(&g, 0, sizeof(g));
    g.n = n;
    for (int j = 0; j < n; ++j) {
      g.a[j] = photo_args(h, j);
      g.start[j] = photo_group_start(h, j);
    }
    g.start[n] = h->plan.blocks;
    e = cudaMemsetAsync(h->photo_gs, 0, (size_t)n * sizeof(GridSync), h->stream);
    if (e == cudaSuccess) e = launch_amg_group(g, h->plan, h->stream);
  } else {
    for (int j = 0; j < n && e == cudaSuccess; ++j) {
      e = cudaMemsetAsync(h->sync, 0, h->sync_bytes, h->stream);
      if (e == cudaSuccess) e = enqueue_solver(h, photo_args(h, j));
    }
  }
  if (e == cudaSuccess) e = launch_photo_add(a, auto_dt ? 1 : 0, h->stream);
  return e;
}

// Queue one explicit step (no host synchronisation).
cudaError_t enqueue_step(avip_mesh* h) {
  NvtxRange step("avip.step");
  cudaError_t e;
  {
    NvtxRange r("avip.poisson_solve");
    if ((e = enqueue_poisson(h)) != cudaSuccess) return e;
  }
  DDArgs a = dd_args(h);
  const bool auto_dt = !(h->ph.dt_fixed > 0.0);
  const bool photo = h->ph.photo_terms > 0;
  {
    NvtxRange r("avip.node_fields");
    if ((e = launch_node_fields(a, auto_dt && !photo ? 1 : 0, h->stream)) != cudaSuccess) return e;
  }
  if (photo) {
    NvtxRange r("avip.photoionisation");
    if ((e = enqueue_photo(h, a, auto_dt)) != cudaSuccess) return e;
  }
  if (auto_dt) {
    NvtxRange r("avip.dt_cells");
    if ((e = launch_dt_cells(a, h->stream)) != cudaSuccess) return e;
  }
  {
    NvtxRange r("avip.fluxes_update");
    if ((e = launch_flux_update(a, h->stream)) != cudaSuccess) return e;
  }
  NvtxRange r("avip.finalize");
  return launch_finalize(h->sc, h->qpart, h->nparts, h->stream);
}

int read_scalars(avip_mesh* h, DevScalars& out) {
  cudaError_t e = cudaMemcpyAsync(&out, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return cuda_status(e);
}

bool ready(const avip_mesh* h) { return h && h->ph.ns > 0 && h->species_declared == h->ph.ns; }

void invalidate_graph(avip_mesh* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->graph_valid = false;
}

// Device copy of the AMG hierarchy with values of type T (float by default, or double): per
// non-coarsest level the composite operators Q, Rf, U, Pf in SELL-32 and the vectors xp (and,
// below the finest level, x and b); the coarsest level's x, b and its dense inverse.
template <typename T>
bool upload_amg_t(avip_mesh* h, const AmgHost& H, AmgDevT<T>*& out, bool record = true) {
  AmgDevT<T> D;
  std::memset(&D, 0, sizeof(D));
  D.nlev = (int32_t)H.lv.size();
  D.nc = H.nc;
  auto put = [&](const Csr& M, SellMatT<T>& dst, int64_t& steps) {
    SellHost S;
    sell_from_csr(M, S, lanes_per_row(M));
    int32_t *slp = nullptr, *slw = nullptr, *rl = nullptr, *col = nullptr;
    T* val = nullptr;
    std::vector<T> v(S.val.begin(), S.val.end());
    const bool ok = upload(h, slp, S.sl_ptr) && upload(h, slw, S.sl_w) && upload(h, rl, S.rlen) &&
                    upload(h, col, S.col, 1) && upload(h, val, v, 1);
    dst = SellMatT<T>{slp, slw, rl, col, val, S.n, S.nslices, S.lpr};
    steps = S.sl_ptr.back() / kSlice;
    return ok;
  };
  // [U | Pf]: Pf's columns shifted past U's n columns
  auto concat = [](const Csr& Uo, const Csr& Pfo) {
    Csr C;
    C.n = Uo.n;
    C.m = Uo.m + Pfo.m;
    C.rp.assign(C.n + 1, 0);
    for (int32_t i = 0; i < C.n; ++i) {
      for (int32_t e = Uo.rp[i]; e < Uo.rp[i + 1]; ++e) {
        C.ci.push_back(Uo.ci[e]);
        C.v.push_back(Uo.v[e]);
      }
      for (int32_t e = Pfo.rp[i]; e < Pfo.rp[i + 1]; ++e) {
        C.ci.push_back(Uo.m + Pfo.ci[e]);
        C.v.push_back(Pfo.v[e]);
      }
      C.rp[i + 1] = (int32_t)C.ci.size();
    }
    return C;
  };
  bool ok = true;
  for (int32_t l = 0; l < D.nlev && ok; ++l) {
    const AmgHostLevel& L = H.lv[l];
    AmgLevelT<T>& dl = D.L[l];
    dl.n = L.A.n;
    const size_t npad = (size_t)((L.A.n + kSlice - 1) / kSlice) * kSlice;
    int64_t rf_steps = 0, up_steps = 0;
    if (l + 1 < D.nlev) {
      T* qd = nullptr;
      std::vector<T> qv(L.Q.v.begin(), L.Q.v.end());  // Q is diagonal: one entry per row, in order
      ok = ok && upload(h, qd, qv, npad) && put(L.Rf, dl.Rf, rf_steps) && put(concat(L.U, L.Pf), dl.UP, up_steps) &&
           zalloc(h, dl.xp, npad);
      dl.qd = qd;
    }
    if (l > 0) ok = ok && zalloc(h, dl.x, npad) && zalloc(h, dl.b, npad);
  }
  T* cinv = nullptr;
  std::vector<T> cv(H.cinv.begin(), H.cinv.end());
  ok = ok && upload(h, cinv, cv, 1);
  D.cinv = cinv;
  auto* dd = static_cast<AmgDevT<T>*>(dev_alloc(h, sizeof(D)));
  ok = ok && dd && cudaMemcpyAsync(dd, &D, sizeof(D), cudaMemcpyHostToDevice, h->stream) == cudaSuccess &&
       cudaStreamSynchronize(h->stream) == cudaSuccess;
  out = dd;
  if (!record) return ok;
  h->amg_levels = D.nlev;
  h->amg_stats.clear();
  for (const AmgHostLevel& L : H.lv) {
    auto nz = [](const Csr& M) -> int64_t { return M.rp.empty() ? 0 : M.rp[M.n]; };
    for (int64_t v : {(int64_t)L.A.n, nz(L.A), nz(L.P), nz(L.Rf), nz(L.U), nz(L.Pf)}) h->amg_stats.push_back(v);
  }
  return ok;
}

// Upload the hierarchy in the handle's preconditioner precision (FP64 values when asked for and
// the solve is not the mixed-precision one) with its preconditioned-residual vector.
bool upload_amg(avip_mesh* h, const AmgHost& H, size_t Np) {
  const bool fp64 = h->opts.precond_fp64 && h->opts.precision == AVIP_PREC_FP64;
  if (fp64) return upload_amg_t<double>(h, H, h->amg) && zalloc(h, h->amg_z, Np) && zalloc(h, h->r2, Np);
  // (the FP64 CG writes its preconditioned residual in FP64 whatever the hierarchy's type; the
  // mixed-precision solve keeps its own FP32 one)
  return upload_amg_t<float>(h, H, h->amg32) && zalloc(h, h->z32, Np) && zalloc(h, h->amg_z, Np) &&
         zalloc(h, h->r2, Np) && zalloc(h, h->rq32, 3 * Np);
}

}  // namespace

extern "C" {

int avip_opts_default(avip_opts* o) {
  if (!o) return AVIP_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->cfl = 0.4;
  o->fourier = 0.25;
  o->a_diel = 0.5;
  o->a_chem = 0.2;
  o->beta = 1.0;
  o->limiter = AVIP_LIM_SWEBY;
  o->precision = AVIP_PREC_FP64;
  o->rtol = 1e-12;
  o->max_iter = 20000;
  o->reorder = 1;
  o->dt_fixed = 0.0;
  o->inner_rtol = 1e-4;
  o->wait_timeout = 2.0;
  return AVIP_OK;
}

// Accepted range of a device-wait limit (seconds).
static bool wait_timeout_ok(double s) { return s >= 0.0 && s <= 60.0; }

const char* avip_status_str(int s) {
  switch (s) {
    case AVIP_OK: return "ok";
    case AVIP_EINVAL: return "invalid argument";
    case AVIP_ENOMEM: return "device allocation failed";
    case AVIP_ENOTCONV: return "PCG did not converge within max_iter";
    case AVIP_ENAN: return "non-finite value detected";
    case AVIP_ECUDA: return "CUDA runtime error";
    case AVIP_ETIMEOUT: return "device wait timed out";
    case AVIP_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* avip_last_error(void) { return g_err; }

int mesh_create(const double* xy, int32_t n_nodes, const int32_t* tris, int32_t n_tris,
                const int32_t* node_bc, const double* phi_D, const avip_opts* opts, avip_mesh_t* out) {
  return mesh_create_hybrid(xy, n_nodes, tris, n_tris, nullptr, 0, node_bc, phi_D, opts, out);
}

int mesh_create_hybrid(const double* xy, int32_t n_nodes, const int32_t* tris, int32_t n_tris,
                       const int32_t* quads, int32_t n_quads, const int32_t* node_bc, const double* phi_D,
                       const avip_opts* opts, avip_mesh_t* out) {
  if (!out) return AVIP_EINVAL;
  *out = nullptr;
  avip_mesh* h = new (std::nothrow) avip_mesh();
  if (!h) return AVIP_ENOMEM;
  if (opts)
    h->opts = *opts;
  else
    avip_opts_default(&h->opts);
  if ((h->opts.alloc == nullptr) != (h->opts.free == nullptr) || !(h->opts.rtol > 0) || h->opts.max_iter < 1 ||
      !(h->opts.v_rise >= 0) || !std::isfinite(h->opts.v_rise) || !wait_timeout_ok(h->opts.wait_timeout) ||
      (h->opts.cluster_size != 0 && h->opts.cluster_size != 2 && h->opts.cluster_size != 4 &&
       h->opts.cluster_size != 8 && h->opts.cluster_size != 16) ||
      (h->opts.scheme != AVIP_FLUX_LLW && h->opts.scheme != AVIP_FLUX_SG) ||
      (h->opts.precision != AVIP_PREC_FP64 && h->opts.precision != AVIP_PREC_MIXED) ||
      (h->opts.precision == AVIP_PREC_MIXED && !(h->opts.inner_rtol > 0 && h->opts.inner_rtol < 1))) {
    delete h;
    return AVIP_EINVAL;
  }
  // the axisymmetric matrix is not symmetric: only BiCGStab (kind 7, FP64) applies
  const bool axi = h->opts.geometry == AVIP_GEOM_AXISYMMETRIC;
  if (axi && (h->opts.precision != AVIP_PREC_FP64 ||
              (h->opts.pcg_kind != 0 && h->opts.pcg_kind != 7 && h->opts.pcg_kind != 9))) {
    std::snprintf(g_err, sizeof(g_err),
                  "axisymmetric meshes need precision FP64 and pcg_kind 0, 7 or 9 (BiCGStab, Jacobi or AMG)");
    delete h;
    return AVIP_EINVAL;
  }
  if ((h->opts.pcg_kind >= 7 && h->opts.pcg_kind <= 9 && h->opts.precision != AVIP_PREC_FP64) ||
      (h->opts.pcg_kind == 10 && h->opts.precision != AVIP_PREC_MIXED)) {
    delete h;
    return AVIP_EINVAL;
  }
  // host-side validation and metrics first: bad meshes are rejected without touching the GPU
  int st = prepare_mesh(xy, n_nodes, tris, n_tris, quads, n_quads, node_bc, phi_D, h->opts.reorder,
                        h->opts.geometry, h->hm, g_err, sizeof(g_err));
  if (st != AVIP_OK) {
    delete h;
    return st;
  }
  h->stream = static_cast<cudaStream_t>(h->opts.stream);
  if (!h->stream) {
    // a private stream keeps the step graph-capturable
    cudaError_t ce = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
      int rc = cuda_status(ce);
      delete h;
      return rc;
    }
    h->own_stream = true;
  }
  HostMesh& m = h->hm;
  h->Npad = m.nslices * kSlice;
  const size_t Np = (size_t)h->Npad;
  bool ok = upload(h, h->sl_ptr, m.sl_ptr) && upload(h, h->sl_w, m.sl_w) && upload(h, h->rlen, m.rlen) &&
            upload(h, h->col, m.col) && upload(h, h->aval, m.aval) && upload(h, h->gx, m.gx) &&
            upload(h, h->gy, m.gy) && upload(h, h->sx, m.sx) && upload(h, h->sy, m.sy) &&
            upload(h, h->cell, m.cell) && upload(h, h->flen, m.flen) && upload(h, h->cw, m.cw) && upload(h, h->e_lo, m.e_lo, 1) && upload(h, h->e_hi, m.e_hi, 1) &&
            upload(h, h->e_sx, m.e_sx, 1) && upload(h, h->e_sy, m.e_sy, 1) && upload(h, h->slot_eid, m.slot_eid) &&
            zalloc(h, h->eflux, (size_t)AVIP_MAX_SPECIES * std::max<size_t>(m.e_lo.size(), 1)) && upload(h, h->x, m.x, Np) &&
            upload(h, h->y, m.y, Np) && upload(h, h->vol, m.vol, Np) && upload(h, h->ivol, inverse_volumes(m.vol), Np) && upload(h, h->dsq, m.dsq, Np) && upload(h, h->dsqinv, m.dsqinv, Np) &&
            upload(h, h->lift, m.lift, Np) && upload(h, h->rhs_scale, m.rhs_scale, Np);
  // initial potential: Dirichlet values on Dirichlet rows, zero elsewhere
  std::vector<double> phi0(Np, 0.0);
  for (int32_t i = 0; i < m.N; ++i)
    if (m.bc[i] == 1) phi0[i] = h->opts.v_rise > 0 ? 0.0 : m.lift[i];  // a ramp starts at 0 V
  ok = ok && upload(h, h->phi, phi0) && upload(h, h->phi1, phi0) && upload(h, h->phi2, phi0) && upload(h, h->phi3, phi0) && zalloc(h, h->b, Np) && zalloc(h, h->r, Np) && zalloc(h, h->xs, Np) &&
       zalloc(h, h->p, Np) && zalloc(h, h->q, Np) && zalloc(h, h->nbuf, 2 * AVIP_MAX_SPECIES * Np) &&
       zalloc(h, h->ndat, 4 * AVIP_MAX_SPECIES * Np) && zalloc(h, h->nm, AVIP_MAX_SPECIES * Np) &&
       zalloc(h, h->src, AVIP_MAX_SPECIES * Np) && zalloc(h, h->Ex, Np) && zalloc(h, h->Ey, Np);
  if (!ok) {
    dev_free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return AVIP_ENOMEM;
  }
  // persistent PCG grid: co-resident blocks, but no more than there are slices to share
  // persistent PCG grid (co-resident blocks): register-resident kernel when the mesh fits
  h->plan = h->opts.precision == AVIP_PREC_MIXED ? pcg_mixed_plan(m.nslices, h->opts.pcg_threads)
                                                 : pcg_plan(m.nslices, h->opts.pcg_kind, h->opts.pcg_threads);
  const bool bicg = axi || h->opts.pcg_kind == 7 || h->opts.pcg_kind == 9;
  // BiCGStab preconditioned by the AMG V-cycle: forced, or automatic above the cluster size
  const bool bicg_amg = bicg && (h->opts.pcg_kind == 9 || (h->opts.pcg_kind == 0 && m.N > kClusterAutoRows));
  if (bicg) {
    h->plan = bicgstab_plan(m.nslices, h->opts.pcg_threads);
    ok = ok && zalloc(h, h->bcg, (bicg_amg ? 5 : 3) * Np);
  } else if (h->opts.pcg_kind == 0 || h->opts.pcg_kind == 5 || h->opts.pcg_kind == 6) {
    // small meshes: one thread-block cluster with everything in shared memory
    const int mixed = h->opts.precision == AVIP_PREC_MIXED ? 1 : 0;
    ClusterHost chd;
    PcgPlan cp = pcg_cluster_plan(m, h->opts.pcg_kind >= 5 ? (1 << 30) : kClusterAutoRows, &h->clay, &chd, mixed);
    if (cp.kind == 5 || cp.kind == 6) {
      int32_t *colL = nullptr, *pptr = nullptr, *pdst = nullptr;
      ok = ok && upload(h, colL, chd.colL) && upload(h, pptr, chd.push_ptr) && upload(h, pdst, chd.push_dst, 1);
      h->clay.colL = colL;
      h->clay.push_ptr = pptr;
      h->clay.push_dst = pdst;
      h->plan = cp;
    }
  }
  // large FP64 meshes (or kinds 8/9 forced): CG (planar) or BiCGStab (axisymmetric)
  // preconditioned by an AMG V-cycle
  if (bicg_amg || (!bicg && h->opts.precision == AVIP_PREC_FP64 &&
                   (h->opts.pcg_kind == 8 || (h->opts.pcg_kind == 0 && h->plan.kind != 5)))) {
    AmgHost H;
    int rc = amg_setup(m, H, g_err, sizeof(g_err));
    if (rc != AVIP_OK) {
      dev_free_all(h);
      if (h->own_stream) cudaStreamDestroy(h->stream);
      delete h;
      return rc;
    }
    ok = ok && upload_amg(h, H, Np);
    h->plan = amg_plan(m.nslices, h->opts.pcg_threads, bicg ? 9 : 8, h->amg ? 1 : 0);
  }
  if (h->opts.precision == AVIP_PREC_MIXED) {
    std::vector<float> a32(m.aval.begin(), m.aval.end());
    ok = ok && upload(h, h->aval32, a32) && zalloc(h, h->e32, Np) && zalloc(h, h->r32, Np) && zalloc(h, h->p32, Np) &&
         zalloc(h, h->q32, Np);
    // FP32 drift-diffusion stage: gradient weights and edge normals rounded once
    std::vector<float> f(m.gx.begin(), m.gx.end());
    ok = ok && upload(h, h->gx32, f);
    f.assign(m.gy.begin(), m.gy.end());
    ok = ok && upload(h, h->gy32, f);
    f.assign(m.sx.begin(), m.sx.end());
    ok = ok && upload(h, h->sx32, f);
    f.assign(m.sy.begin(), m.sy.end());
    ok = ok && upload(h, h->sy32, f) && zalloc(h, h->ndat32, 4 * AVIP_MAX_SPECIES * Np);
  }
  // large mixed-precision meshes (or kind 10 forced): FP32 inner CG preconditioned by an FP32
  // AMG V-cycle, FP64 iterative refinement of the residual
  if (h->opts.precision == AVIP_PREC_MIXED && !bicg &&
      (h->opts.pcg_kind == 10 || (h->opts.pcg_kind == 0 && h->plan.kind != 6))) {
    AmgHost H;
    int rc = amg_setup(m, H, g_err, sizeof(g_err));
    if (rc != AVIP_OK) {
      dev_free_all(h);
      if (h->own_stream) cudaStreamDestroy(h->stream);
      delete h;
      return rc;
    }
    ok = ok && upload_amg(h, H, Np);
    h->plan = amg_plan(m.nslices, h->opts.pcg_threads, 10, 0);
  }
  // mid-size planar meshes (or kind 11 forced): the AMG-preconditioned solve on one cluster
  if (!bicg && (h->opts.pcg_kind == 11 ||
                (h->opts.pcg_kind == 0 && m.N > kClusterAmgMinRows && m.N <= kClusterAutoRows))) {
    const PcgPlan cp = amg_cluster_plan(h->opts.cluster_size, m.N);
    if (cp.kind == 11) {
      AmgHost H;
      int rc = amg_setup(m, H, g_err, sizeof(g_err));
      if (rc != AVIP_OK) {
        dev_free_all(h);
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return rc;
      }
      ok = ok && upload_amg(h, H, Np);
      h->plan = cp;
    }
  }
  h->nparts = flux_blocks(m.N);
  h->sync_bytes = sizeof(GridSync) + sizeof(unsigned) * (size_t)(h->plan.blocks + 1);
  ok = ok && zalloc(h, h->parts, (size_t)h->plan.blocks * 8) &&
       zalloc(h, h->qpart, (size_t)std::max(h->nparts, flux_partials_max(m.N))) &&
       zalloc(h, h->sync, (h->sync_bytes + sizeof(GridSync) - 1) / sizeof(GridSync)) && zalloc(h, h->sc, 1);
  if (ok) h->flags = reinterpret_cast<unsigned*>(h->sync + 1);
  if (!ok) {
    dev_free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return AVIP_ENOMEM;
  }
  DevScalars s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.dt_bits = 0x7ff0000000000000ULL;  // +inf
  s0.run_dt_min = INFINITY;
  cudaError_t e = cudaMemcpyAsync(h->sc, &s0, sizeof(s0), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    int rc = cuda_status(e);
    dev_free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return rc;
  }
  std::memset(&h->ph, 0, sizeof(h->ph));
  h->ph.beta = h->opts.beta;
  h->ph.limiter = h->opts.limiter;
  h->ph.scheme = h->opts.scheme;
  h->ph.dd_fp32 = h->opts.precision == AVIP_PREC_MIXED ? 1 : 0;
  h->ph.cfl = h->opts.cfl;
  h->ph.fourier = h->opts.fourier;
  h->ph.a_diel = h->opts.a_diel;
  h->ph.a_chem = h->opts.a_chem;
  h->ph.dt_fixed = h->opts.dt_fixed;
  h->ph.src_idx[0] = 0;
  h->ph.src_idx[1] = 1;
  h->ph.src_idx[2] = -1;
  *out = h;
  return AVIP_OK;
}

int mesh_destroy(avip_mesh_t h) {
  if (!h) return AVIP_OK;
  cudaStreamSynchronize(h->stream);
  invalidate_graph(h);
  dev_free_all(h);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return AVIP_OK;
}

int mesh_set_stream(avip_mesh_t h, void* stream) {
  if (!h) return AVIP_EINVAL;
  cudaStreamSynchronize(h->stream);
  if (!stream) return AVIP_OK;  // keep the current (private or given) stream
  if (h->own_stream) cudaStreamDestroy(h->stream);
  h->own_stream = false;
  h->stream = static_cast<cudaStream_t>(stream);
  invalidate_graph(h);
  return AVIP_OK;
}

int mesh_set_wait_timeout(avip_mesh_t h, double seconds) {
  if (!h || !wait_timeout_ok(seconds)) return AVIP_EINVAL;
  if (h->opts.wait_timeout != seconds) {
    h->opts.wait_timeout = seconds;
    invalidate_graph(h);  // the captured step carries the old limit in its kernel arguments
  }
  return AVIP_OK;
}

int mesh_info(avip_mesh_t h, int64_t* info) {
  if (!h || !info) return AVIP_EINVAL;
  info[0] = h->hm.N;
  info[1] = h->hm.T;
  info[2] = h->hm.E;
  info[3] = h->hm.nnz;
  info[4] = h->plan.kind;
  info[5] = h->plan.blocks;
  info[6] = h->plan.tpb;
  info[7] = (int64_t)h->bytes;
  return AVIP_OK;
}

int solver_levels(avip_mesh_t h, int64_t* out, int32_t max_levels) {
  if (!h || (max_levels > 0 && !out) || max_levels < 0) return AVIP_EINVAL;
  const int32_t nl = (h->plan.kind >= 8 && h->plan.kind <= 11) ? h->amg_levels : 0;
  for (int32_t l = 0; l < nl && l < max_levels; ++l)
    for (int k = 0; k < AVIP_LEVEL_STATS; ++k)
      out[AVIP_LEVEL_STATS * l + k] = h->amg_stats[AVIP_LEVEL_STATS * (size_t)l + k];
  return nl;
}

int species_set(avip_mesh_t h, int32_t s, int32_t charge, int32_t mob_model, const double* mob_params, double D,
                int32_t bnd_mode, const double* n0) {
  if (!h || s < 0 || s >= AVIP_MAX_SPECIES || !mob_params || !n0) return AVIP_EINVAL;
  if (s > h->species_declared) return AVIP_ESTATE;
  if ((charge != -1 && charge != 1) || (mob_model != AVIP_MOB_CONST && mob_model != AVIP_MOB_POWER) ||
      (bnd_mode != AVIP_BND_NEUMANN && bnd_mode != AVIP_BND_OUTFLOW) || !(D >= 0) || !std::isfinite(D))
    return AVIP_EINVAL;
  if (mob_model == AVIP_MOB_POWER && !(mob_params[1] > 0 && mob_params[3] > 0)) return AVIP_EINVAL;
  const HostMesh& m = h->hm;
  std::vector<double> nn(m.N);
  for (int32_t i = 0; i < m.N; ++i) {
    nn[i] = n0[m.perm[i]];
    if (!std::isfinite(nn[i])) return AVIP_ENAN;
  }
  SpeciesParams& sp = h->ph.sp[s];
  sp.q = (double)charge;
  for (int k = 0; k < 4; ++k) sp.mob[k] = mob_params[k];
  sp.D = D;
  sp.mob_log_ref = mob_model == AVIP_MOB_POWER ? std::log(mob_params[1]) : 0.0;
  sp.mob_model = mob_model;
  sp.bnd_mode = bnd_mode;
  if (s == h->species_declared) h->species_declared++;
  h->ph.ns = h->species_declared;
  // density into the current parity buffer
  DevScalars sc;
  int rc = read_scalars(h, sc);
  if (rc) return rc;
  double* dst = h->nbuf + ((size_t)sc.parity * AVIP_MAX_SPECIES + s) * h->Npad;
  cudaError_t e = cudaMemcpyAsync(dst, nn.data(), nn.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  invalidate_graph(h);
  return cuda_status(e);
}

int source_set(avip_mesh_t h, int32_t model, const double* params, const int32_t* idx) {
  if (!h) return AVIP_EINVAL;
  if (model == AVIP_SRC_NONE) {
    h->ph.src_model = 0;
    invalidate_graph(h);
    return AVIP_OK;
  }
  if (!params || !idx ||
      (model != AVIP_SRC_TOWNSEND && model != AVIP_SRC_TOWNSEND_ATTACH && model != AVIP_SRC_MORROW_LOWKE))
    return AVIP_EINVAL;
  if (idx[0] < 0 || idx[0] >= AVIP_MAX_SPECIES || idx[1] < 0 || idx[1] >= AVIP_MAX_SPECIES) return AVIP_EINVAL;
  const bool three = model != AVIP_SRC_TOWNSEND;
  if (three && (idx[2] < 0 || idx[2] >= AVIP_MAX_SPECIES || idx[2] == idx[0] || idx[2] == idx[1]))
    return AVIP_EINVAL;
  if (idx[0] == idx[1]) return AVIP_EINVAL;
  const int np = model == AVIP_SRC_MORROW_LOWKE ? 5 : 3;
  for (int k = 0; k < np; ++k)
    if (!(params[k] >= 0) || !std::isfinite(params[k])) return AVIP_EINVAL;
  h->ph.src_model = model;
  for (int k = 0; k < 5; ++k) h->ph.src_params[k] = k < np ? params[k] : 0.0;
  for (int k = 0; k < 3; ++k) h->ph.src_idx[k] = three || k < 2 ? idx[k] : -1;
  invalidate_graph(h);
  return AVIP_OK;
}

int photo_set(avip_mesh_t h, int32_t n_terms, const double* a, const double* kappa, double c) {
  if (!h || n_terms < 0 || n_terms > AVIP_MAX_PHOTO_TERMS || (n_terms > 0 && (!a || !kappa)) ||
      !(c >= 0) || !std::isfinite(c))
    return AVIP_EINVAL;
  for (int j = 0; j < n_terms; ++j)
    if (!(a[j] >= 0) || !std::isfinite(a[j]) || !(kappa[j] > 0) || !std::isfinite(kappa[j])) return AVIP_EINVAL;
  if (!h->photo.empty()) {
    std::snprintf(g_err, sizeof(g_err), "photoionisation terms can be set once per handle");
    return AVIP_ESTATE;
  }
  if (n_terms == 0) return AVIP_OK;
  const int kind = h->plan.kind;
  if (h->opts.precision != AVIP_PREC_FP64 || kind == 4 || kind == 6 || kind == 10) {
    std::snprintf(g_err, sizeof(g_err), "photoionisation needs the FP64 solvers");
    return AVIP_EINVAL;
  }
  const HostMesh& m = h->hm;
  const size_t Np = (size_t)h->Npad;
  const bool amg = kind == 8 || kind == 9 || kind == 11;
  // solutions of the terms, then two history vectors per term
  bool ok = zalloc(h, h->photo_psi, (size_t)(1 + kPredictorHistory) * n_terms * Np) && zalloc(h, h->photo_hist, n_terms) &&
            zalloc(h, h->photo_I, Np) &&
            zalloc(h, h->photo_S, Np) && zalloc(h, h->photo_zero, Np) && zalloc(h, h->sc_aux, n_terms);
  // side by side on the whole-GPU AMG solvers, when every term gets a group of blocks
  const bool group = (kind == 8 || kind == 9) && n_terms > 1 && h->plan.blocks >= n_terms;
  if (ok && group) {
    ok = zalloc(h, h->photo_work, (size_t)kPhotoWork * n_terms * Np) && zalloc(h, h->photo_gs, n_terms) &&
         (h->amg || kind == 9 || zalloc(h, h->photo_rq32, (size_t)3 * n_terms * Np));
  }
  for (int j = 0; j < n_terms && ok; ++j) {
    // (K + kappa_j^2 V) S_j = c a_j V I with S_j = 0 on the Dirichlet nodes: the unscaled
    // Poisson values are recovered from the scaled ones, the diagonal of the free rows gains
    // kappa_j^2 V_i, and the result is scaled symmetrically by its own diagonal.
    const double k2 = kappa[j] * kappa[j];
    std::vector<double> dh(Np, 1.0), dhinv(Np, 1.0), rhs(Np, 0.0), val(m.aval.size(), 0.0);
    for (int32_t i = 0; i < m.N; ++i)
      if (m.bc[i] != 1) {
        dh[i] = std::sqrt(m.dsq[i] * m.dsq[i] + k2 * m.vol[i]);
        dhinv[i] = 1.0 / dh[i];
        rhs[i] = c * a[j] * m.vol[i] * dhinv[i];
      }
    for (int32_t sl = 0; sl < m.nslices; ++sl)
      for (int l = 0; l < kSlice; ++l) {
        const int32_t i = sl * kSlice + l;
        if (i >= m.N) continue;
        for (int32_t k = 0; k < m.rlen[i]; ++k) {
          const int64_t e = (int64_t)m.sl_ptr[sl] + (int64_t)k * kSlice + l;
          const int32_t col = m.col[e];
          if (m.bc[i] == 1) {
            val[e] = k == 0 ? 1.0 : 0.0;
          } else if (k == 0) {
            val[e] = 1.0;
          } else {
            const double K = m.aval[e] * m.dsq[i] * m.dsq[col];
            val[e] = K / (dh[i] * dh[col]);
          }
        }
      }
    avip_mesh::PhotoTerm t;
    ok = upload(h, t.aval, val) && upload(h, t.dsq, dh) && upload(h, t.dsqinv, dhinv) && upload(h, t.rhs, rhs);
    if (ok && amg) {
      HostMesh hm;
      hm.N = m.N;
      hm.nslices = m.nslices;
      hm.geometry = m.geometry;
      hm.rlen = m.rlen;
      hm.sl_ptr = m.sl_ptr;
      hm.col = m.col;
      hm.bc = m.bc;
      hm.aval = std::move(val);
      hm.dsq.assign(dh.begin(), dh.begin() + m.N);
      AmgHost H;
      if (amg_setup(hm, H, g_err, sizeof(g_err)) != AVIP_OK) return AVIP_EINVAL;
      if (h->amg)
        ok = upload_amg_t<double>(h, H, t.amg, false);
      else
        ok = upload_amg_t<float>(h, H, t.amg32, false);
    }
    h->photo.push_back(t);
  }
  if (!ok) return AVIP_ENOMEM;
  h->ph.photo_terms = n_terms;
  h->photo_group = group;
  invalidate_graph(h);
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? AVIP_OK : AVIP_ECUDA;
}

int photo_stats(avip_mesh_t h, int32_t* n_terms, int32_t* iters, double* relres, int32_t* side_by_side) {
  if (!h || !n_terms || !side_by_side) return AVIP_EINVAL;
  const int n = h->ph.photo_terms;
  *n_terms = n;
  *side_by_side = h->photo_group ? 1 : 0;
  if (n == 0) return AVIP_OK;
  DevScalars st[AVIP_MAX_PHOTO_TERMS];
  cudaError_t e = cudaMemcpyAsync(st, h->sc_aux, (size_t)n * sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  for (int j = 0; j < n; ++j) {
    if (iters) iters[j] = st[j].pcg_iters;
    if (relres) relres[j] = st[j].pcg_relres;
  }
  return AVIP_OK;
}

int poisson_solve(avip_mesh_t h, int32_t* iters_out, double* relres_out) {
  if (!ready(h)) return h ? AVIP_ESTATE : AVIP_EINVAL;
  // clear the status a failed earlier run left (a solve is skipped while it says ENAN/ETIMEOUT)
  cudaError_t e = launch_run_reset(h->sc, h->stream);
  if (e == cudaSuccess) e = enqueue_poisson(h);
  if (e == cudaSuccess) e = launch_node_fields(dd_args(h), 0, h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  DevScalars sc;
  int rc = read_scalars(h, sc);
  if (rc) return rc;
  if (iters_out) *iters_out = sc.pcg_iters;
  if (relres_out) *relres_out = sc.pcg_relres;
  return sc.pcg_status;
}

static int run_impl(avip_mesh_t h, int32_t nsteps, double dt, avip_stats* stats, bool use_graph) {
  if (!ready(h)) return h ? AVIP_ESTATE : AVIP_EINVAL;
  if (nsteps < 0) return AVIP_EINVAL;
  DevScalars s0;
  int rc = read_scalars(h, s0);
  if (rc) return rc;
  const double saved_dt = h->ph.dt_fixed;
  if (dt > 0.0) {
    if (h->ph.dt_fixed != dt) invalidate_graph(h);
    h->ph.dt_fixed = dt;
  }
  cudaError_t e = launch_run_reset(h->sc, h->stream);
  if (use_graph && nsteps > 1 && e == cudaSuccess) {
    if (!h->graph_valid) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e2 = enqueue_step(h);
        e = cudaStreamEndCapture(h->stream, &g);
        if (e2 != cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e == cudaSuccess) {
        h->graph_valid = true;
      } else {
        cudaGetLastError();
        h->graph = nullptr;
        use_graph = false;  // capture unsupported here: launch the same kernels directly
        e = cudaSuccess;
      }
    }
    for (int32_t k = 0; k < nsteps && e == cudaSuccess && use_graph; ++k) {
      NvtxRange r("avip.step_graph");
      e = cudaGraphLaunch(h->graph, h->stream);
    }
    if (!use_graph)
      for (int32_t k = 0; k < nsteps && e == cudaSuccess; ++k) e = enqueue_step(h);
  } else {
    for (int32_t k = 0; k < nsteps && e == cudaSuccess; ++k) e = enqueue_step(h);
  }
  h->ph.dt_fixed = saved_dt;
  if (dt > 0.0 && saved_dt != dt) invalidate_graph(h);
  if (e != cudaSuccess) return cuda_status(e);
  DevScalars sc;
  rc = read_scalars(h, sc);
  if (rc) return rc;
  if (stats) {
    stats->steps = sc.run_steps;
    stats->pcg_iters_total = sc.run_iters_total;
    stats->pcg_iters_max = sc.run_iters_max;
    stats->status = sc.status;
    stats->dt_min = sc.run_dt_min;
    stats->dt_max = sc.run_dt_max;
    stats->t = sc.t;
    stats->charge = sc.charge;
    stats->charge_start = s0.charge;
    stats->relres_max = sc.run_relres_max;
  }
  if (sc.status == AVIP_ETIMEOUT) {
    // leave the handle usable: clear the barrier state
    cudaMemsetAsync(h->sync, 0, h->sync_bytes, h->stream);
    cudaStreamSynchronize(h->stream);
  }
  return sc.status;
}

int dd_step(avip_mesh_t h, double dt, double* dt_used) {
  avip_stats st;
  int rc = run_impl(h, 1, dt, &st, false);
  if (dt_used) *dt_used = st.dt_max;
  return rc;
}

int run_steps(avip_mesh_t h, int32_t nsteps, avip_stats* stats) { return run_impl(h, nsteps, 0.0, stats, true); }

// Eager launches with CUDA events around every kernel on the handle's stream: all steps are
// queued first (the events of each step in their own slots), the call then waits once for the
// last event and adds up the intervals, so the device runs the steps back to back.
int run_steps_timed(avip_mesh_t h, int32_t nsteps, double* kernel_ms, avip_stats* stats) {
  if (!ready(h)) return h ? AVIP_ESTATE : AVIP_EINVAL;
  if (nsteps < 0 || !kernel_ms) return AVIP_EINVAL;
  for (int k = 0; k < AVIP_TIMED_KERNELS; ++k) kernel_ms[k] = 0.0;
  DevScalars s0;
  int rc = read_scalars(h, s0);
  if (rc) return rc;
  constexpr int kEv = 8;  // per step: 6 boundaries of the timed stages, 2 around photoionisation
  std::vector<cudaEvent_t> ev((size_t)nsteps * kEv, nullptr);
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  if (e == cudaSuccess) e = launch_run_reset(h->sc, h->stream);
  const bool auto_dt = !(h->ph.dt_fixed > 0.0);
  const bool photo = h->ph.photo_terms > 0;
  for (int32_t step = 0; step < nsteps && e == cudaSuccess; ++step) {
    NvtxRange r("avip.step_timed");
    cudaEvent_t* E = ev.data() + (size_t)step * kEv;
    DDArgs a = dd_args(h);
    e = cudaMemsetAsync(h->sync, 0, h->sync_bytes, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(E[0], h->stream);
    if (e == cudaSuccess) e = enqueue_pcg_only(h);
    if (e == cudaSuccess) e = cudaEventRecord(E[1], h->stream);
    if (e == cudaSuccess) e = launch_node_fields(a, auto_dt && !photo ? 1 : 0, h->stream);
    // the photoionisation solves and source update are timed on their own
    if (e == cudaSuccess && photo) e = cudaEventRecord(E[6], h->stream);
    if (e == cudaSuccess && photo) e = enqueue_photo(h, a, auto_dt);
    if (e == cudaSuccess && photo) e = cudaEventRecord(E[7], h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(E[2], h->stream);
    if (e == cudaSuccess && auto_dt) e = launch_dt_cells(a, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(E[3], h->stream);
    if (e == cudaSuccess) e = launch_flux_update(a, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(E[4], h->stream);
    if (e == cudaSuccess) e = launch_finalize(h->sc, h->qpart, h->nparts, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(E[5], h->stream);
  }
  if (e == cudaSuccess && nsteps > 0) e = cudaEventSynchronize(ev[(size_t)(nsteps - 1) * kEv + 5]);
  for (int32_t step = 0; step < nsteps && e == cudaSuccess; ++step) {
    cudaEvent_t* E = ev.data() + (size_t)step * kEv;
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, E[k], E[k + 1]);
      kernel_ms[k] += ms;
    }
    if (e == cudaSuccess && photo) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, E[6], E[7]);
      kernel_ms[5] += ms;
      kernel_ms[1] -= ms;
    }
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_status(e);
  DevScalars sc;
  rc = read_scalars(h, sc);
  if (rc) return rc;
  if (stats) {
    stats->steps = sc.run_steps;
    stats->pcg_iters_total = sc.run_iters_total;
    stats->pcg_iters_max = sc.run_iters_max;
    stats->status = sc.status;
    stats->dt_min = sc.run_dt_min;
    stats->dt_max = sc.run_dt_max;
    stats->t = sc.t;
    stats->charge = sc.charge;
    stats->charge_start = s0.charge;
    stats->relres_max = sc.run_relres_max;
  }
  return sc.status;
}

static int to_host_perm(avip_mesh_t h, const double* dev, double* host_out) {
  std::vector<double> tmp(h->hm.N);
  cudaError_t e = cudaMemcpyAsync(tmp.data(), dev, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  for (int32_t i = 0; i < h->hm.N; ++i) host_out[h->hm.perm[i]] = tmp[i];
  return AVIP_OK;
}

int field_get(avip_mesh_t h, int32_t which, int32_t s, double* host_out) {
  if (!h || !host_out) return AVIP_EINVAL;
  switch (which) {
    case AVIP_FIELD_PHI: return to_host_perm(h, h->phi, host_out);
    case AVIP_FIELD_EX: return to_host_perm(h, h->Ex, host_out);
    case AVIP_FIELD_EY: return to_host_perm(h, h->Ey, host_out);
    case AVIP_FIELD_VOLUME: return to_host_perm(h, h->vol, host_out);
    case AVIP_FIELD_PHOTO:
      if (!h->photo_S) return AVIP_ESTATE;
      return to_host_perm(h, h->photo_S, host_out);
    case AVIP_FIELD_DENSITY: {
      if (s < 0 || s >= h->ph.ns) return AVIP_EINVAL;
      DevScalars sc;
      int rc = read_scalars(h, sc);
      if (rc) return rc;
      return to_host_perm(h, h->nbuf + ((size_t)sc.parity * AVIP_MAX_SPECIES + s) * h->Npad, host_out);
    }
    default: return AVIP_EINVAL;
  }
}

int state_size(avip_mesh_t h, int64_t* n) {
  if (!h || !n) return AVIP_EINVAL;
  *n = (int64_t)(h->ph.ns + 1 + kPredictorHistory) * h->hm.N + 2;
  return AVIP_OK;
}

// Device buffers of the checkpoint copies; false if they cannot be allocated.
static bool state_buffers(avip_mesh* h) {
  if (h->d_stage) return true;
  int64_t n = 0;
  state_size(h, &n);
  return upload(h, h->d_perm, h->hm.perm) && zalloc(h, h->d_stage, (size_t)n) && zalloc(h, h->d_state_flag, 1);
}

static StateArgs state_args(avip_mesh* h) {
  StateArgs s;
  std::memset(&s, 0, sizeof(s));
  s.N = h->hm.N;
  s.ns = h->ph.ns;
  s.Npad = h->Npad;
  s.perm = h->d_perm;
  s.stage = h->d_stage;
  s.nbuf = h->nbuf;
  s.phi = h->phi;
  s.phi1 = h->phi1;
  s.phi2 = h->phi2;
  s.phi3 = h->phi3;
  s.sc = h->sc;
  s.flag = h->d_state_flag;
  return s;
}

// One kernel writes the state in the caller's layout to device memory, one copy brings it to
// `out` (pinned host memory makes that copy a direct transfer).
int state_get(avip_mesh_t h, double* out) {
  if (!ready(h) || !out) return AVIP_EINVAL;
  if (!state_buffers(h)) return AVIP_ENOMEM;
  int64_t n = 0;
  state_size(h, &n);
  cudaError_t e = launch_state_take(state_args(h), h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->d_stage, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return cuda_status(e);
}

// One copy brings the caller's state to device memory, a kernel checks that every entry is
// finite (AVIP_ENAN, and nothing installed, otherwise), another installs it.
int state_set(avip_mesh_t h, const double* in) {
  if (!ready(h) || !in) return AVIP_EINVAL;
  const size_t N = (size_t)h->hm.N;
  const double hn = in[(size_t)(h->ph.ns + 1) * N + 1 + kPredictorHistory * N];
  if (!(hn >= 0.0 && hn <= (double)kPredictorHistory && hn == std::floor(hn))) return AVIP_EINVAL;
  if (!state_buffers(h)) return AVIP_ENOMEM;
  int64_t n = 0;
  state_size(h, &n);
  StateArgs sa = state_args(h);
  sa.t = in[(size_t)(h->ph.ns + 1) * N];
  sa.hist = (int32_t)hn;
  int32_t flag = 0;
  cudaError_t e = cudaMemcpyAsync(h->d_stage, in, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_state_flag, 0, sizeof(int32_t), h->stream);
  if (e == cudaSuccess) e = launch_state_check(sa, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, h->d_state_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (flag) return AVIP_ENAN;
  e = launch_state_put(sa, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return cuda_status(e);
}

}  // extern "C"

// ============================================================================================
// Batches: many independent discharge instances advanced together.  One step of a batch is
// one persistent cluster-resident PCG launch for every instance (each resident cluster solves
// instances in decreasing-size order) followed by one launch per drift-diffusion stage that
// covers every instance's nodes or cells; the step is captured once as a CUDA graph and
// replayed.  The cluster size is either given or picked by timing the candidates on the
// batch itself (state saved and restored around the trial).
namespace avip {
int cluster_batch_capacity(int C, size_t smem);
PcgPlan pcg_cluster_plan_fixed(const HostMesh& m, int C, ClusterLayout* out, ClusterHost* hd, int mixed);
cudaError_t launch_pcg_cluster_batch(const PcgArgs* args, const ClusterLayout* lays, const int32_t* order, int count,
                                     int C, int nclusters, size_t smem, cudaStream_t st);
cudaError_t launch_dd_batch(const DDArgs* args, const int32_t* node_pref, const int32_t* cell_pref, int count,
                            int node_blocks, int cell_blocks, int threads, cudaStream_t st);
cudaError_t launch_run_reset_batch(const DDArgs* args, int count, cudaStream_t st);
int dd_threads();
}  // namespace avip

struct avip_batch {
  std::vector<avip_mesh*> m;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  int C = 16, nclusters = 0;
  size_t smem = 0;
  PcgArgs* d_pargs = nullptr;
  ClusterLayout* d_lays = nullptr;
  DDArgs* d_dargs = nullptr;
  int32_t *d_order = nullptr, *d_npref = nullptr, *d_cpref = nullptr;
  int node_blocks = 0, cell_blocks = 0;
  int dd_threads = 256;  // threads per block of the drift-diffusion stages (autotuned)
  cudaGraphExec_t graph = nullptr;
  // per candidate cluster size: layouts (device arrays owned by the batch)
  std::vector<ClusterLayout> lays;
};

namespace {

void* batch_alloc(avip_batch* b, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  b->allocs.push_back(p);
  return p;
}

template <typename T>
T* batch_upload(avip_batch* b, const std::vector<T>& v) {
  T* d = static_cast<T*>(batch_alloc(b, v.size() * sizeof(T)));
  if (d && !v.empty() && cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return nullptr;
  return d;
}

void batch_free(avip_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
}

// Build the device tables for cluster size C; false if some instance does not fit.
bool batch_configure(avip_batch* b, int C) {
  const int n = (int)b->m.size();
  std::vector<ClusterLayout> lays(n);
  size_t smem = 0;
  for (int k = 0; k < n; ++k) {
    ClusterHost hd;
    if (b->m[k]->amg || b->m[k]->amg32) {
      // an AMG instance keeps its vectors in global memory: no shared-memory layout to fit
      std::memset(&lays[k], 0, sizeof(ClusterLayout));
      hd.colL.assign(1, 0);
      hd.push_ptr.assign(1, 0);
    } else {
      PcgPlan p = pcg_cluster_plan_fixed(b->m[k]->hm, C, &lays[k], &hd,
                                         b->m[k]->opts.precision == AVIP_PREC_MIXED ? 1 : 0);
      if (p.kind == 0) return false;
      smem = std::max(smem, (size_t)p.maxs);
    }
    lays[k].colL = batch_upload(b, hd.colL);
    lays[k].push_ptr = batch_upload(b, hd.push_ptr);
    std::vector<int32_t> pd = hd.push_dst;
    if (pd.empty()) pd.push_back(0);
    lays[k].push_dst = batch_upload(b, pd);
    if (!lays[k].colL || !lays[k].push_ptr || !lays[k].push_dst) return false;
  }
  const int cap = cluster_batch_capacity(C, smem);
  if (cap < 1) return false;
  b->C = C;
  b->smem = smem;
  b->nclusters = std::min(cap, n);
  b->lays = lays;
  b->d_lays = batch_upload(b, lays);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  return b->d_lays != nullptr;
}

// Partition of the drift-diffusion stages: T threads per block, each instance's nodes and cells
// in whole blocks (block prefix sums in instance order); false if the tables cannot be written.
bool batch_set_dd(avip_batch* b, int T) {
  const int count = (int)b->m.size();
  std::vector<int32_t> npref(count + 1, 0), cpref(count + 1, 0);
  for (int k = 0; k < count; ++k) {
    npref[k + 1] = npref[k] + (b->m[k]->hm.N + T - 1) / T;
    cpref[k + 1] = cpref[k] + (b->m[k]->hm.T + T - 1) / T;
  }
  if (cudaMemcpyAsync(b->d_npref, npref.data(), npref.size() * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->d_cpref, cpref.data(), cpref.size() * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  b->node_blocks = npref[count];
  b->cell_blocks = cpref[count];
  b->dd_threads = T;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  return true;
}

cudaError_t batch_enqueue_step(avip_batch* b) {
  cudaError_t e = launch_pcg_cluster_batch(b->d_pargs, b->d_lays, b->d_order, (int)b->m.size(), b->C, b->nclusters,
                                           b->smem, b->stream);
  if (e != cudaSuccess) return e;
  return launch_dd_batch(b->d_dargs, b->d_npref, b->d_cpref, (int)b->m.size(), b->node_blocks, b->cell_blocks,
                         b->dd_threads, b->stream);
}

// Save (dir = 0) or restore (dir = 1) every instance's densities, potential, predictor history
// and scalars.
cudaError_t batch_snapshot(avip_batch* b, std::vector<void*>& buf, int dir) {
  cudaError_t e = cudaSuccess;
  size_t j = 0;
  for (avip_mesh* h : b->m) {
    const size_t nb = (size_t)2 * AVIP_MAX_SPECIES * h->Npad * sizeof(double);
    const size_t pb = (size_t)h->Npad * sizeof(double);
    struct Item { void* dev; size_t bytes; } items[6] = {{h->nbuf, nb},  {h->phi, pb},  {h->phi1, pb},
                                                        {h->phi2, pb}, {h->phi3, pb}, {h->sc, sizeof(DevScalars)}};
    for (auto& it : items) {
      if (dir == 0) {
        void* p = batch_alloc(b, it.bytes);
        if (!p) return cudaErrorMemoryAllocation;
        buf.push_back(p);
        e = cudaMemcpyAsync(p, it.dev, it.bytes, cudaMemcpyDeviceToDevice, b->stream);
      } else {
        e = cudaMemcpyAsync(it.dev, buf[j++], it.bytes, cudaMemcpyDeviceToDevice, b->stream);
      }
      if (e != cudaSuccess) return e;
    }
  }
  return e;
}

}  // namespace

extern "C" {

int batch_create(const avip_mesh_t* meshes, int32_t count, int32_t cluster_size, avip_batch_t* out) {
  if (!meshes || count < 1 || !out ||
      (cluster_size != 0 && cluster_size != 2 && cluster_size != 4 && cluster_size != 8 && cluster_size != 16))
    return AVIP_EINVAL;
  *out = nullptr;
  avip_batch* b = new (std::nothrow) avip_batch();
  if (!b) return AVIP_ENOMEM;
  for (int k = 0; k < count; ++k) {
    avip_mesh* h = meshes[k];
    if (!ready(h)) {
      delete b;
      return h ? AVIP_ESTATE : AVIP_EINVAL;
    }
    if (h->plan.kind == 7 || h->plan.kind == 9 || h->ph.photo_terms > 0) {  // the batched solver is CG
      std::snprintf(g_err, sizeof(g_err), "batches take planar meshes solved by CG, without photoionisation");
      delete b;
      return AVIP_EINVAL;
    }
    cudaStreamSynchronize(h->stream);
    b->m.push_back(h);
  }
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return AVIP_ECUDA;
  }
  // argument tables, decreasing-size order, block prefix sums
  std::vector<PcgArgs> pa(count);
  std::vector<DDArgs> da(count);
  std::vector<int32_t> order(count), npref(count + 1, 0), cpref(count + 1, 0);
  for (int k = 0; k < count; ++k) {
    pa[k] = pcg_args(b->m[k]);
    da[k] = dd_args(b->m[k]);
    da[k].eflux = nullptr;  // batched flux kernel: each row evaluates its edges
    da[k].partials = b->m[k]->qpart;
    order[k] = k;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->m[x]->hm.N > b->m[y]->hm.N; });
  b->d_pargs = batch_upload(b, pa);
  b->d_dargs = batch_upload(b, da);
  b->d_order = batch_upload(b, order);
  b->d_npref = batch_upload(b, npref);
  b->d_cpref = batch_upload(b, cpref);
  if (!b->d_pargs || !b->d_dargs || !b->d_order || !b->d_npref || !b->d_cpref || !batch_set_dd(b, dd_threads())) {
    batch_free(b);
    cudaStreamDestroy(b->stream);
    delete b;
    return AVIP_ENOMEM;
  }
  bool ok = false;
  if (cluster_size != 0) {
    ok = batch_configure(b, cluster_size);
  } else {
    // autotune on the batch itself, then restore its state: the cluster size of the solves
    // (16, 8, 4 or 2 CTAs: fewer, faster clusters or more, smaller ones), timed over two steps,
    // then for that size the block (node and cell partition) of the drift-diffusion stages,
    // 256 or 128 threads, timed over the stages alone
    std::vector<void*> snap;
    cudaError_t e = batch_snapshot(b, snap, 0);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](auto&& body, float& ms) {
      e = cudaEventRecord(e0, b->stream);
      for (int s = 0; s < 2 && e == cudaSuccess; ++s) e = body();
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      ms = 0.f;
      if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess) e = batch_snapshot(b, snap, 1);
    };
    float best = 0.f;
    int bestC = 0;
    for (int C : {16, 8, 4, 2}) {
      if (e != cudaSuccess || !batch_configure(b, C)) continue;
      float ms = 0.f;
      timed([&] { return batch_enqueue_step(b); }, ms);
      if (e == cudaSuccess && (bestC == 0 || ms < best)) {
        best = ms;
        bestC = C;
      }
    }
    if (e == cudaSuccess && bestC != 0) ok = batch_configure(b, bestC);
    float bestT_ms = 0.f;
    int bestT = 0;
    for (int T : {256, 128}) {
      if (!ok || e != cudaSuccess || !batch_set_dd(b, T)) continue;
      float ms = 0.f;
      timed([&] { return launch_dd_batch(b->d_dargs, b->d_npref, b->d_cpref, (int)b->m.size(), b->node_blocks,
                                         b->cell_blocks, b->dd_threads, b->stream); }, ms);
      if (e == cudaSuccess && (bestT == 0 || ms < bestT_ms)) {
        bestT_ms = ms;
        bestT = T;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ok && e == cudaSuccess && bestT != 0) ok = batch_set_dd(b, bestT);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) ok = false;
  }
  if (!ok) {
    std::snprintf(g_err, sizeof(g_err), "batch: an instance does not fit the cluster shared memory");
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    cudaStreamDestroy(b->stream);
    delete b;
    return AVIP_EINVAL;
  }
  *out = b;
  return AVIP_OK;
}

int batch_destroy(avip_batch_t b) {
  if (!b) return AVIP_OK;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  cudaStreamDestroy(b->stream);
  delete b;
  return AVIP_OK;
}

// The states of every instance of a batch, concatenated in the order the handles were given
// (each instance's block as state_get lays it out): every instance's copy is queued on the
// batch's stream and the call waits once, instead of once per instance.
int batch_state_get(avip_batch_t b, double* out) {
  if (!b || !out) return AVIP_EINVAL;
  size_t off = 0;
  cudaError_t e = cudaSuccess;
  for (avip_mesh* h : b->m) {
    if (!state_buffers(h)) return AVIP_ENOMEM;
    int64_t n = 0;
    state_size(h, &n);
    if (e == cudaSuccess) e = launch_state_take(state_args(h), b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + off, h->d_stage, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    off += (size_t)n;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return cuda_status(e);
}

// Install the concatenated states of batch_state_get: AVIP_EINVAL (a history count outside
// 0..3) or AVIP_ENAN (a non-finite entry) install nothing.
int batch_state_set(avip_batch_t b, const double* in) {
  if (!b || !in) return AVIP_EINVAL;
  const size_t count = b->m.size();
  std::vector<size_t> off(count + 1, 0);
  for (size_t k = 0; k < count; ++k) {
    avip_mesh* h = b->m[k];
    int64_t n = 0;
    state_size(h, &n);
    off[k + 1] = off[k] + (size_t)n;
    const double hn = in[off[k + 1] - 1];
    if (!(hn >= 0.0 && hn <= (double)kPredictorHistory && hn == std::floor(hn))) return AVIP_EINVAL;
    if (!state_buffers(h)) return AVIP_ENOMEM;
  }
  std::vector<int32_t> flags(count, 0);
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < count && e == cudaSuccess; ++k) {
    avip_mesh* h = b->m[k];
    e = cudaMemcpyAsync(h->d_stage, in + off[k], (off[k + 1] - off[k]) * sizeof(double), cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_state_flag, 0, sizeof(int32_t), b->stream);
    if (e == cudaSuccess) e = launch_state_check(state_args(h), b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&flags[k], h->d_state_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  for (int32_t f : flags)
    if (f) return AVIP_ENAN;
  for (size_t k = 0; k < count && e == cudaSuccess; ++k) {
    avip_mesh* h = b->m[k];
    StateArgs sa = state_args(h);
    const size_t N = (size_t)h->hm.N;
    sa.t = in[off[k] + (size_t)(h->ph.ns + 1) * N];
    sa.hist = (int32_t)in[off[k + 1] - 1];
    e = launch_state_put(sa, b->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return cuda_status(e);
}

int batch_info(avip_batch_t b, int64_t* info) {
  if (!b || !info) return AVIP_EINVAL;
  info[0] = b->C;
  info[1] = b->nclusters;
  info[2] = (int64_t)b->smem;
  info[3] = (int64_t)b->m.size();
  info[4] = b->dd_threads;
  return AVIP_OK;
}

int batch_set_dd_threads(avip_batch_t b, int32_t threads) {
  if (!b || (threads != 128 && threads != 256)) return AVIP_EINVAL;
  return batch_set_dd(b, threads) ? AVIP_OK : AVIP_ECUDA;
}

int batch_run_steps(avip_batch_t b, int32_t nsteps, avip_stats* stats) {
  if (!b || nsteps < 0) return AVIP_EINVAL;
  const int n = (int)b->m.size();
  std::vector<DevScalars> s0(n);
  for (int k = 0; k < n; ++k) {
    cudaError_t e = cudaMemcpyAsync(&s0[k], b->m[k]->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  cudaError_t e = launch_run_reset_batch(b->d_dargs, n, b->stream);
  if (e == cudaSuccess && !b->graph && nsteps > 1) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = batch_enqueue_step(b);
      e = cudaStreamEndCapture(b->stream, &g);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->graph = nullptr;
      e = cudaSuccess;
    }
  }
  for (int32_t s = 0; s < nsteps && e == cudaSuccess; ++s)
    e = b->graph ? cudaGraphLaunch(b->graph, b->stream) : batch_enqueue_step(b);
  if (e != cudaSuccess) return cuda_status(e);
  std::vector<DevScalars> sc(n);
  for (int k = 0; k < n && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(&sc[k], b->m[k]->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int status = AVIP_OK;
  for (int k = 0; k < n; ++k) {
    if (stats) {
      stats[k].steps = sc[k].run_steps;
      stats[k].pcg_iters_total = sc[k].run_iters_total;
      stats[k].pcg_iters_max = sc[k].run_iters_max;
      stats[k].status = sc[k].status;
      stats[k].dt_min = sc[k].run_dt_min;
      stats[k].dt_max = sc[k].run_dt_max;
      stats[k].t = sc[k].t;
      stats[k].charge = sc[k].charge;
      stats[k].charge_start = s0[k].charge;
      stats[k].relres_max = sc[k].run_relres_max;
    }
    if (status == AVIP_OK && sc[k].status != AVIP_OK) status = sc[k].status;
  }
  return status;
}

}  // extern "C"
