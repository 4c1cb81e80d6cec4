// Internal layout shared by the host mesh preparation, the kernels and the C ABI.
//
// Device data layout (nodes renumbered in Morton order, SELL-32 sparse storage):
//   * rows are grouped in slices of 32 consecutive nodes; slice s owns the element range
//     [sl_ptr[s], sl_ptr[s] + 32 * sl_w[s]) with element (lane, k) at sl_ptr[s] + 32 k + lane,
//     so a warp reading slot k of its 32 rows issues one fully coalesced load;
//   * slot 0 of every row is the diagonal (column = row); slots 1..flen-1 are the neighbours
//     across a mesh edge (a cell side), ascending; slots flen..rlen-1 the other vertices of the
//     row's quadrangles (coupled by the Poisson matrix and the gradient, no flux), ascending;
//     slots >= rlen are padding and never read (flen == rlen on triangle meshes);
//   * per element: col (int32), aval (Poisson matrix after Dirichlet elimination), gx/gy
//     (nodal-gradient weights G_ik), sx/sy (edge normal S_ij oriented row -> col; in slot 0
//     the boundary nodal normal S_i^b).
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/avip.h"

namespace avip {

constexpr double kECharge = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr int kSlice = 32;

struct HostMesh {
  int32_t N = 0, T = 0, E = 0;        // nodes, cells (triangles + quadrangles), undirected edges
  int32_t Q = 0;                      // quadrangles among the T cells
  int32_t nvmax = 3;                  // 3 (triangles only) or 4
  int32_t nslices = 0;
  int64_t nnz = 0;                    // structural nonzeros (diag + 2 E)
  int64_t nelem = 0;                  // SELL elements incl. padding
  std::vector<int32_t> perm;          // new -> caller index
  std::vector<int32_t> iperm;         // caller -> new index
  int32_t geometry = 0;               // AVIP_GEOM_*
  std::vector<double> x, y, vol;      // new order; vol = dual volume (per radian when axisymmetric)
  std::vector<int32_t> bc;            // new order
  std::vector<int32_t> cell;          // nvmax*T, new indices, counter-clockwise (SoA: v0[T], v1[T], ...;
                                      // v3 = -1 for the triangles of a hybrid mesh)
  std::vector<double> dxmin;          // T, shortest side
  std::vector<double> cw;             // T, 1 / (n_v dxmin): |sum of the n_v nodal V| * cw = |V_cell| / dx
  double dxmin_all = 0.0;             // shortest side of the mesh
  std::vector<int32_t> rlen;          // N (padded to nslices*32 with 0)
  std::vector<int32_t> flen;          // N (padded likewise): 1 + number of edge neighbours
  std::vector<int32_t> sl_ptr, sl_w;  // nslices
  std::vector<int32_t> col;           // nelem
  std::vector<double> aval, gx, gy, sx, sy;  // nelem (aval: D^-1/2 K D^-1/2)
  std::vector<double> dsq, dsqinv;    // N: sqrt(K_ii) and its inverse (symmetric Jacobi scaling)
  // edges (lo < hi, ordered by lo then hi) with the normal S oriented lo -> hi, and per SELL
  // element of an edge slot the edge id, bit 31 set when the row is the edge's hi end
  std::vector<int32_t> e_lo, e_hi, slot_eid;
  std::vector<double> e_sx, e_sy;
  std::vector<double> lift;           // N: free rows -sum_{k in D} K_ik phi_D,k ; Dirichlet rows phi_D (scaled by 1/sqrt(K_ii))
  std::vector<double> rhs_scale;      // N: free rows e V_i / eps0 ; Dirichlet rows 0 (scaled by 1/sqrt(K_ii))
};

// Builds every metric and sparse structure; returns AVIP_OK or AVIP_EINVAL.
// geometry: AVIP_GEOM_PLANAR or AVIP_GEOM_AXISYMMETRIC (second coordinate = radius >= 0).
// quads (4 node indices per cell, may be NULL with n_quads = 0): planar geometry only.
int prepare_mesh(const double* xy, int32_t n_nodes, const int32_t* tris, int32_t n_tris, const int32_t* quads,
                 int32_t n_quads, const int32_t* node_bc, const double* phi_D, int reorder, int geometry,
                 HostMesh& out, char* err, size_t errlen);

// ----------------------------------------------------------------- AMG hierarchy (host)
constexpr int kAmgMaxLevels = 12;
struct Csr {  // compressed sparse rows, n x m
  int32_t n = 0, m = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> v;
};
struct AmgHostLevel {
  Csr A, P, R;                 // level matrix; prolongator from the next level; R = P^T
  std::vector<double> dinv;    // 1 / diag(A)
  double lmax = 1.0;           // estimate of the largest eigenvalue of D^-1 A
  // smoother: x = Q b from x = 0 and x <- x + Q (b - A x) from a given x, Q = omega D^-1
  double omega = 0.0;
  // composite operators of the two-phase V-cycle (non-coarsest levels only):
  //   Q  (n x n)      pre-smoothing from zero (diagonal)
  //   Rf (n' x n)     = R (I - A Q): restriction of the pre-smoothed residual
  //   U  (n x n)      = 2 I - Q A:  the pre-smoothed iterate through the post-smoother
  //   Pf (n x n')     = (I - Q A) P: the coarse correction through the post-smoother
  Csr Q, Rf, U, Pf;
};
struct AmgHost {
  std::vector<AmgHostLevel> lv;  // lv.back() is the coarsest level
  int32_t nc = 0;                // coarsest size
  std::vector<double> cinv;      // dense inverse of the coarsest matrix (row-major)
};
// Builds the smoothed-aggregation hierarchy of the scaled Poisson matrix of `m`, with the
// composite operators of every non-coarsest level.
int amg_setup(const HostMesh& m, AmgHost& out, char* err, size_t errlen);

// SELL-32 form of a CSR matrix with `lpr` lanes per row (1, 2, 4, 8, 16 or 32): a slice holds
// 32 / lpr consecutive rows; step k of a slice is 32 contiguous elements, entries k*lpr ..
// k*lpr + lpr - 1 of each of its rows (row r of the slice at r*lpr + e % lpr); a slice has as
// many steps as its longest row needs; padding holds column 0 and value 0.  With lpr = 1 this is
// the layout of the mesh matrix.
struct SellHost {
  int32_t n = 0, nslices = 0, lpr = 1;
  std::vector<int32_t> sl_ptr, sl_w, rlen, col;
  std::vector<double> val;
};
void sell_from_csr(const Csr& A, SellHost& out, int lpr = 1);
// Lanes per row for a streamed operator: the smallest power of two (at most 32) that leaves
// at most 8 stored entries per lane on an average row.
int lanes_per_row(const Csr& A);

// ----------------------------------------------------------------- kernel argument blocks
struct SellView {  // device pointers of the SELL-32 structure
  const int32_t* sl_ptr;
  const int32_t* sl_w;
  const int32_t* rlen;
  const int32_t* col;
  const double* aval;
  const double* gx;
  const double* gy;
  const double* sx;
  const double* sy;
  int32_t N;
  int32_t nslices;
};

template <typename T>
struct SellMatT {  // device pointers of a SELL-32 matrix with values of type T
  const int32_t* sl_ptr;  // nslices + 1 element offsets
  const int32_t* sl_w;    // steps per slice
  const int32_t* rlen;
  const int32_t* col;
  const T* val;
  int32_t n;
  int32_t nslices;
  int32_t lpr;            // lanes per row (SellHost)
};
using SellMat = SellMatT<double>;

// One level of the two-phase V-cycle on the device (values of type T: float by default, double
// on request).  Down phase: xp = Q b (n rows; Q diagonal) and b' = Rf b (n' rows of the next level); up
// phase: x = [U | Pf] [xp; x'] (n rows; UP holds U's columns as they are and Pf's shifted by n).
// Level 0 takes its right-hand side and writes its solution through the solver's own vectors;
// x and b are used from level 1 on.
template <typename T>
struct AmgLevelT {
  SellMatT<T> Rf, UP;   // empty on the coarsest level
  const T* qd;          // the smoother Q = omega D^-1 (its diagonal, n entries)
  T* xp;                // pre-smoothed iterate Q b
  T* x;                 // level solution
  T* b;                 // level right-hand side
  int32_t n;
};
template <typename T>
struct AmgDevT {
  int32_t nlev;         // levels including the coarsest
  int32_t nc;           // coarsest size
  const T* cinv;        // coarsest dense inverse, nc x nc row-major
  AmgLevelT<T> L[kAmgMaxLevels];
};
using AmgLevelDev = AmgLevelT<double>;
using AmgDev = AmgDevT<double>;

struct SpeciesParams {
  double q;           // charge number (-1, +1)
  double mob[4];
  double D;
  double mob_log_ref;  // log(mob[1]) for AVIP_MOB_POWER (set on the host)
  int32_t mob_model;
  int32_t bnd_mode;
};

struct Physics {
  int32_t ns;
  int32_t src_model;
  int32_t src_idx[3];
  int32_t limiter;
  int32_t scheme;     // AVIP_FLUX_*
  int32_t dd_fp32;    // 1: gradients, velocities, sources and fluxes in FP32 (mixed precision)
  int32_t photo_terms;  // > 0: photoionisation source from that many Helmholtz solves
  double src_params[5];   // {A, B, nu_att} or {A, B, A_eta, B_eta, beta_r} (AVIP_SRC_MORROW_LOWKE)
  double beta, cfl, fourier, a_diel, a_chem;
  double dt_fixed;
  double dt_fourier;  // min over cells and species of fourier dx^2 / D (constant per mesh)
  SpeciesParams sp[AVIP_MAX_SPECIES];
};

// Grid-wide barrier / reduction state (device memory, zeroed before each cooperative launch).
struct GridSync {
  unsigned int count;
  unsigned int gen;
  int abort;
  int pad;
  double red[8];
};

// Device scalars of a handle (one block of device memory).
struct DevScalars {
  unsigned long long dt_bits;   // running min of candidate time steps (bit pattern of a
                                // positive double orders like the integer)
  double dt;                    // time step used by the current step
  double t;                     // simulated time
  double charge;                // Q after the last step
  int32_t parity;               // which density buffer is current
  int32_t status;               // first error of the current run (AVIP_*)
  int32_t pcg_iters;            // iterations of the last solve
  int32_t pcg_status;
  double pcg_relres;            // final true relative residual of the last solve
  double pcg_bnorm;
  // run statistics (accumulated by the finalize kernel)
  int32_t run_steps;
  int32_t run_iters_total;
  int32_t run_iters_max;
  int32_t pcg_outer;            // refinement steps of the last mixed-precision solve
  int32_t phi_hist;             // earlier potentials kept for the predictor (0 .. 3)
  double run_dt_min, run_dt_max, run_relres_max;
};

// Jacobi-PCG is run on the symmetrically scaled system
//   (D^-1/2 K D^-1/2) x = D^-1/2 b,   phi = D^-1/2 x,
// whose CG iterates are those of Jacobi-preconditioned CG on K phi = b; the preconditioned
// residual z = D^-1 r becomes the plain residual of the scaled system.
struct PcgArgs {
  SellView A;             // A.aval holds the scaled matrix D^-1/2 K D^-1/2
  const double* dsq;      // sqrt(K_ii)
  const double* dsqinv;   // 1 / sqrt(K_ii)
  const double* rhs_scale;  // scaled: e V_i / (eps0 sqrt(K_ii)) on free rows, 0 on Dirichlet rows
  const double* lift;       // scaled Dirichlet lift
  const double* nbuf;     // density buffers: nbuf[(parity * AVIP_MAX_SPECIES + s) * Npad + i]
  int32_t Npad;
  int32_t ns;
  double q[AVIP_MAX_SPECIES];
  double* phi;            // potential (warm start in, solution out)
  double* x;              // scaled iterate
  double* b;              // scaled right-hand side
  double* r;
  double* p;
  double* q_ap;           // scaled A p
  unsigned* flags;        // [0] grid-reduction arrival counter (zeroed before each launch)
  double* parts;          // grid barrier partials, 2 * gridDim.x * 4
  GridSync* sync;
  DevScalars* sc;          // status, time and density parity of the handle
  DevScalars* res;         // where the solve reports iterations / residual (sc, or the
                           // auxiliary block of the photoionisation solves)
  const double* rhs_src;   // non-null: b = rhs_scale * rhs_src + lift instead of the charge density
  double* phi1;            // non-null: the three previous solutions phi_{n-1}, phi_{n-2},
  double* phi2;            // phi_{n-3} (predictor)
  double* phi3;
  int32_t* hist;           // how many of them are valid (0, 1, 2); advanced by the solve
  double rtol;
  double v_rise;          // > 0: the Dirichlet lift is scaled by min(t / v_rise, 1) (voltage ramp)
  unsigned long long spin_ns;  // bound of every grid-barrier wait (the handle's wait_timeout)
  int32_t max_iter;
  int32_t use_density_rhs;  // 1: b from densities; 0: b already in `b`
  // mixed precision: FP32 copy of the scaled matrix and FP32 inner-CG vectors
  const float* aval32;
  float* e32;
  float* r32;
  float* p32;
  float* q32;
  double inner_rtol;
  // BiCGStab (non-symmetric systems): three more vectors s, t and the shadow residual, each
  // Npad long, at bcg + k * Npad (v = A p lives in q_ap)
  double* bcg;
  // AMG-preconditioned solvers (kinds 8-11): the hierarchy in device memory, FP32 (amg32,
  // default) or FP64 (amg); the preconditioned residual z (of the hierarchy's type: z32 or z);
  // r2: the second buffer of the CG residual (the update r - alpha q is written to the other
  // buffer while neighbours still gather the old one)
  const AmgDev* amg;
  double* z;
  const AmgDevT<float>* amg32;
  float* z32;
  double* r2;
  float* rq32;            // FP32 hierarchy: FP32 copies of the two residual buffers and of q
                          // (3 x Npad), the vectors the finest down phase gathers
  int32_t amg_mixed;      // 1: FP32 inner CG + FP64 refinement (kind 10); 0: FP64 CG
};

// Systems solved side by side in one cooperative launch (the photoionisation terms): system j
// by the blocks start[j] .. start[j+1] - 1, with its own arguments (vectors, hierarchy, barrier
// state flags / parts / sync, statistics block res).
struct AmgGroupArgs {
  PcgArgs a[AVIP_MAX_PHOTO_TERMS];
  int32_t n;
  int32_t start[AVIP_MAX_PHOTO_TERMS + 1];
};

// Kernel and grid of a PCG launch.
struct PcgPlan {
  int kind = 1;    // 1 streaming, 2 register-resident, 4 mixed precision, 5 cluster-resident,
                   // 6 cluster-resident mixed precision, 7 BiCGStab (non-symmetric matrix),
                   // 8 AMG-preconditioned CG, 9 AMG-preconditioned BiCGStab, 10 mixed precision
                   // with the AMG preconditioner (FP32 inner CG + V-cycle, FP64 refinement),
                   // 11 AMG-preconditioned CG (FP64 or mixed) on one thread-block cluster
  int tpb = 768;
  int maxs = 0;    // slices per warp (register-resident); dynamic shared memory bytes (cluster);
                   // 1 for an FP64 AMG hierarchy (kinds 8, 9, 11), 0 for the FP32 one
  int blocks = 1;
};
PcgPlan pcg_plan(int nslices, int kind, int requested_tpb);
PcgPlan pcg_mixed_plan(int nslices, int requested_tpb);
PcgPlan bicgstab_plan(int nslices, int requested_tpb);
PcgPlan amg_plan(int nslices, int requested_tpb, int kind, int fp64);  // kind 8 (CG), 9 (BiCGStab), 10 (mixed)
PcgPlan amg_cluster_plan(int want, int n);  // kind 11 for n rows (one cluster of `want` CTAs or 16 / 8; kind 0 if none fits)

// Cluster-resident solve (kind 5): rows, halo and matrix slices per CTA of the cluster.
struct ClusterLayout {
  int32_t spc;        // slices per CTA
  int32_t rows;       // spc * 32
  int32_t hmax;       // largest halo (rows of other CTAs read by one CTA)
  int32_t max_elems;  // largest SELL element count of one CTA's slices
  int32_t mat_smem;   // 1: the CTA copies its matrix slices into shared memory
  int32_t mixed;      // 1: FP32 inner CG + FP64 refinement (matrix slices kept in FP32)
  const int32_t* colL;      // per SELL element: local index (own row, or rows + halo slot)
  const int32_t* push_ptr;  // per row: range of push_dst
  const int32_t* push_dst;  // (reader rank << 24) | halo slot
};
struct ClusterHost {
  std::vector<int32_t> colL, push_ptr, push_dst;
};
PcgPlan pcg_cluster_plan(const HostMesh& m, int max_rows, ClusterLayout* out, ClusterHost* hd, int mixed = 0);

#ifdef __CUDACC__
// Factor of the Dirichlet values at the simulated time of the solve: min(t / v_rise, 1) during
// a voltage ramp, exactly 1 otherwise (so the lift is used unchanged).
__device__ __forceinline__ double dirichlet_gain(const PcgArgs& a) {
  if (!(a.v_rise > 0.0)) return 1.0;
  const double t = *((volatile const double*)&a.sc->t);
  return t >= a.v_rise ? 1.0 : t / a.v_rise;
}

// Number of earlier solutions available to the predictor (read by every block at entry, before
// the solve's first barrier; the solve's leader advances it at the end).
__device__ __forceinline__ int history_length(const PcgArgs& a) {
  return a.phi1 ? *((volatile const int*)a.hist) : 0;
}

// Initial guess of row i from the last solutions: the polynomial through the last hist + 1
// potentials at equal steps, evaluated one step ahead: cubic 4 phi_n - 6 phi_{n-1} +
// 4 phi_{n-2} - phi_{n-3} once three earlier solutions exist (on the streamer workloads about
// one CG iteration in ten fewer than the quadratic one), quadratic 3 phi_n - 3 phi_{n-1} +
// phi_{n-2} with two, linear with one, phi_n otherwise; the row's history is shifted at the
// same time (each row is owned by one thread of the solve).
constexpr int kPredictorHistory = 3;
__device__ __forceinline__ double predict_phi(const PcgArgs& a, int i, int hist) {
  const double p0 = a.phi[i];
  if (!a.phi1) return p0;
  const double p1 = a.phi1[i], p2 = a.phi2[i], p3 = a.phi3[i];
  a.phi3[i] = p2;
  a.phi2[i] = p1;
  a.phi1[i] = p0;
  if (hist >= 3) return fma(4.0, p0 + p2, fma(-6.0, p1, -p3));
  if (hist == 2) return fma(3.0, p0 - p1, p2);
  if (hist == 1) return fma(2.0, p0, -p1);
  return p0;
}

// One more earlier solution available to the next solve (called by the solve's leader).
__device__ __forceinline__ void advance_history(const PcgArgs& a) {
  if (a.phi1) *a.hist = *a.hist < kPredictorHistory ? *a.hist + 1 : kPredictorHistory;
}

// A solve is skipped when an earlier stage of the run left non-finite data (AVIP_ENAN) or a
// device wait gave up (AVIP_ETIMEOUT): every block (or CTA of a cluster) reads the same value
// at entry, so all leave together.
__device__ __forceinline__ bool solve_skipped(const DevScalars* sc) {
  const int st = *((volatile const int*)&sc->status);
  return st == AVIP_ENAN || st == AVIP_ETIMEOUT;
}
#endif

// Checkpoint copies between the caller's layout (caller numbering: densities, phi, t, the
// predictor history, its count) and the device state: perm[i] is the caller index of internal
// node i, stage the state in the caller's layout (device memory).
struct StateArgs {
  int32_t N, ns, Npad;
  const int32_t* perm;
  double* stage;
  double *nbuf, *phi, *phi1, *phi2, *phi3;
  DevScalars* sc;
  int32_t* flag;  // state_check: set to 1 when an entry is not finite
  double t;       // state_put: simulated time and predictor history count to install
  int32_t hist;
};

struct DDArgs {
  SellView A;
  Physics ph;
  const double* x;        // node coordinates
  const double* y;
  const double* vol;
  const double* ivol;     // 1 / V_i
  const double* phi;
  double* nbuf;           // density ping-pong buffers
  double* ndat;           // per species per node: gx, gy, vx, vy (4 doubles)
  double* nm;             // per species per node: n * mu
  double* src;            // per species per node: source rate
  double* Ex;
  double* Ey;
  double* photo_I;        // per node: ionisation rate alpha |W_e| n_e (written when ph.photo_terms > 0)
  const double* photo_psi;  // ph.photo_terms solutions S_ph,j, each Npad long
  double* photo_S;        // per node: S_ph = sum_j S_ph,j
  const int32_t* cell;    // SoA v0[T], v1[T], v2[T] (, v3[T] when nvmax == 4; -1 for triangles)
  const double* cw;       // per cell 1 / (n_v dx_min)
  // edge fluxes computed once per edge (FP64 single-instance path; eflux == nullptr: each
  // row evaluates the fluxes of its edges itself)
  const int32_t* e_lo;
  const int32_t* e_hi;
  const double* e_sx;
  const double* e_sy;
  const int32_t* slot_eid;
  double* eflux;          // [species][E]: flux from lo to hi
  int32_t E;
  const int32_t* flen;    // per row: slots 1..flen-1 carry the mesh edges
  int32_t T;
  int32_t nvmax;
  int32_t Npad;
  double* partials;       // per-block charge partials
  DevScalars* sc;
  // mixed precision (ph.dd_fp32): FP32 copies of the gradient weights and edge normals, and
  // the FP32 per-species node records gx, gy, vx, vy (float4)
  const float* gx32;
  const float* gy32;
  const float* sx32;
  const float* sy32;
  float* ndat32;
};

}  // namespace avip
