/*
 * avip.h -- C ABI of the GB300 (sm_103a) library for the Poisson-coupled drift-diffusion
 * step of the AVIP low-temperature plasma method (arXiv 2201.01291).
 *
 * One explicit time step on an unstructured triangle, quadrangle or hybrid mesh:
 *   1. potential phi from  -lap(phi) = rho/eps0  with Dirichlet / zero-normal-field
 *      boundaries (section "Integrating the Poisson equation", Eq. poisson, Eq.
 *      poisson_discretization_cartesian, Eq. coeff_matriceA, "Boundary conditions"),
 *      solved on the device by conjugate gradients preconditioned by a smoothed-aggregation
 *      AMG V-cycle (planar meshes above 500 nodes; Jacobi-preconditioned CG below, and as an
 *      option), or by BiCGStab for the non-symmetric axisymmetric matrix (the paper names no
 *      linear solver);
 *   2. E = -grad(phi) with Green-Gauss cell gradients through nodal normals;
 *   3. edge-based limited Lax-Wendroff + central diffusion fluxes of every charged species
 *      (section "Development of TVD schemes", Eq. vertex_centered_flux) with the node-flux
 *      boundary closure (section "Boundary conditions in AVIP");
 *   4. field-dependent ionisation source (section "Bagheri benchmark");
 *   5. explicit update under the cell-based time step (section "Time step computation").
 *
 * Conventions for every entry point:
 *   - Return value: AVIP_OK (0) or a negative AVIP_E* status; nothing aborts, traps or exits.
 *   - Host arrays passed in are copied; the library never keeps a caller pointer.
 *   - Node arrays (in and out) use the caller's node numbering.  The library renumbers nodes
 *     internally (Morton order) and hides the permutation.
 *   - All device memory belongs to the handle.  It comes from opts->alloc/opts->free when
 *     given (e.g. a framework's caching allocator), else from cudaMalloc/cudaFree.
 *   - All work is queued on the handle's stream (opts->stream, or mesh_set_stream); calls
 *     that return host data synchronise that stream.  One handle per host thread.
 *   - SI units throughout (m, V, m^-3, m^2/(V s), m^2/s, s).
 */
#ifndef AVIP_H
#define AVIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define AVIP_OK        0
#define AVIP_EINVAL   -1  /* bad argument: index out of range, degenerate cell, unknown model */
#define AVIP_ENOMEM   -2  /* device allocation failed */
#define AVIP_ENOTCONV -3  /* PCG reached max_iter; phi is left at the last iterate           */
#define AVIP_ENAN     -4  /* a non-finite density, potential or time step was detected      */
#define AVIP_ECUDA    -5  /* a CUDA runtime call failed                                      */
#define AVIP_ETIMEOUT -6  /* a device-side wait gave up (bounded spin); the handle is reset  */
#define AVIP_ESTATE   -7  /* call out of order (e.g. stepping before every species is set)  */

/* ---- model identifiers ------------------------------------------------------------- */
#define AVIP_MOB_CONST 0   /* mu = p[0]                                                    */
#define AVIP_MOB_POWER 1   /* mu = p[0] * (max(|E|, p[3]) / p[1]) ^ p[2]                  */
#define AVIP_SRC_NONE 0
#define AVIP_SRC_TOWNSEND 1          /* alpha(|E|) = A exp(-B/|E|); S = alpha mu_e |E| n_e  */
#define AVIP_SRC_TOWNSEND_ATTACH 2   /* plus attachment nu_a n_e moved from e to the anion  */
#define AVIP_SRC_MORROW_LOWKE 3      /* three-species air chemistry of the section "Hyperbole
                                        electrodes": with w = mu_e |E|, alpha = A exp(-B/|E|),
                                        eta = A_eta exp(-B_eta/|E|) and recombination rate beta_r,
                                        S_e = (alpha - eta) w n_e - beta_r n_e n_p,
                                        S_p = alpha w n_e - beta_r n_e n_p - beta_r n_n n_p,
                                        S_n = eta w n_e - beta_r n_n n_p                        */
#define AVIP_BND_NEUMANN 0 /* boundary node flux F = F_C ("Neumann")                        */
#define AVIP_BND_OUTFLOW 1 /* boundary node flux F = F_C + F_D ("supersonic")              */
#define AVIP_LIM_SWEBY 0   /* Psi(r) = max(0, min(beta r, 1), min(r, beta))                 */
#define AVIP_LIM_VANLEER 1 /* Psi(r) = (r + |r|)/(1 + |r|)                                  */
#define AVIP_FLUX_LLW 0    /* limited Lax-Wendroff convection + central diffusion (default)   */
#define AVIP_FLUX_SG 1     /* Scharfetter-Gummel on the edge-tangential part of S_ij, centred
                              scheme on its normal part (section "Scharfetter Gummel scheme") */
#define AVIP_PREC_FP64 0   /* every stage in FP64                                           */
#define AVIP_PREC_MIXED 1  /* FP32 inner PCG + FP64 iterative refinement of the residual;
                              FP32 gradients, velocities, sources and edge fluxes; the state,
                              the update, the time-step reduction and the charge sum in FP64 */
#define AVIP_MAX_SPECIES 4
/* Geometry of the (x, y) plane.  AXISYMMETRIC: y is the radius r >= 0 about the x axis and
 * every volume and face integral carries the weight r (sections "Axisymmetric configuration"
 * of the Poisson chapter and the axisymmetric flux form of the transport chapter): r-weighted
 * Poisson rows, which make the matrix non-symmetric (solved by Jacobi-scaled BiCGStab),
 * r-weighted edge and boundary normals, dual volumes of revolution.  Volumes, charges and the
 * VOLUME field are then per radian (the common factor 2 pi is left out). */
#define AVIP_GEOM_PLANAR 0
#define AVIP_GEOM_AXISYMMETRIC 1

#define AVIP_FIELD_PHI 0
#define AVIP_FIELD_EX 1
#define AVIP_FIELD_EY 2
#define AVIP_FIELD_DENSITY 3  /* species index in `s`                                       */
#define AVIP_FIELD_VOLUME 4   /* median-dual nodal volume V_i (per radian if axisymmetric)  */
#define AVIP_FIELD_PHOTO 5    /* photoionisation source S_ph of the last step (photo_set)   */
#define AVIP_MAX_PHOTO_TERMS 3

typedef void* (*avip_alloc_fn)(size_t bytes, void* ctx);
typedef void (*avip_free_fn)(void* ptr, void* ctx);

/* Run-time choices.  The paper fixes no DD constants; these defaults are project choices:
 * CFL 0.4 (the stiff advection case), Fourier 0.25, A_D 0.5, A_tau 0.2, min-mod (beta 1). */
typedef struct avip_opts {
  double cfl, fourier, a_diel, a_chem; /* time-step constants (section "Time step computation") */
  double beta;                         /* Sweby limiter parameter, 1 <= beta <= 2             */
  int32_t limiter;                     /* AVIP_LIM_*                                          */
  int32_t precision;                   /* AVIP_PREC_*                                         */
  double rtol;                         /* stop when ||b - K phi||_2 <= rtol ||b||_2 over the
                                          free rows of the diagonally scaled system (Dirichlet
                                          rows hold their value exactly and are not counted) */
  int32_t max_iter;                    /* PCG iteration cap per solve                         */
  int32_t reorder;                     /* 1 = Morton renumbering (default), 0 = keep order    */
  double dt_fixed;                     /* > 0: use this time step instead of the automatic one */
  double inner_rtol;                   /* mixed precision: FP32 inner reduction per refinement */
  int32_t pcg_threads;                 /* solver block size (256/512/768/1024; 0 = the kind's default:
                                          768, 1024 for the AMG-preconditioned CG) */
  int32_t pcg_kind;                    /* solver kernel: 0 auto, 1 streaming, 2 register-resident,
                                          5 cluster, 7 BiCGStab (the only one for AXISYMMETRIC),
                                          8 CG preconditioned by an AMG V-cycle (auto for planar
                                          FP64 meshes above 20,000 nodes), 9 BiCGStab
                                          preconditioned by it (auto for AXISYMMETRIC meshes
                                          above 20,000 nodes), 10 the mixed-precision form of
                                          8, 11 the AMG solve on one thread-block cluster (auto
                                          for planar meshes of 501 to 20,000 nodes) */
  void* stream;                        /* cudaStream_t for all work; NULL = default stream    */
  avip_alloc_fn alloc;                 /* optional device allocator (both or neither)         */
  avip_free_fn free;
  void* alloc_ctx;
  int32_t geometry;                    /* AVIP_GEOM_* (default PLANAR)                          */
  int32_t scheme;                      /* AVIP_FLUX_* edge flux (default LLW)                   */
  double v_rise;                       /* > 0: every Dirichlet value rises linearly from 0 at
                                          t = 0 to its phi_D at t = v_rise and stays there (the
                                          anode ramp of the section "Hyperbole electrodes"; a
                                          grounded electrode, phi_D = 0, stays at 0); 0 = constant */
  double wait_timeout;                 /* seconds a device-side wait of a cooperative solver
                                          (a grid-wide barrier) may last before the kernel gives
                                          up: its blocks leave, the call returns AVIP_ETIMEOUT and
                                          the handle stays usable.  Default 2; 0 gives up at the
                                          first wait that is not already satisfied (a test of the
                                          failure path); at most 60 */
  int32_t precond_fp64;                /* AMG solvers of the FP64 path: 0 (default) applies the
                                          V-cycle preconditioner with FP32 values and vectors
                                          (the Krylov iterate, the products with the Poisson
                                          matrix, the residuals and the stopping test stay
                                          FP64, so the solution meets rtol all the same); 1
                                          applies it in FP64 */
  int32_t cluster_size;                /* solver kind 11 (the AMG solve on one thread-block
                                          cluster): CTAs of its cluster, 2, 4, 8 or 16; 0 = 16
                                          when schedulable, else 8.  Smaller clusters leave room
                                          for more handles solving at the same time */
} avip_opts;

/* Per-run statistics filled by run_steps / dd_step. */
typedef struct avip_stats {
  int32_t steps;             /* steps completed in this call                                */
  int32_t pcg_iters_total;   /* PCG iterations summed over the call                         */
  int32_t pcg_iters_max;     /* largest per-step PCG iteration count                        */
  int32_t status;            /* AVIP_OK or the first error seen                             */
  double dt_min, dt_max;     /* time steps taken                                            */
  double t;                  /* simulated time after the call                               */
  double charge;             /* Q = e sum_s q_s sum_i V_i n_s,i after the call (C/m)        */
  double charge_start;       /* Q before the call                                           */
  double relres_max;         /* largest final PCG relative residual                         */
} avip_stats;

typedef struct avip_mesh* avip_mesh_t;

/* Fill `o` with the defaults above. */
int avip_opts_default(avip_opts* o);

/* Build a mesh handle.
 *   xy[2*n_nodes]   node coordinates, interleaved (x0,y0,x1,y1,...);
 *   tris[3*n_tris]  0-based node indices, either orientation (made counter-clockwise);
 *   node_bc[n_nodes] 0 = free node (interior or zero-normal-field side), 1 = Dirichlet,
 *                    2 = node of a Neumann (zero normal field) side: the natural condition,
 *                    treated as 0;
 *   phi_D[n_nodes]  Dirichlet potential (read where node_bc == 1).
 * Computes the metrics of the section "Nomenclature and notations" (cell volumes, nodal
 * normals, median-dual volumes, edge normals, boundary nodal normals) and the Poisson matrix
 * of Eq. coeff_matriceA (with opts->geometry AXISYMMETRIC: their r-weighted forms of the
 * axisymmetric sections), renumbers, and uploads everything.  Errors: AVIP_EINVAL for
 * out-of-range indices, zero-area cells, a mesh with no Dirichlet node, a negative radius or
 * a non-positive Poisson diagonal (AXISYMMETRIC), AXISYMMETRIC with AVIP_PREC_MIXED or with
 * a pcg_kind other than 0, 7 or 9; AVIP_ENOMEM. */
int mesh_create(const double* xy, int32_t n_nodes, const int32_t* tris, int32_t n_tris,
                const int32_t* node_bc, const double* phi_D, const avip_opts* opts,
                avip_mesh_t* out);

/* Build a mesh handle on a hybrid mesh of triangles and quadrangles (planar geometry only).
 *   tris[3*n_tris]   triangles as for mesh_create (n_tris may be 0, tris then may be NULL);
 *   quads[4*n_quads] quadrangles, 4 node indices in boundary order, either orientation (made
 *                    counter-clockwise), non-self-intersecting (n_quads may be 0).
 * The other arguments are those of mesh_create.  The metrics are the n_v-vertex forms of the
 * section "Nomenclature and notations": cell volume by the shoelace formula, nodal normal
 * S_k = -(n_d/n_v^f) times the sum of the two faces adjacent to k (Eq. node_normal), dual volume
 * V_tau/n_v, dual faces from the side midpoints to the cell centre (vertex mean), boundary
 * normals from the sides that belong to one cell; Poisson matrix of Eq. coeff_matriceA over all
 * n_v^2 vertex pairs.  The time-step limits of the section "Time step computation" take the
 * cell average of n_v vertices and the shortest side.  Errors: those of mesh_create, plus
 * AVIP_EINVAL for a quadrangle index out of range, a zero-area quadrangle, n_tris + n_quads < 1,
 * or quadrangles with opts->geometry AXISYMMETRIC.  info[1] of mesh_info counts all cells. */
int mesh_create_hybrid(const double* xy, int32_t n_nodes, const int32_t* tris, int32_t n_tris,
                       const int32_t* quads, int32_t n_quads, const int32_t* node_bc, const double* phi_D,
                       const avip_opts* opts, avip_mesh_t* out);

/* Host-only inspection of the preparation mesh_create / mesh_create_hybrid performs (no device
 * is touched): the metrics of the section "Nomenclature and notations" in the caller's
 * numbering.  Arguments as for mesh_create_hybrid, plus geometry (AVIP_GEOM_*).
 *   counts[3]  out: number of edges E, stored entries of the Poisson matrix, cells;
 *   vol        out (may be NULL): [n_nodes] dual volumes (per radian if axisymmetric);
 *   edges      out (may be NULL): [2 E] node pairs (i, j), i < j, sorted by (i, j);
 *   S_edge     out (may be NULL): [2 E] edge normal S_ij (x, y), oriented i -> j;
 *   S_b        out (may be NULL): [2 n_nodes] boundary nodal normals S_i^b (0 inside).
 * Call once with NULL outputs to learn E.  Errors: those of mesh_create_hybrid's host
 * validation (AVIP_EINVAL; avip_inspect_error() gives the reason). */
int mesh_inspect(const double* xy, int32_t n_nodes, const int32_t* tris, int32_t n_tris, const int32_t* quads,
                 int32_t n_quads, const int32_t* node_bc, const double* phi_D, int32_t geometry, int64_t* counts,
                 double* vol, int32_t* edges, double* S_edge, double* S_b);
const char* avip_inspect_error(void);

/* Release every device and host resource of the handle.  NULL is accepted. */
int mesh_destroy(avip_mesh_t h);

/* Queue subsequent work of the handle on `stream` (a cudaStream_t). */
int mesh_set_stream(avip_mesh_t h, void* stream);

/* Change the handle's wait_timeout (see avip_opts; 0 <= seconds <= 60, else AVIP_EINVAL).
 * Takes effect from the next call that steps or solves. */
int mesh_set_wait_timeout(avip_mesh_t h, double seconds);

/* Declare species s (0 <= s < AVIP_MAX_SPECIES; species must be declared 0,1,2,... in order)
 * of the drift-diffusion system (section "Drift-diffusion equations"): charge in units of e
 * (-1 or +1), mobility model AVIP_MOB_* with 4 parameters, diffusion coefficient D,
 * boundary closure AVIP_BND_*, and the initial density n0[n_nodes] (host, caller order). */
int species_set(avip_mesh_t h, int32_t s, int32_t charge, int32_t mob_model,
                const double* mob_params, double D, int32_t bnd_mode, const double* n0);

/* Source model (section "Bagheri benchmark"): params = {A, B, nu_att} for TOWNSEND and
 * TOWNSEND_ATTACH; {A, B, A_eta, B_eta, beta_r} for MORROW_LOWKE (section "Hyperbole
 * electrodes"; all >= 0, SI units: 1/m, V/m, 1/m, V/m, m^3/s).  idx = {electron, positive ion,
 * negative ion (-1 if none; required, and the three distinct, for TOWNSEND_ATTACH and
 * MORROW_LOWKE)} species indices.  AVIP_EINVAL for an unknown model, a negative or non-finite
 * parameter or an index out of range. */
int source_set(avip_mesh_t h, int32_t model, const double* params, const int32_t* idx);

/* Photoionisation source (section "Case 3" of the streamer benchmark: the three-term
 * exponential fit of the radiative transfer by Helmholtz equations).  Each step, after the
 * ionisation rate I_ion = alpha |W_e| n_e is known, n_terms equations
 *     -lap S_j + kappa_j^2 S_j = a_j c I_ion,   S_j = 0 on the Dirichlet nodes,
 *     zero normal derivative on the other boundaries,
 * are solved (vertex-centred: (K + kappa_j^2 V) S_j = a_j c V I_ion with the Poisson matrix K and
 * the dual volumes V) by the handle's own solver kind with the term's own diagonal scaling and,
 * for the AMG kinds, its own hierarchy (built here, once; with the whole-GPU AMG kinds the
 * terms are solved side by side in one launch, see photo_stats), started from the cubic
 * extrapolation of its last four solutions; S_ph = sum_j S_j is added to the electron and positive-ion sources (idx[0], idx[1] of
 * source_set) before the time step and the update, and enters the chemical time-step limit.
 *   a[n_terms]     A_j p_O2^2 (1/m^2)  — with A_j, lambda_j the coefficients of the fit;
 *   kappa[n_terms] lambda_j p_O2 (1/m), > 0;
 *   c              I = c I_ion: quenching and photo-efficiency factor
 *                  (p_q/(p + p_q)) xi nu_u/nu_i (dimensionless), >= 0.
 * Requires the FP64 solvers (AVIP_EINVAL with AVIP_PREC_MIXED); may be called once per handle
 * (AVIP_ESTATE after that); n_terms = 0 is a no-op; at most AVIP_MAX_PHOTO_TERMS terms.  A
 * handle with photoionisation cannot join a batch.  The solves' iteration counts are not part
 * of avip_stats (those count the Poisson solves); a solve that fails sets the run status. */
int photo_set(avip_mesh_t h, int32_t n_terms, const double* a, const double* kappa, double c);

/* The photoionisation solves of the last step (waits for the handle's stream): *n_terms the
 * number of terms (0 without photo_set); per term j, iters[j] its iterations and relres[j] its
 * final true relative residual (arrays of AVIP_MAX_PHOTO_TERMS entries, either may be NULL);
 * *side_by_side 1 when the terms are solved at the same time in one launch, each on its own
 * share of the grid (the whole-GPU AMG solver kinds 8 and 9), 0 when one after another.
 * AVIP_EINVAL for a NULL handle, n_terms or side_by_side. */
int photo_stats(avip_mesh_t h, int32_t* n_terms, int32_t* iters, double* relres, int32_t* side_by_side);

/* Solve the Poisson problem for the current densities, starting from the cubic
 * extrapolation of the last potentials (the last one alone after mesh_create or a state with
 * no history).  Every call advances that history.
 * iters_out / relres_out (may be NULL) receive the PCG iteration count and the final true
 * relative residual.  AVIP_ENOTCONV if max_iter was reached. */
int poisson_solve(avip_mesh_t h, int32_t* iters_out, double* relres_out);

/* One explicit step: Poisson, E, gradients, time step (dt <= 0: automatic, else dt), fluxes,
 * source, update.  dt_used may be NULL. */
int dd_step(avip_mesh_t h, double dt, double* dt_used);

/* nsteps explicit steps queued without host synchronisation (replayed as a CUDA graph);
 * synchronises once at the end and fills `stats` (may be NULL). */
int run_steps(avip_mesh_t h, int32_t nsteps, avip_stats* stats);

/* Measurement variant of run_steps: the same kernels launched one by one (no graph) with CUDA
 * events recorded on the handle's stream around each of them; every step is queued before the
 * call waits (once, for the last event).  kernel_ms[AVIP_TIMED_KERNELS]
 * receives the summed device time of {Poisson solve, nodal fields, cell time step, fluxes +
 * update, finalize, photoionisation solves + source update} over the call; `stats` (may be
 * NULL) as for run_steps. */
#define AVIP_TIMED_KERNELS 6
int run_steps_timed(avip_mesh_t h, int32_t nsteps, double* kernel_ms, avip_stats* stats);

/* Copy a nodal field to host memory, caller numbering: AVIP_FIELD_* (s = species index for
 * densities).  out[n_nodes] doubles. */
int field_get(avip_mesh_t h, int32_t which, int32_t s, double* host_out);

/* Checkpoint / resume.  state layout, caller numbering: [n_species * n_nodes densities]
 * [n_nodes phi][t][n_nodes phi_{n-1}][n_nodes phi_{n-2}][n_nodes phi_{n-3}][h], where
 * phi_{n-1}, phi_{n-2}, phi_{n-3} and h (0 .. 3 of them valid) are the history of the Poisson
 * solver's initial-guess predictor (cubic extrapolation of the last potentials), so that a
 * resumed run repeats the uninterrupted one bit for bit (with photoionisation the Helmholtz
 * solutions and their histories are not part of the state: a resumed run then agrees within
 * the solve tolerance); size = (n_species + 4) * n_nodes + 2 doubles.  state_set
 * returns AVIP_EINVAL for h outside {0, 1, 2, 3}, AVIP_ENAN for a non-finite entry. */
int state_size(avip_mesh_t h, int64_t* n_doubles);
int state_get(avip_mesh_t h, double* host_state);
int state_set(avip_mesh_t h, const double* host_state);

/* info[8] = {n_nodes, n_cells (triangles + quadrangles), n_edges, nnz of the Poisson matrix, PCG kernel kind
 * (1 streaming, 2 register-resident, 4 mixed precision, 5 cluster-resident, 6 cluster mixed,
 * 7 BiCGStab, 8 AMG-preconditioned CG, 9 AMG-preconditioned BiCGStab, 10 mixed AMG, 11 AMG on one
 * cluster), solver blocks,
 * PCG threads per block, device bytes held by the handle}. */
int mesh_info(avip_mesh_t h, int64_t* info8);

/* Multigrid hierarchy of the AMG-preconditioned solvers (kinds 8-11; the paper names no solver, this
 * reports the set-up built for this project's preconditioner).  Returns the number of levels
 * (finest first, the last one inverted densely), or 0 when the handle uses another solver; for
 * the first min(levels, max_levels) levels writes AVIP_LEVEL_STATS values per level at
 * out[AVIP_LEVEL_STATS * l]: rows, stored entries of the level matrix A, of the prolongator P
 * from the next level, and of the composite operators the V-cycle applies, Rf = R (I - A Q),
 * U = 2 I - Q A and Pf = (I - Q A) P (Q: the smoother, with A's sparsity); the last four are 0
 * on the coarsest level.  AVIP_EINVAL for a NULL handle or a NULL `out` with max_levels > 0. */
#define AVIP_LEVEL_STATS 6
int solver_levels(avip_mesh_t h, int64_t* out, int32_t max_levels);

/* ---- batches (many independent instances per step) -------------------------------------
 * A batch advances several mesh handles together: per step, one persistent launch solves the
 * Poisson system of every instance (one thread-block cluster per instance at a time, largest
 * instances first), then one launch per drift-diffusion stage covers every instance; the step
 * is captured as a CUDA graph and replayed.  Each instance keeps its own state, time step and
 * statistics, and gives the same result alone and in the batch (tests check it).
 *   meshes[count]: FP64 handles with every species set; they must outlive the batch and must
 *                  not be stepped on their own while the batch runs;
 *   cluster_size:  2, 4, 8 or 16 CTAs per cluster, or 0 to pick by timing each on the batch
 *                  (the instances' state is saved and restored around the trial): fewer, larger
 *                  clusters solve each instance faster, more, smaller ones run more at once; with
 *                  0 the block of the drift-diffusion stages (256 or 128 threads, i.e. the rows
 *                  and edges each block takes) is then timed the same way (256 otherwise).
 * AVIP_EINVAL if an instance solved by the shared-memory Jacobi-PCG does not fit one cluster's
 * shared memory (it holds every vector of its instance there; about 100k nodes at most with 16
 * CTAs); instances with an AMG hierarchy keep their vectors in global memory. */
typedef struct avip_batch* avip_batch_t;
int batch_create(const avip_mesh_t* meshes, int32_t count, int32_t cluster_size, avip_batch_t* out);
/* nsteps steps of every instance; stats[count] (may be NULL) receives per-instance statistics. */
int batch_run_steps(avip_batch_t b, int32_t nsteps, avip_stats* stats);
/* info[5] = {cluster size, resident clusters, dynamic shared memory bytes per CTA, count,
 * threads per block of the drift-diffusion stages}. */
int batch_info(avip_batch_t b, int64_t* info);
/* Set the block of the batch's drift-diffusion stages (128 or 256 threads; AVIP_EINVAL
 * otherwise), overriding the autotuner's choice; results do not depend on it. */
int batch_set_dd_threads(avip_batch_t b, int32_t threads);
/* Checkpoint of a whole batch: the states of its instances concatenated in the order the
 * handles were given to batch_create, each laid out as state_get lays it out (the sum of their
 * state_size entries).  One wait per call whatever the number of instances.  batch_state_set
 * installs nothing when an entry is not finite (AVIP_ENAN) or a history count is outside 0..3
 * (AVIP_EINVAL). */
int batch_state_get(avip_batch_t b, double* host_state);
int batch_state_set(avip_batch_t b, const double* host_state);
int batch_destroy(avip_batch_t b);

/* No-allocation Jacobi-preconditioned CG for callers that cannot allocate device memory.
 * The paper has no counterpart: it exists for code that must not call cudaMalloc or any
 * allocating routine, for example a real-time loop with a fixed memory budget that forbids
 * allocation after start-up (an allocation may block or fail under fragmentation), or a
 * framework that owns all device memory through its own pool; mesh_create allocates, so such
 * code cannot use a handle.  It places the Dirichlet-eliminated Poisson matrix (or any
 * symmetric positive definite matrix) in device memory as CSR and solves A x = b:
 *   row_ptr[n+1], col[nnz], val[nnz], b[n]  device pointers, read only;
 *   x[n]  device pointer: initial guess in, solution out (b = 0 gives x = 0);
 *   stop when ||b - A x||_2 <= rtol ||b||_2 (true residual), at most max_iter iterations;
 *   stream: cudaStream_t the solve is queued on (NULL = default).
 * The call is synchronous: it copies the status back and waits for `stream`, so it blocks the
 * host thread until the solve ends.  iters_out / relres_out (may be NULL) receive the
 * iteration count and ||b - A x|| / ||b|| of the returned x.
 * Work vectors live in one fixed array compiled into the library (AVIP_STATIC_PCG_MAX_ROWS
 * rows, about 10.5 MB, present on every GPU that loads the library until exit).  The first
 * call made on a device looks up that array's device address (no allocation); after
 * cudaDeviceReset of that device the entry point must not be called on it again.  Calls that
 * overlap on the GPU share the array and race: order them on one stream.
 * Returns AVIP_EINVAL for n > AVIP_STATIC_PCG_MAX_ROWS or bad arguments, AVIP_ENOTCONV when
 * max_iter was reached (x holds the last iterate).  Allocates nothing. */
#define AVIP_STATIC_PCG_MAX_ROWS 262144
int pcg_csr_static(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* val, const double* b,
                   double* x, double rtol, int32_t max_iter, void* stream, int32_t* iters_out, double* relres_out);

/* Roofline denominators measured on the current device (the paper has no counterpart: a
 * measurement aid).  which = AVIP_PROBE_FP64_FMA: FP64 fused multiply-add rate in TFLOP/s (8
 * independent FMA chains per thread, every SM full, 2 flops per FMA); AVIP_PROBE_HBM_COPY:
 * device-memory copy bandwidth in GB/s (1 GiB copied between two buffers larger than L2, read
 * plus write bytes).  Best of 5 launches timed with CUDA events on `stream` (NULL = default)
 * after one untimed launch; the call waits for them and writes the figure to *value_out.  It
 * allocates and frees its own device buffers (2 GiB for the copy).  AVIP_EINVAL for an unknown
 * `which` or a NULL value_out, AVIP_ENOMEM, AVIP_ECUDA. */
#define AVIP_PROBE_FP64_FMA 0
#define AVIP_PROBE_HBM_COPY 1
int peak_probe(int32_t which, void* stream, double* value_out);

/* Accuracy check of the library's own FP64 exponential, logarithm, power and reciprocal (used by
 * the local-field mobility and Townsend closures and by the limiter ratio of the FP64 path; the
 * paper has no counterpart): max_rel_err[4] receives the largest relative difference from the
 * CUDA math library's exp, log, pow and from the IEEE quotient 1/x over 65,536 log-spaced
 * arguments (exp on [-700, 700], log on positive arguments from 1e-300 to 1e300, pow on bases
 * from 1e-6 to 1e6 with exponents -0.2, 0.5, -1.7, 2.3, the reciprocal on +-1e-300 to +-1e300).
 * Runs one kernel on the current device and waits for it.  AVIP_EINVAL, AVIP_ENOMEM, AVIP_ECUDA. */
int fp64_math_check(double* max_rel_err);

/* Human-readable text of a status code (static storage). */
const char* avip_status_str(int status);

/* Detail of the last AVIP_EINVAL / AVIP_ECUDA raised on this host thread (static storage). */
const char* avip_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AVIP_H */
