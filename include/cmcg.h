/*
 * cmcg.h -- C ABI of the controllability method (CMCG) for time-harmonic
 * Maxwell's equations on tetrahedral meshes, GB300 (sm_103a) implementation.
 *
 * Paper: T. Chaumont-Frelet, M. J. Grote, S. Lanteri, J. H. Tang, "A
 * controllability method for Maxwell's equations", arXiv:2106.02858.
 *
 * Problem (Eq. maxwell_freq_strong / maxwell_time_strong): find complex (e, h)
 * with  i w eps e + curl h = j,  i w mu h - curl e = 0  in Omega,
 * e x n = 0 on the PEC part of the boundary and the first-order impedance
 * (Silver-Mueller) condition on the rest.  CMCG (Section 2.2, Algorithms
 * init / grad / cmcg) minimises J(U0) = 1/2 ||(I - P_w) U0 - G||^2 by
 * conjugate gradients, where P_w advances the discontinuous-Galerkin
 * time-domain scheme (Section 5.2.2, Eq. DG_semidiscrete / ode_system; RK2 or
 * RK4, Algorithms rk2 / rk4) over one period T = 2 pi / w, P*_w is its
 * discrete adjoint (Section 4.1.2) and the answer is the filtered field
 * F_{psi,w} U0 = (2/T) int_0^T U(t) e^{-i w t} dt (Eq. filter_rhs, Section 5.4).
 *
 * ---------------------------------------------------------------------------
 * Data layout at this boundary (all fields are double precision, row-major):
 *
 *   nodal field of one tetrahedron:   [component][node]
 *   full field:                       [tet][component][node]
 *     6 components for (E, H) = (Ex, Ey, Ez, Hx, Hy, Hz); 3 for e, h or j.
 *   nodes of order q (Np = (q+1)(q+2)(q+3)/6): the equispaced lattice points
 *     (i, j, k)/q, i, j, k >= 0, i + j + k <= q, of the unit tetrahedron
 *     (0,0,0), (1,0,0), (0,1,0), (0,0,1), enumerated with k outermost, then j,
 *     then i fastest; the physical node of tet (v0, v1, v2, v3) is
 *     v0 + r (v1 - v0) + s (v2 - v0) + t (v3 - v0).
 *   face f of a tetrahedron is the face opposite its vertex f.
 *   face tags: 0 interior (must be shared by exactly two tetrahedra),
 *              1 perfectly conducting, 2 impedance (Silver-Mueller, Z = sqrt(mu/eps)).
 *
 * Ownership: the caller owns every pointer it passes.  Inputs are copied (to
 * the device) during the call; outputs are written before the call returns.
 * The library owns the device state of a handle from cmcg_create to
 * cmcg_destroy.  "_device" entry points take device pointers (same layout,
 * double precision) and run on the handle's stream; they return once the
 * work is complete (they synchronise the stream).
 *
 * Errors: every int-returning call returns CMCG_OK (0) on success, a
 * negative CMCG_ERR_* code on failure (output buffers are then unspecified
 * for device entry points and untouched for host entry points), or
 * CMCG_NOT_CONVERGED (> 0) when cmcg_solve reached max_iter; its outputs are
 * then valid (Algorithm cmcg returns the last iterate).  The solves stop a
 * problem with CMCG_ERR_UNSTABLE when a CG direction D has
 * |(I - P) D| > 100 |D| in the (eps, mu) norm (the period map grows the
 * energy by orders of magnitude: a step beyond the stability limit, e.g. a
 * forced steps_per_period), CMCG_ERR_CG_BREAKDOWN when (D, A) <= 0 and
 * CMCG_ERR_NONFINITE when a reduction is not finite.  A stage kernel that
 * waits on the tensor cores gives up after about one second and the call
 * then returns CMCG_ERR_DEVICE_TIMEOUT (its outputs are not valid).
 *
 * Threading: one handle per host thread at a time.
 *
 * Typical use (error checks omitted):
 *
 *   cmcg_options o;  cmcg_default_options(&o);
 *   o.order = 2;  o.precision = CMCG_FP32;            // FP32 sweeps, FP64 CG scalars
 *   cmcg_mesh m = {nv, verts, nt, tets, face_tags};
 *   cmcg_handle* h;  cmcg_create(&m, eps, mu, omega, &o, &h);   // validates, lays out, tunes
 *   cmcg_info info;
 *   cmcg_solve(h, j_re, j_im, 1e-6, 1000, e_re, e_im, h_re, h_im, &info);
 *   cmcg_destroy(h);
 *
 * Many sources or meshes of one order: cmcg_create_batch + cmcg_solve_batch.
 * Incident fields on impedance faces: cmcg_set_boundary_data before the solve.
 * The limiting-amplitude baseline: cmcg_fw_solve.  A request server with
 * continuous batching: cmcg_server_create / add_model / submit / poll.
 */
#ifndef CMCG_H
#define CMCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum cmcg_status {
  CMCG_OK = 0,
  CMCG_NOT_CONVERGED = 1,
  CMCG_PENDING = 2,
  CMCG_ERR_INVALID_ARG = -1,
  CMCG_ERR_NONCONFORMING_MESH = -2,
  CMCG_ERR_OUT_OF_MEMORY = -3,
  CMCG_ERR_UNSTABLE = -4,
  CMCG_ERR_CG_BREAKDOWN = -5,
  CMCG_ERR_NONFINITE = -6,
  CMCG_ERR_DEVICE_TIMEOUT = -7,
  CMCG_ERR_CUDA = -8,
  CMCG_ERR_NO_DEVICE = -9
};

enum cmcg_precision { CMCG_FP64 = 0, CMCG_FP32 = 1 };
enum cmcg_flux { CMCG_FLUX_UPWIND = 0, CMCG_FLUX_CENTRED = 1 };
enum cmcg_tag { CMCG_TAG_INTERIOR = 0, CMCG_TAG_PEC = 1, CMCG_TAG_IMPEDANCE = 2 };

/* A conforming tetrahedral mesh (Section 5.2.2).  verts: double[nv][3];
 * tets: int32[nt][4] vertex indices; face_tags: uint8[nt][4]. */
typedef struct cmcg_mesh {
  int64_t nv;
  const double* verts;
  int64_t nt;
  const int32_t* tets;
  const uint8_t* face_tags;
} cmcg_mesh;

/* Options.  Fill with cmcg_default_options() first.
 *   order:            polynomial degree q in {1, 2, 3}; q = 1 uses RK2 +
 *                     trapezoid filter, q = 2, 3 use RK4 + Hermite filter
 *                     (Section 5.3 / 5.4; q = 2 is not in the paper and is
 *                     read as RK4 with c_2 = 0.12).
 *   precision:        CMCG_FP64 or CMCG_FP32 for the time sweeps; CG
 *                     scalars, dot products and the cost functional are FP64
 *                     in both.
 *   flux:             CMCG_FLUX_UPWIND (the paper's scheme) or
 *                     CMCG_FLUX_CENTRED (energy-conserving, for tests).
 *   c_q:              CFL constant of Eq. cfl; <= 0 selects 0.12 for every
 *                     order.  Section 5.3 prints 0.24 for P1 / RK2 (a 2D
 *                     constant); on 3D meshes of 8^3 cubes and more with
 *                     permittivity jumps it makes one RK2 period grow a mode
 *                     tenfold and more, so P1 uses half of it by default (pass
 *                     0.24 to get the printed value).
 *   steps_per_period: > 0 forces M (dt = T / M) instead of the CFL choice.
 *   hbm_budget_bytes: > 0 makes cmcg_create fail with
 *                     CMCG_ERR_OUT_OF_MEMORY if the handle would need more
 *                     device memory than this.
 *   device:           CUDA device ordinal.
 *   stage_variant:    0 = time the stage-kernel forms on this mesh at
 *                     creation and keep the fastest; k > 0 forces form k - 1.
 *                     FP32: 0, 1, 2 = two threads per tetrahedron (E / H)
 *                     with at least 1, 3, 4 resident 128-thread blocks per
 *                     SM; 3, 4, 5 = four threads per tetrahedron (E / H x
 *                     node half) with at least 4, 5, 6; 6 = the volume and
 *                     lift contractions on the tensor cores (tcgen05, three
 *                     TF32 products per FP32 product, FP32 accumulation),
 *                     two threads per tetrahedron.  FP64: 0 = two threads
 *                     per tetrahedron; 1, 2 = four threads with at least
 *                     2, 3.  Other k: CMCG_ERR_INVALID_ARG.  Results do not
 *                     depend on it beyond rounding.
 *   stage_overlap:    0 = decide by timing when the form is timed (on when
 *                     the form is forced); 1 = on; 2 = off.  On: each stage
 *                     is launched with programmatic stream serialisation, so
 *                     its blocks start and load the mesh data while the
 *                     previous stage finishes.  Results are identical.
 *   launch_graphs:    0 or 1 = each period sweep (its stage launches) is
 *                     captured once as a CUDA graph on a private stream and
 *                     replayed on the handle's stream; 2 = direct launches.
 *                     If the driver refuses the capture, the handle falls
 *                     back to direct launches.  Results are identical. */
typedef struct cmcg_options {
  int order;
  int precision;
  int flux;
  int steps_per_period;
  double c_q;
  int64_t hbm_budget_bytes;
  int device;
  int stage_variant;
  int stage_overlap;
  int launch_graphs;
  int reserved[4];
} cmcg_options;

/* Per-solve report. */
typedef struct cmcg_info {
  int iters;            /* CG iterations taken */
  int periods;          /* periods simulated: 3 + 2 iters (Algorithms init, grad, final filter) */
  int steps_per_period; /* M */
  int status;           /* same as the return value */
  double rel_residual;  /* ||R|| / ||R0|| in the (eps, mu) norm at exit */
  double dt;            /* T / M */
  double solve_ms;      /* wall time of the solve on the device */
  double reserved[5];
} cmcg_info;

typedef struct cmcg_handle cmcg_handle;

/* Fills *opt with: order 1, FP64, upwind, CFL choice, no budget, device 0. */
void cmcg_default_options(cmcg_options* opt);

/* Human-readable text for a status code (static storage). */
const char* cmcg_status_string(int status);

/* Host-only checks of a mesh and its data (no CUDA call): index ranges,
 * non-degenerate tetrahedra, eps, mu > 0, omega > 0, order, tags, and
 * conformity (every face shared by at most two tetrahedra, interior faces
 * untagged, every unshared face tagged PEC or impedance, face nodes
 * coincide).  Writes M (steps per period of Eq. cfl) to *steps if non-NULL. */
int cmcg_validate(const cmcg_mesh* mesh, const double* eps, const double* mu, double omega,
                  const cmcg_options* opt, int* steps);

/* Host-only: the reference matrices the library builds for order q (unit
 * reference tetrahedron, boundary node order): mass[Np*Np], dr/ds/dt[Np*Np]
 * (d phi_j / d r at node i, row i), lift[Np*4*Nfp] = M^{-1} times the face mass
 * of each face (face f, face-node order = increasing volume node).  Any
 * pointer may be NULL.  Returns CMCG_ERR_INVALID_ARG for q outside 1..3. */
int cmcg_reference_matrices(int order, double* mass, double* dr, double* ds, double* dt, double* lift);

/* Builds a handle: validates (as cmcg_validate), computes connectivity and
 * geometry, chooses M (Eq. cfl), uploads the mesh in the device layout and
 * allocates the CG state.  eps, mu: double[nt], element-constant, > 0. */
int cmcg_create(const cmcg_mesh* mesh, const double* eps, const double* mu, double omega,
                const cmcg_options* opt, cmcg_handle** out);

/* One problem of a batch: a mesh, its element permittivity / permeability and
 * its angular frequency. */
typedef struct cmcg_problem {
  const cmcg_mesh* mesh;
  const double* eps;
  const double* mu;
  double omega;
} cmcg_problem;

/* Builds a handle over a batch of nprob independent problems sharing the
 * options (order, precision, flux, device ...); meshes, materials, frequencies
 * and steps per period may differ (many sources on one mesh: pass the same
 * mesh nprob times).  Every stage launch covers all problems; each problem
 * keeps its own CG state and stops when it converges.  The single-problem
 * entry points (dgtd_*, cmcg_inner, cmcg_solve[_device]) need nprob == 1. */
int cmcg_create_batch(int nprob, const cmcg_problem* probs, const cmcg_options* opt, cmcg_handle** out);

/* ---------------------------------------------------------------------------
 * Element partition (sharding).  The DG operator couples tetrahedra only through
 * face fluxes (Section 5.2.2), so a part of an element partition needs, per RK
 * stage, the stage values of the tetrahedra across its cut faces (its ghosts),
 * and CMCG needs, per CG iteration, its FP64 inner products summed over the
 * parts (Section 2.2, Algorithm cmcg).  The paper has no partitioned solver.
 *
 * cmcg_partition_slabs (host only): part[k] in [0, nparts) for every
 * tetrahedron: tetrahedra sorted by the centroid coordinate `axis` (0, 1, 2)
 * and cut into nparts slabs of (nearly) equal count.
 *
 * cmcg_shard_plan (host only): the local mesh of part p: its owned tetrahedra
 * in increasing global order, then its ghosts (the other parts' tetrahedra that
 * share a face with an owned one) in increasing global order.
 * global_of_local[n_owned + n_ghost]; per ghost g: ghost_owner_part[g] and
 * ghost_owner_local[g] (its index in the owner's local numbering);
 * local_tags[(n_owned + n_ghost) * 4]: the mesh's face tags, a ghost's face
 * whose neighbour is not in the local mesh tagged PEC.  Output arrays may be
 * NULL (call once with NULLs to get the counts).
 *
 * cmcg_create_sharded: one handle over the parts of `part` (nparts >= 1, every
 * part owning a tetrahedron), all on opt->device.  Every part steps with the M
 * of the whole mesh; after every stage each ghost receives its owner's values
 * (a halo-exchange kernel between the parts' device buffers); ghosts carry no
 * weight in the inner products, whose per-part sums are added before every CG
 * scalar.  The single-problem entry points (cmcg_solve[_device],
 * dgtd_period_forward / adjoint [_device], dgtd_apply, cmcg_inner,
 * cmcg_get_sizes) take it with arrays of the whole mesh; the batch, FW,
 * boundary-data and conductivity entry points return CMCG_ERR_INVALID_ARG.
 * Results equal those of cmcg_create on the whole mesh up to rounding. */
int cmcg_partition_slabs(const cmcg_mesh* mesh, int nparts, int axis, int32_t* part);
int cmcg_shard_plan(const cmcg_mesh* mesh, const int32_t* part, int nparts, int p, int64_t* n_owned, int64_t* n_ghost,
                    int32_t* global_of_local, int32_t* ghost_owner_part, int32_t* ghost_owner_local,
                    uint8_t* local_tags);
int cmcg_create_sharded(const cmcg_mesh* mesh, const double* eps, const double* mu, double omega,
                        const cmcg_options* opt, int nparts, const int32_t* part, cmcg_handle** out);

/* Number of problems of a handle (0 for NULL). */
int cmcg_batch_size(const cmcg_handle* h);

/* nt, steps per period and dt of problem p.  Any output pointer may be NULL. */
int cmcg_get_problem(const cmcg_handle* h, int p, int64_t* nt, int* steps, double* dt);

/* Releases the device state.  NULL is ignored. */
void cmcg_destroy(cmcg_handle* h);

/* Uses the given cudaStream_t (as void*) for all later work of the handle;
 * NULL selects the legacy default stream. */
int cmcg_set_stream(cmcg_handle* h, void* stream);

/* Stage-kernel form in use (0-based, as stage_variant - 1) and, when it was
 * chosen by timing at creation, the measured microseconds per stage of each
 * form (10 entries: [0..6] indexed by form, see stage_variant; [7] the chosen
 * form with stage_overlap on; [8], [9] unused; -1 where not timed or rejected by
 * the device).  Any pointer may be NULL. */
int cmcg_get_tuning(const cmcg_handle* h, int* variant, double* us_per_stage);

/* Sizes of the handle: nt, Np, M (steps per period), dt, number of doubles of
 * one full field (6 Np nt).  Any pointer may be NULL. */
int cmcg_get_sizes(const cmcg_handle* h, int64_t* nt, int* np, int* steps, double* dt, int64_t* field_len);

/* Phi(t, U) = Re(J e^{i w t}) + B U (Eq. ode_system), or Sigma B Sigma U when
 * adjoint != 0 (no source then).  u, out: double[nt][6][Np]; j_re, j_im:
 * double[nt][3][Np] current density (NULL = no source; j_im may be NULL). */
int dgtd_apply(cmcg_handle* h, double t, const double* u, const double* j_re, const double* j_im, int adjoint,
               double* out);

/* One period forward (Section 4.1.2): uT = P_{psi,w} u0 with the source j
 * (P_w if j_re is NULL).  If filt_re and filt_im are non-NULL they receive
 * the filtered field F_{psi,w} u0 (Section 5.4), double[nt][6][Np] each.
 * Every sweep runs the RK polynomial of Algorithms rk2 / rk4 in nested form,
 * v <- U + (dt / k) (B v + g_k) for k = s, ..., 1; with a source, g_k is the
 * combination of Re(J e^{i w t}) at t_m, t_m + dt/2, t_m + dt for which the
 * nested form equals Algorithm rk4 exactly (g_4 = f(t_m), g_3 = (f(t_m) +
 * f(t_m + dt/2)) / 2, g_2 = (f(t_m) + 2 f(t_m + dt/2)) / 3, g_1 = (f(t_m) +
 * 4 f(t_m + dt/2) + f(t_m + dt)) / 6; for RK2 g_2 = f(t_m), g_1 = f(t_m + dt/2)),
 * so the results differ from the printed form by rounding only. */
int dgtd_period_forward(cmcg_handle* h, const double* u0, const double* j_re, const double* j_im, double* uT,
                        double* filt_re, double* filt_im);

/* One period of the discrete adjoint: w0 = P*_w wT = Sigma P_w Sigma wT
 * (Lemma dual_propagators; the magnetic sign is flipped inside the kernels). */
int dgtd_period_adjoint(cmcg_handle* h, const double* wT, double* w0);

/* Device-pointer forms of the two sweeps (same layout, double). */
int dgtd_period_forward_device(cmcg_handle* h, const double* u0, const double* j_re, const double* j_im, double* uT,
                               double* filt_re, double* filt_im);
int dgtd_period_adjoint_device(cmcg_handle* h, const double* wT, double* w0);

/* The CMCG solve (Algorithm cmcg with Algorithms init and grad, initial
 * guess 0, residual form) followed by the filter: (e, h) = F_{psi,w} U0.
 * j_re, j_im: double[nt][3][Np] (j_im may be NULL); tol: stop when
 * ||R|| <= tol ||R0|| in the (eps, mu) norm; max_iter >= 0.  e_re, e_im, h_re,
 * h_im: double[nt][3][Np] each, caller-allocated.  info may be NULL. */
int cmcg_solve(cmcg_handle* h, const double* j_re, const double* j_im, double tol, int max_iter, double* e_re,
               double* e_im, double* h_re, double* h_im, cmcg_info* info);

/* Several frequencies in one solve (the Conclusion, Section 7: CMCG can compute the
 * solutions of several frequencies "in one shot").  The handle's omega is the base
 * frequency w0 (its period T0 = 2 pi / w0 and M as for a single solve); harmonic h
 * has the frequency harmonics[h] w0 (an integer >= 1) and the current density
 * j_re[h] + i j_im[h].  CMCG runs once on the period T0 with the summed source
 * Re(sum_h J_h e^{i harmonics[h] w0 t}); then one filtered sweep from its U0 per
 * harmonic, with the filter of Eq. filter at that harmonic's frequency over T0,
 * writes e_re[h], e_im[h], h_re[h], h_im[h]: the time-harmonic field of frequency
 * harmonics[h] w0.  Cost: one CMCG solve plus nharm - 1 sweeps.  nharm in 1..64;
 * arrays of nharm host pointers to double[nt][3][Np] (j_im may be NULL, or any
 * j_im[h]); single-problem handles only (not batch or sharded).  info: the one
 * CG's report (periods include the extra sweeps). */
int cmcg_solve_multifreq(cmcg_handle* h, int nharm, const int* harmonics, const double* const* j_re,
                         const double* const* j_im, double tol, int max_iter, double* const* e_re,
                         double* const* e_im, double* const* h_re, double* const* h_im, cmcg_info* info);

/* (u, v)_{eps,mu} = sum_K int_K eps E_u . E_v + mu H_u . H_v (Eq. innerproduct),
 * i.e. V^T M U with the block-diagonal DG mass matrix, evaluated on the device
 * in FP64 (the fields are first rounded to the handle's precision).  u, v:
 * double[nt][6][Np] host arrays. */
int cmcg_inner(cmcg_handle* h, const double* u, const double* v, double* out);

/* Largest nt accepted by cmcg_inner_noalloc (128 tetrahedra per block x 8192 blocks). */
#define CMCG_NOALLOC_MAX_TETS 1048576

/* The paper has no counterpart: this is cmcg_inner without a handle and
 * without any device allocation, for callers that cannot call cudaMalloc where
 * they need the inner product (code whose device memory all belongs to its own
 * pool allocator, stream-ordered pipelines that cudaMalloc / cudaFree would
 * synchronise, callers that hold no handle because cmcg_create allocates).
 * Computes (u, v)_{eps,mu} = sum_K w_K0 E_u.Mref E_v + w_K1 H_u.Mref H_v with the
 * unit-tetrahedron mass matrix Mref of order q, accumulated in FP64.
 *   order: q in 1..3;  nt: 1..CMCG_NOALLOC_MAX_TETS (larger: CMCG_ERR_INVALID_ARG,
 *   nothing launched);  u, v: device double[nt][6][Np] in the boundary layout;
 *   w: device double[nt][2] = (eps_K, mu_K) times |det(v1-v0, v2-v0, v3-v0)|
 *   (six times the volume of K);  out: device double[1].
 * Runs on `stream` (a cudaStream_t, NULL = legacy default stream) of the
 * current device and returns once its two kernels are launched; *out is valid
 * when the stream reaches that point.  It reduces through a 64 KiB static
 * device array that every GPU loading the library holds until the process
 * exits.  The first call on a device does a one-time set-up (uploads the mass
 * matrices, looks up the array's device address); make that first call before
 * any stream capture.  All calls share the array: calls that overlap on the
 * GPU race. */
int cmcg_inner_noalloc(int order, int64_t nt, const double* u, const double* v, const double* w, double* out,
                       void* stream);

/* CMCG for every problem of a batch handle (Algorithm cmcg per problem; all
 * problems sweep together, converged ones stop updating).  Arrays of nprob
 * host pointers: j_re[p], j_im[p] (j_im or any j_im[p] may be NULL) are
 * double[nt_p][3][Np]; e_re[p], e_im[p], h_re[p], h_im[p] likewise.  info (may
 * be NULL) receives nprob reports.  Returns the most severe status over the
 * problems (an error, else CMCG_NOT_CONVERGED if any problem reached max_iter). */
int cmcg_solve_batch(cmcg_handle* h, const double* const* j_re, const double* const* j_im, double tol, int max_iter,
                     double* const* e_re, double* const* e_im, double* const* h_re, double* const* h_im,
                     cmcg_info* info);

/* cmcg_solve_batch restricted to problems [0, n) of the handle (1 <= n <= nprob):
 * the other problems are skipped by every kernel, so one handle built for a
 * capacity of n_max requests can serve any smaller group.  Arrays hold n host
 * pointers. */
int cmcg_solve_batch_n(cmcg_handle* h, int n, const double* const* j_re, const double* const* j_im, double tol,
                       int max_iter, double* const* e_re, double* const* e_im, double* const* h_re,
                       double* const* h_im, cmcg_info* info);

/* Continuous batching on a batch handle (the serving runtime's engine; the paper
 * has no counterpart).  Problem p of the handle is slot p.
 *   cmcg_slot_admit: starts a request in an empty slot: host j_re, j_im
 *     (double[nt_p][3][Np]; j_im may be NULL) are copied before it returns.
 *   cmcg_slot_round: advances every busy slot by one step of its solve in the
 *     same sweeps: Algorithm init for admitted slots, one CG iteration
 *     (Algorithm grad and the update of Algorithm cmcg) for iterating slots, the
 *     final filter for slots whose CG stopped (converged, broke down, or reached
 *     max_iter); done (NULL or int[nprob]) receives 1 for the slots whose result
 *     became ready in this round.  Requests admitted between rounds join the
 *     next round while the others continue.
 *   cmcg_slot_take: copies a ready result (e, h as in cmcg_solve; any pointer
 *     may be NULL) and its report, empties the slot and returns its status.
 *   cmcg_slot_state: 0 empty, 1 admitted, 2 iterating, 3 filter pending,
 *     4 result ready (CMCG_ERR_INVALID_ARG for a bad slot).
 * A slot's arithmetic is that of cmcg_solve of the same problem alone with
 * the same kernel form (stage_variant): results do not depend on the other
 * slots.  Not for sharded handles.  tol and max_iter apply to every slot. */
int cmcg_slot_admit(cmcg_handle* h, int slot, const double* j_re, const double* j_im);
int cmcg_slot_round(cmcg_handle* h, double tol, int max_iter, int* done);
int cmcg_slot_take(cmcg_handle* h, int slot, double* e_re, double* e_im, double* h_re, double* h_im, cmcg_info* info);
int cmcg_slot_state(const cmcg_handle* h, int slot);

/* Checkpoint / resume of a slot between rounds (the paper has no counterpart).
 * cmcg_slot_save writes the state of an admitted, iterating or filter-pending
 * slot -- its CG state U0, R, D, the FP64 CG scalars, and its source -- into
 * buf (at least cmcg_slot_state_bytes(h, slot) bytes, host memory) and empties
 * the slot.  cmcg_slot_restore puts such a state into an empty slot of any
 * handle whose problem in that slot has the same mesh size, order, precision,
 * M, dt and omega (else CMCG_ERR_INVALID_ARG); the request then continues as
 * if it had never stopped (the same bits).  The state is in the handle's
 * internal layout and precision, for the same library build. */
int64_t cmcg_slot_state_bytes(const cmcg_handle* h, int slot);
int cmcg_slot_save(cmcg_handle* h, int slot, void* buf, int64_t len);
int cmcg_slot_restore(cmcg_handle* h, int slot, const void* buf, int64_t len);

/* Device memory held by a handle, in bytes (the figure cmcg_create checks
 * against hbm_budget_bytes). */
int64_t cmcg_device_bytes(const cmcg_handle* h);

/* Device-pointer form of cmcg_solve_batch (the pointer arrays live on the host). */
int cmcg_solve_batch_device(cmcg_handle* h, const double* const* j_re, const double* const* j_im, double tol,
                            int max_iter, double* const* e_re, double* const* e_im, double* const* h_re,
                            double* const* h_im, cmcg_info* info);

/* Device-pointer form of cmcg_solve (same layout, double). */
int cmcg_solve_device(cmcg_handle* h, const double* j_re, const double* j_im, double tol, int max_iter,
                      double* e_re, double* e_im, double* h_re, double* h_im, cmcg_info* info);

/* Number of kernels the library launched on this handle since creation (a
 * counter kept on the host at every launch). */
int64_t cmcg_kernel_launches(const cmcg_handle* h);

/* Impedance-face data g (the incident-field datum of the impedance traces,
 * Section 5.2.2) for problem `problem` of the handle: on every impedance face
 * the upwind flux sees the exterior state (E+, H+) = (Re(g e^{i w t}), 0) with
 * the boundary tetrahedron's own Z.  An incident field (E_i, H_i) of that
 * medium is passed exactly by g = E_i - Z n x H_i (n the outward normal).
 * g_re, g_im: host double[nt][4][3][Nfp] (tetrahedron, face opposite vertex f,
 * component x y z, face node in increasing volume-node order); read on
 * impedance faces only; g_im may be NULL (= 0); g_re NULL clears the data.
 * The data enter every sweep that carries the source j (cmcg_solve,
 * cmcg_fw_solve, dgtd_period_forward and dgtd_apply with j given; pass j = 0
 * for a problem driven by g alone) and stay until cleared or replaced.  The
 * first call allocates two field vectors on the device. */
int cmcg_set_boundary_data(cmcg_handle* h, int problem, const double* g_re, const double* g_im);

/* Conductivity sigma_K >= 0 of every tetrahedron of problem `problem`
 * (Eq. maxwell_time_strong, Section 1: eps dE/dt + sigma E + curl H = J; the
 * coefficients of Section 3.1; the term (sigma E_h, v_h) of the DG scheme,
 * Section 5.2.2): the E rows of the operator gain -(sigma_K / eps_K) E.  The
 * adjoint stays Sigma P Sigma (the term is symmetric and acts on E only).
 * sigma: host double[nt] in the mesh's order, or NULL to remove it (sigma = 0,
 * the paper's experiments).  The time step is the one of Eq. cfl; a sigma with
 * dt sigma_K / eps_K > 2 (beyond the explicit step's real stability interval)
 * or a negative or non-finite value returns CMCG_ERR_INVALID_ARG and changes
 * nothing.  It applies to every later sweep and solve of the handle. */
int cmcg_set_conductivity(cmcg_handle* h, int problem, const double* sigma);

/* Limiting-amplitude baseline ("full wave", FW, Section 6): marches the
 * scheme with the time-harmonic source from rest for `periods` periods,
 * U = P_{psi,w}^periods 0, then returns the filtered field F_{psi,w} U of one
 * further period (Section 2.1).  The source is T-periodic, so P_{psi,w} U =
 * P_w U + P_{psi,w} 0: the march runs as one source sweep, then one source-free
 * sweep and one vector addition per further period (equal up to rounding).
 * Cost: periods + 1 sweeps, two of them with the source; no CG.  By
 * the limiting amplitude principle (Section 1) the result tends to the CMCG
 * result as periods grows when transients decay.  periods >= 0; buffers as in
 * cmcg_solve.  cmcg_fw_solve_batch runs every problem of a batch handle
 * (arrays of nprob host pointers, as in cmcg_solve_batch). */
int cmcg_fw_solve(cmcg_handle* h, const double* j_re, const double* j_im, int periods, double* e_re, double* e_im,
                  double* h_re, double* h_im);
int cmcg_fw_solve_batch(cmcg_handle* h, int periods, const double* const* j_re, const double* const* j_im,
                        double* const* e_re, double* const* e_im, double* const* h_re, double* const* h_im);

/* Sweep timing.  cmcg_profile_enable(h, 1) resets the counters and makes
 * every later period sweep record a CUDA event on the handle's stream before
 * its first and after its last stage; 0 stops recording.  cmcg_profile_read
 * waits for the recorded events and returns the summed sweep times and stage
 * launch counts, separately for source-free sweeps (P_w, P*_w) and sweeps with
 * the source or the filter (P_{psi,w}, F_{psi,w}).
 * A sweep's time covers its stage kernels back to back, launch gaps included.
 * Any output pointer may be NULL. */
int cmcg_profile_enable(cmcg_handle* h, int on);
int cmcg_profile_read(cmcg_handle* h, double* free_ms, int64_t* free_stages, double* source_ms,
                      int64_t* source_stages);

/* Measured arithmetic peaks of a device (a measurement utility; the paper has no
 * counterpart): *fp32_tflops from 8 independent FMA chains per thread on every
 * SM, *tf32_tflops from back-to-back tensor-core MMAs (tcgen05 kind::tf32,
 * M = 128, N = 256, K = 8, one accumulator in tensor memory per SM).  Each is
 * one timed launch after a warm-up launch.  Either pointer may be NULL (not
 * measured).  CMCG_ERR_DEVICE_TIMEOUT if the MMA wait (bounded, ~1 s) ran out. */
int cmcg_measure_peaks(int device, double* fp32_tflops, double* tf32_tflops);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of CMCG requests (no counterpart in the paper;
 * it serves many independent solves of the paper's method).
 *
 * A server holds registered models (mesh, eps, mu, omega, order) and a queue
 * of requests (one source each).  Worker threads, each with its own CUDA
 * stream, take the model of the oldest request (waiting at most max_wait_ms
 * for more of it) and run a pooled batch handle of that model as slots
 * (cmcg_slot_*): each round advances every busy slot by one step of its solve,
 * and between rounds queued requests of the model take the slots that finished
 * requests left free, while the other slots keep iterating.  Handles of
 * different workers run concurrently.  New handles are created only while the
 * server's device memory stays within hbm_budget_bytes (0 = no limit);
 * otherwise a worker waits for a pooled handle.  Every handle of a model uses
 * the kernel form chosen when the model was registered, so a request's result
 * is the one it gets when solved alone, whatever shares its handle.  Requests
 * carry a volume source only (no impedance-face data). */
typedef struct cmcg_server cmcg_server;

typedef struct cmcg_server_options {
  int device;
  int precision;      /* CMCG_FP32 (default) or CMCG_FP64 */
  int max_batch;      /* default slots per handle of a model (default 8) */
  int workers;        /* worker threads / streams (default 2) */
  double max_wait_ms; /* micro-batching window (default 2) */
  double tol;         /* CG tolerance of every request (default 1e-6) */
  int max_iter;       /* default 1000 */
  int64_t hbm_budget_bytes;
  int stage_variant;  /* 0: choose per model by timing; k > 0: as cmcg_options.stage_variant */
  int reserved[7];
} cmcg_server_options;

void cmcg_server_default_options(cmcg_server_options* opt);
int cmcg_server_create(const cmcg_server_options* opt, cmcg_server** out);

/* Registers a model (copied) with batch capacity max_batch (0 = server
 * default); builds its first handle.  *model receives its id. */
int cmcg_server_add_model(cmcg_server* s, const cmcg_mesh* mesh, const double* eps, const double* mu, double omega,
                          int order, int max_batch, int* model);

/* Queues one request (j_re, j_im: double[nt][3][Np], copied; j_im may be
 * NULL).  *ticket identifies it. */
int cmcg_server_submit(cmcg_server* s, int model, const double* j_re, const double* j_im, int64_t* ticket);

/* Result of a request.  wait == 0: returns CMCG_PENDING while it is queued or
 * running.  Otherwise (or once done) copies (e, h) (double[nt][3][Np] each; any
 * pointer may be NULL), the solve report, and latency_ms[0] = submit to
 * completion, latency_ms[1] = submit to start (may be NULL), forgets the
 * ticket and returns the request's status.  A ticket is taken by one poll:
 * while one thread waits on it, a poll of the same ticket from another thread
 * returns CMCG_ERR_INVALID_ARG (as does any poll after the result was taken). */
int cmcg_server_poll(cmcg_server* s, int64_t ticket, int wait, double* e_re, double* e_im, double* h_re,
                     double* h_im, cmcg_info* info, double* latency_ms);

/* Requests completed, requests queued, device bytes held, handles created. */
int cmcg_server_stats(cmcg_server* s, int64_t* completed, int64_t* queued, int64_t* bytes_in_use, int* handles);

/* Drains the queue, joins the workers and releases every handle. */
void cmcg_server_destroy(cmcg_server* s);

#ifdef __cplusplus
}
#endif

#endif /* CMCG_H */
