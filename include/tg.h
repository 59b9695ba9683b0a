/* tg.h -- C ABI of the GB300 library for the operator-split multispecies glioblastoma step.
 *
 * Model: Subramanian, Gholami, Biros, "Simulation of glioblastoma growth using a 3D
 * multispecies tumor model with mass effect" (arXiv:1810.05370).  Section 2 states the PDEs
 * (Eq. e:gog for the species, Eq. e:screening / e:lame / e:forcingfunction for the mass
 * effect, Eq. e:edema for the edema); Section 3 states the operator split that one call of
 * tg_step advances by dt:
 *   S0  diffusion faces and proliferation field from the step's start (Eq. e:diffusion_tensor,
 *       e:reaction_op);
 *   S1  semi-Lagrangian transport of p, i, n, g, w (conservative form) and f along v
 *       (Section 3, RK2 characteristics, cubic interpolation);
 *   S2  Crank-Nicolson diffusion of i, o and edema l, solved by Jacobi-preconditioned CG; the
 *       increment of i is taken from g and w in proportion g/(g+w);
 *   S3  reaction of p, i, n, g, w (Eq. e:p - e:w: logistic growth, go-or-grow switching,
 *       hypoxic death);  S4 oxygen reaction (Eq. e:ox);  S5 edema reaction (Eq. e:edema);
 *   S6  screened elasticity (eta I - L_h) u = -b (Eq. e:screening with Eq. e:lame and
 *       e:forcingfunction), CG from u extrapolated in time (see tg_reset_history),
 *       preconditioned by Jacobi
 *       or (Section 3) by the exact inverse of the constant-coefficient operator with the
 *       domain means of mu, lambda, eta;
 *   S7  v = (u^{n+1} - u^n) / dt.
 * Spatial operators are second-order finite differences on a periodic box (7-point
 * variable-coefficient diffusion, 19-point variable-coefficient Navier-Lame); the paper's
 * pseudo-spectral discretisation is not used.  The spectral elasticity preconditioner
 * (TG_PRECOND_SPECTRAL) inverts the finite-difference operator's own discrete symbol with
 * FFTs and needs every grid size to be a power of two between 4 and 2048.
 *
 * Conventions for every entry point:
 *  - Arrays are FP64, C-contiguous, indexed [z][y][x] (x fastest), n[0]*n[1]*n[2] elements,
 *    in DEVICE memory on the current CUDA device, and at least 16-byte aligned.
 *  - The library never allocates device memory.  The caller owns the state arrays and one
 *    workspace of tg_workspace_bytes() bytes; both are borrowed until tg_free.
 *  - All GPU work is ordered on the stream given to tg_init (a cudaStream_t, NULL = legacy
 *    default stream).  In TG_MIXED the oxygen solve of S2 runs on a second stream that the
 *    context creates on first use; it starts after and ends before the given stream's work
 *    around it (events), so callers see one stream.  Calls return after the work they queued
 *    has finished (the solvers read their convergence flags back), so buffers may be reused
 *    on return.
 *  - Errors are returned as tg_status; nothing is printed and no global state is kept.
 *    After any error other than TG_ERR_ARG the context refuses further work with
 *    TG_ERR_STATE (the state arrays are then unspecified) until it is freed.
 *  - A context is used by one host thread at a time.
 */
#ifndef TG_H
#define TG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tg_ctx tg_ctx;

typedef enum {
  TG_OK = 0,
  TG_ERR_ARG = 1,        /* invalid argument (null pointer, bad grid, dt <= 0, ...)            */
  TG_ERR_CUDA = 2,       /* a CUDA runtime call or kernel launch failed                       */
  TG_ERR_NOCONV = 3,     /* a CG solve reached its iteration limit                            */
  TG_ERR_NONFINITE = 4,  /* a residual norm became NaN or Inf                                 */
  TG_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up                                */
  TG_ERR_STATE = 6,      /* the context is unusable after an earlier error                   */
  TG_ERR_WORKSPACE = 7   /* workspace missing, too small or misaligned                        */
} tg_status;

typedef enum {
  TG_FP64 = 0,   /* every operation in FP64                                                   */
  TG_MIXED = 1   /* FP32 stencils and interpolation, FP64 reductions and outer refinement    */
} tg_precision;

/* Periodic box [0, L[0]) x [0, L[1]) x [0, L[2]) with n[d] nodes per axis, spacing
 * h_d = L[d] / n[d] (Section 3 uses a uniform grid on a fictitious box).  n[d] >= 4. */
typedef struct {
  int32_t n[3];
  double L[3];
} tg_grid;

/* Model parameters, Table t:setup.  Per-species arrays use the order
 * (tumor = p + i + n, gray matter g, white matter w, CSF f, background bg). */
typedef struct {
  double k_g, k_w, k_f, k_scale;   /* K = k_scale (k_g g + k_w w + k_f f)   Eq. e:diffusion_tensor */
  double rho_g, rho_w, rho_i_frac; /* rho = rho_g g + rho_w w; invasive rho_i = rho_i_frac rho    */
  double alpha0, beta0, gamma, sigma_b; /* Eq. e:alpha, e:beta, e:death                            */
  double o_hyp, o_inv, o_heal;     /* hypoxia / invasion thresholds, healthy oxygen level        */
  double delta_s, delta_p;         /* oxygen supply and consumption, Eq. e:ox                    */
  double eps_H;                    /* smoothed Heaviside H(x) = (1 + tanh(x / eps_H)) / 2          */
  double E[5], nu[5], eta[5];      /* Young's modulus, Poisson ratio, screening, Eq. e:lame       */
  double E_scale, zeta;            /* E multiplier; force b = zeta tanh(p+n) grad(p+n)           */
  double delta_e, delta_half, delta_l; /* edema source, half-saturation, drainage, Eq. e:edema     */
  double rtol_diff, rtol_elas;     /* CG stops at |r|_2 <= rtol |rhs|_2                          */
  int32_t maxit_diff, maxit_elas;  /* CG iteration limits (TG_ERR_NOCONV beyond)                */
  int32_t precond_elas;            /* elasticity preconditioner: TG_PRECOND_JACOBI,
                                      TG_PRECOND_SPECTRAL (Section 3: constant coefficients
                                      averaged over the domain, inverted by FFT) or
                                      TG_PRECOND_SPECTRAL_SCALED                             */
  int32_t model;                   /* TG_MODEL_MULTISPECIES (Eq. e:gog) or TG_MODEL_SINGLE   */
} tg_params;

#define TG_PRECOND_JACOBI 0
#define TG_PRECOND_SPECTRAL 1
/* TG_PRECOND_SPECTRAL_SCALED (this library's, not the paper's): the spectral inverse between
 * two diagonal scalings, z = s A0^{-1} (s r) with s = (D0 / D)^{1/2} per component and node,
 * D the diagonal of the variable-coefficient operator and D0 that of the constant-coefficient
 * one A0.  Symmetric positive definite; equal to TG_PRECOND_SPECTRAL where the coefficients
 * equal their means, exact for a diagonal operator.  On the brain workloads, whose domain-mean
 * screening is set by the background, it needs about a third of the plain spectral
 * preconditioner's iterations.  Same grid rule and workspace as TG_PRECOND_SPECTRAL. */
#define TG_PRECOND_SPECTRAL_SCALED 2

/* TG_MODEL_SINGLE: the single-species model of Eq. e:rd with its split from Section 3 --
 * semi-Lagrangian transport of (c, g, w) and f, Crank-Nicolson diffusion of c whose increment
 * leaves g and w in proportion g/(g+w), one Heun step of the logistic reaction
 * R = rho c (1 - c) (Eq. e:reac_op) with g and w losing R in the same proportion, then the
 * elasticity solve with b = zeta tanh(c) grad c (Eq. e:force) and Lame coefficients with c as
 * the tumor species.  The tumor density c is carried in tg_state.p; i and n must be zero
 * (they are transported but nothing creates them); o and l are left untouched.  Contexts
 * with TG_INIT_ADJOINT, tapes and batches support the multispecies model only. */
#define TG_MODEL_MULTISPECIES 0
#define TG_MODEL_SINGLE 1

/* Device pointers to the caller's state (species and materials of Section 2.3; u is the
 * displacement of Eq. e:screening, v = u_t its velocity).  bg is read only. */
typedef struct {
  double *p, *i, *n, *g, *w, *f, *o, *l, *bg;
  double *u[3], *v[3];
} tg_state;

/* Solver statistics of one call.  it_* of the last step; *_total summed over the call. */
typedef struct {
  int64_t steps;
  int32_t it_diff[3];        /* CG iterations of the i, o, l solves                           */
  int32_t it_elas;           /* CG iterations of the elasticity solve (inner, summed, in MIXED) */
  int32_t it_elas_outer;     /* refinement sweeps of the elasticity solve (1 in FP64)        */
  double relres_diff[3];     /* final |r| / |rhs|                                            */
  double relres_elas;
  int64_t it_diff_total;
  int64_t it_elas_total;
  int64_t launches;          /* CUDA kernels this call queued                                */
  double t_elas_matvec_ms;   /* with timing on: summed duration of the elasticity operator   */
  int64_t n_elas_matvec;     /*   kernel over the launches that did work, and their count    */
  double t_phase_ms[4];      /* with timing on: device time of S0-S1, S2, S3-S5 and S6-S7     */
                             /*   (event to event on the stream), summed over the call's steps */
  double t_spec_update_ms;   /* with timing on, TG_MIXED with a spectral preconditioner: summed */
  int64_t n_spec_update;     /*   duration of the CG update fused with the first FFT pass and  */
                             /*   its count (the launches that did work)                       */
} tg_stats;

/* Bytes of workspace tg_init needs for this grid, parameters and precision (0 on invalid
 * arguments, including a spectral preconditioner on a grid it does not support).  params may
 * be NULL: Jacobi preconditioning.  Only params->precond_elas changes the size. */
size_t tg_workspace_bytes(const tg_grid* grid, const tg_params* params, tg_precision prec);

/* Bytes of workspace for a context created with TG_INIT_ADJOINT (adjoint scratch included). */
size_t tg_workspace_bytes_adjoint(const tg_grid* grid, const tg_params* params,
                                  tg_precision prec);

/* Bytes of one step's tape (the forward values tg_adjoint_step needs): 26 FP64 fields. */
size_t tg_tape_bytes(const tg_grid* grid);

/* Create a context over the caller's state and workspace and compute the initial
 * displacement u^0 from the initial species (Eq. e:gog_elasticity at t = 0, CG from u = 0),
 * setting v^0 = 0.  With flags & TG_INIT_KEEP_UV the given u, v are kept (resuming from a
 * saved state).  With flags & TG_INIT_ADJOINT the workspace must hold
 * tg_workspace_bytes_adjoint() bytes and the context can run tg_adjoint_step.  stats may be
 * NULL.  On success *out receives the context. */
#define TG_INIT_KEEP_UV 1u
#define TG_INIT_ADJOINT 2u
tg_status tg_init(const tg_grid* grid, const tg_params* params, tg_precision prec,
                  const tg_state* state, void* workspace, size_t workspace_bytes,
                  void* cuda_stream, uint32_t flags, tg_ctx** out, tg_stats* stats);

/* Advance the state by nsteps steps of size dt (Section 3 multispecies split S0-S7).
 * tape is NULL, or (with nsteps == 1) a 256-byte aligned device buffer of tg_tape_bytes()
 * that receives the step's forward values for tg_adjoint_step.  stats may be NULL. */
tg_status tg_step(tg_ctx* ctx, double dt, int32_t nsteps, void* tape, tg_stats* stats);

/* One step of dt for a caller whose state lives in host memory.  in and out hold HOST
 * pointers (page-locked for asynchronous copies; pageable memory works but copies
 * synchronously), one array of nvox doubles per field in the layout of tg_state; they may be
 * the same.  The state is copied from in into the context's device state, the step runs
 * (tg_step, no tape), and the new state is copied to out, bg included (unchanged).  The
 * copies overlap the step where the split allows: u goes up on a copy stream while S0-S5
 * run (only S6 reads it) and p, i, n, g, w, f, o, l, bg come down while S6-S7 run (nothing
 * after S5 changes them); the other fields go up before S0, and u, v come down after S7.
 * Returns once out holds the new state.  Errors as tg_step. */
tg_status tg_step_host(tg_ctx* ctx, const tg_state* in, tg_state* out, double dt,
                       tg_stats* stats);

/* Discrete adjoint of one step (the paper's stated next goal, adjoint-based parameter
 * estimation, Section 5).  tape holds what tg_step recorded for this step.  lam holds the
 * adjoint of every state field after the step (device arrays, bg ignored) and is
 * overwritten with the adjoint before the step.  grad[5] (host) is incremented by the step's
 * contribution to dJ/d(k_scale, rho, o_hyp, o_inv, E_scale), where rho moves rho_g and rho_w
 * together.  Linear solves are differentiated as exact inverses; the adjoint elasticity
 * solve iterates in FP32 inside FP64 residual refinement and stops at the FP64 tolerance
 * rtol_elas, like the forward solve of TG_MIXED.  The context must have been created with
 * TG_INIT_ADJOINT; its state arrays are not used except bg. */
tg_status tg_adjoint_step(tg_ctx* ctx, double dt, const void* tape, tg_state* lam,
                          double grad[5]);

/* Contribution of the initial elasticity solve u^0 = M(q^0)^{-1}(-b(q^0)) to grad (only
 * E_scale enters it), given the adjoint lam_u of u^0.  The context's state must hold q^0 and
 * u^0.  Needs TG_INIT_ADJOINT. */
tg_status tg_adjoint_init(tg_ctx* ctx, double* const lam_u[3], double grad[5]);

/* Solve (eta I - L_h) u = rhs with preconditioned CG, coefficients from the current
 * state (Eq. e:lame), starting from the given u.  rhs == NULL means rhs = -b with the force
 * b of Eq. e:forcingfunction from the current state (the solve S6 performs); otherwise rhs
 * holds three device arrays.  u holds three device arrays, overwritten with the solution. */
tg_status tg_solve_elasticity(tg_ctx* ctx, double* const rhs[3], double* u[3], tg_stats* stats);

/* Mass-effect diagnostics of the current state (Section 3): per node, the trace of the stress
 * T = lambda tr(E) I + 2 mu E (Eq. e:hook, Lame coefficients of Eq. e:lame from the state),
 * the in-plane maximum shear stress sqrt(((T_xx - T_yy)/2)^2 + T_xy^2) (Eq. e:princ_stress)
 * and J = det(I + grad u) (Eq. e:jacobian), grad u by centred differences; and summaries.
 * fields: NULL, or three device arrays (any of them NULL) receiving tr T, the shear and J.
 * seed (host, physical coordinates in the box) and u_threshold define d_max.  out (host,
 * required) receives the summaries. */
typedef struct {
  double jac_min, jac_max;   /* extremes of J                                               */
  double jac_dev_l2;         /* (h_x h_y h_z sum (J - 1)^2)^(1/2)                             */
  double trace_min, trace_max;
  double shear_max;          /* largest in-plane maximum shear stress                       */
  double d_max;              /* largest periodic distance from seed of a node with
                                |u| >= u_threshold (0 if there is none)                     */
} tg_diag;
tg_status tg_diagnostics(tg_ctx* ctx, const double seed[3], double u_threshold,
                         double* const fields[3], tg_diag* out);

/* Replace the parameters used by later calls (e.g. a parameter sweep on one context).
 * Switching to TG_PRECOND_SPECTRAL or TG_PRECOND_SPECTRAL_SCALED needs a context whose
 * workspace was sized for either (TG_ERR_WORKSPACE otherwise).  Clears the step history (see
 * tg_reset_history). */
tg_status tg_set_params(tg_ctx* ctx, const tg_params* params);

/* The starting guess of a step's elasticity solve (the paper names none) is u extrapolated in
 * time: linearly, u^n + dt v^n, on a context's first step, and quadratically,
 * u^n + dt v^n + dt (v^n - v^{n-1}), on later ones, for which the context keeps v^{n-1} in its
 * workspace.  The solution is the same within rtol_elas either way; the quadratic start needs
 * fewer iterations.  A caller that overwrites u or v between steps (restoring a checkpoint,
 * say) calls tg_reset_history so that the next step starts linearly again; without it the
 * result is still correct to the tolerance, only the iteration count (and so the exact
 * iterate) differs.  tg_init and tg_set_params clear the history too. */
tg_status tg_reset_history(tg_ctx* ctx);

/* Optional kernel timing for profiling.  With enable != 0 every kernel launch of tg_step and
 * tg_solve_elasticity is bracketed by two CUDA events on the stream it is launched on, and
 * the elapsed time between them is added to that kernel's total.  A CG solve queues its
 * iterations ahead of its convergence test, and the iterations queued after convergence
 * return at once; their launches are left out, so the totals cover the launches that did
 * work.  The stats of a call report the elasticity operator's and the mixed spectral CG
 * update's totals (t_elas_matvec_ms, t_spec_update_ms); tg_kernel_times reports every
 * kernel.  Switching timing on resets the totals.  The events are created on first use
 * (host-side objects, no device allocation) and reused every step. */
tg_status tg_set_timing(tg_ctx* ctx, int32_t enable);

/* One kernel's timing totals since timing was last switched on (see tg_set_timing). */
typedef struct {
  const char* name;    /* the kernel's name in the library (static string)                 */
  double ms;           /* summed device time of its launches that did work, in ms           */
  int64_t launches;    /* how many launches that sum covers                                  */
} tg_kernel_time;

/* Writes up to capacity entries (kernels with at least one timed launch, in a fixed order)
 * to out and returns how many such kernels there are; -1 if ctx is NULL, capacity < 0 or out
 * is NULL with capacity > 0.  Host only; reads no device memory. */
int32_t tg_kernel_times(const tg_ctx* ctx, tg_kernel_time* out, int32_t capacity);

/* Elasticity solve that allocates nothing and needs no workspace or context.
 *
 * The paper has no counterpart to this entry point; it exists for callers that may not
 * allocate device memory themselves, for example code running inside a host application
 * that owns every device allocation (a fixed memory pool or budget), or a latency-critical
 * loop that cannot afford the implicit device synchronisation of cudaMalloc.  Instead of a
 * caller workspace it uses one scratch array compiled into the library
 * (TG_STATIC_SCRATCH_BYTES of device memory, held on every GPU that loads the library until
 * the process exits), so it only accepts small grids: n[0]*n[1]*n[2] <= TG_STATIC_MAX_VOXELS.
 * Larger grids are rejected with TG_ERR_WORKSPACE before any GPU work.
 *
 * It computes what tg_solve_elasticity computes on a context over the same state: the Lame
 * and screening fields from the state's species (p, i, n, g, w, f, bg are read; the other
 * state pointers are ignored), then (eta I - L_h) u = rhs by Jacobi-preconditioned CG from the
 * given u (params->precond_elas is ignored here); rhs == NULL means rhs = -b (the force of Eq. e:forcingfunction).  All work goes to
 * cuda_stream and the call returns after it has finished.
 *
 * The first call on a device looks up the scratch array's device address (with that device
 * current) and caches it; make that first call before any stream capture.  Every call on a
 * device shares the one scratch array and leaves its contents behind: calls whose GPU work
 * overlaps (two host threads, or two streams) race and give wrong results, so serialise them. */
#define TG_STATIC_MAX_VOXELS 32768
#define TG_STATIC_SCRATCH_BYTES (16u << 20)
tg_status tg_solve_elasticity_static(const tg_grid* grid, const tg_params* params,
                                     const tg_state* state, double* const rhs[3], double* u[3],
                                     void* cuda_stream, tg_stats* stats);

/* ---------------------------------------------------------------------------------------
 * Batches: many simulations (different grids and parameters) stepped together in TG_MIXED
 * precision.  Each simulation has its own state (caller-owned, as for tg_init); the batch
 * runs the Crank-Nicolson and elasticity solves of all simulations in persistent cooperative
 * kernels that walk one list of (simulation, tile) work items, with per-simulation CG state,
 * and replays one captured CUDA graph per step (a stream other than the legacy default
 * stream is needed for the graph; otherwise the same work is launched directly).  Grid-wide
 * waits inside the persistent kernels are bounded in time (TG_ERR_TIMEOUT). */
typedef struct tg_batch tg_batch;

typedef struct {
  int64_t steps;
  int64_t it_elas_total;    /* inner FP32 elasticity iterations, summed over simulations */
  int64_t it_elas_max;      /* largest per-simulation count of one step                   */
  int64_t sweeps_total;     /* refinement sweeps (residual evaluations), summed             */
  int64_t it_diff_total;    /* CN iterations (three solves), summed                          */
  double relres_elas_max;   /* largest final |r|/|rhs| of an elasticity solve               */
  int64_t launches;         /* kernels launched (the graph's count per replay)              */
  int32_t graph;            /* 1 when the step ran as a replayed CUDA graph                 */
  int32_t tile_depth;       /* z depth of the work tiles                                    */
  int32_t coop_blocks;      /* blocks of the persistent elasticity solver                   */
  int32_t pad;
} tg_batch_stats;

typedef struct {            /* what tg_batch_autotune measured */
  int32_t count;
  int32_t best_zc, best_blocks;
  int32_t zc[32], blocks[32];
  float ms[32];
} tg_batch_tune;

/* Workspace bytes for a batch (per-simulation workspaces plus the batch lists); 0 if invalid.
 * Only TG_MIXED is supported. */
size_t tg_batch_workspace_bytes(int32_t nsims, const tg_grid* grids, tg_precision prec);

/* Create the batch: nsims simulations with their own grid, parameters and state; computes
 * each u^0 (as tg_init).  All work goes to cuda_stream. */
tg_status tg_batch_init(int32_t nsims, const tg_grid* grids, const tg_params* params,
                        const tg_state* states, tg_precision prec, void* workspace,
                        size_t workspace_bytes, void* cuda_stream, tg_batch** out);

/* Choose the work-tile depth and the persistent grid size by timing a short run of the
 * elasticity inner solver on the current states (which it does not change).  result may be
 * NULL. */
tg_status tg_batch_autotune(tg_batch* batch, double dt, tg_batch_tune* result);

/* Concurrent batches.  The same simulations, each stepped by the single-simulation path --
 * its own elasticity preconditioner as its params give it (the scaled spectral one where the
 * grid allows it), the double-FP32 refinements, the Neumann inner CN solves, the extrapolated
 * elasticity starts -- on a CUDA stream of its own.  A pool of nthreads host threads (0: up to
 * 8) drives them: each thread takes the largest simulation not yet stepped and advances it by
 * all nsteps of a tg_batch_step call, so several simulations' kernels share the GPU.  Members
 * may mix grids, preconditioners, models and precisions' solvers (prec applies to all).  The
 * workspace holds one tg_workspace_bytes(grid, params, prec) region per member, each rounded
 * up to 256 bytes: tg_batch_concurrent_workspace_bytes gives the total, 0 if any member is
 * invalid.  The states are read after the work already queued on cuda_stream; each
 * tg_batch_step returns with every member's step complete.  tg_batch_autotune has nothing to
 * tune (result zeroed) and tg_batch_set_timeout nothing to limit; tg_batch_stats report the
 * summed iteration counts and launches (graph, tile_depth, coop_blocks are 0).  The first
 * member that fails stops the others at their next simulation and its status is returned;
 * the batch then refuses further steps (TG_ERR_STATE). */
size_t tg_batch_concurrent_workspace_bytes(int32_t nsims, const tg_grid* grids,
                                           const tg_params* params, tg_precision prec);
tg_status tg_batch_concurrent_init(int32_t nsims, const tg_grid* grids, const tg_params* params,
                                   const tg_state* states, tg_precision prec, void* workspace,
                                   size_t workspace_bytes, int32_t nthreads, void* cuda_stream,
                                   tg_batch** out);

/* Advance every simulation by nsteps steps of dt (the split of tg_step). */
tg_status tg_batch_step(tg_batch* batch, double dt, int32_t nsteps, tg_batch_stats* stats);

/* Time limit of one grid-wide wait in the persistent kernels (default 20 s). */
tg_status tg_batch_set_timeout(tg_batch* batch, uint64_t timeout_ns);

void tg_batch_free(tg_batch* batch);

/* Release the context (host memory only; the caller's buffers are untouched). */
void tg_free(tg_ctx* ctx);

/* Static description of a status code. */
const char* tg_error_string(tg_status status);

#ifdef __cplusplus
}
#endif
#endif
