/* oracle.h -- plain, slow CPU restatement of the operator-split glioblastoma step.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the reference the CUDA library is checked against.  It
 * shares no code, header, table or helper with the CUDA library, and only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Model: Subramanian, Gholami, Biros, "Simulation of glioblastoma growth using a 3D
 * multispecies tumor model with mass effect" (arXiv:1810.05370).  Section 2 gives the PDEs,
 * Section 3 the operator split.  Every routine below names the equation it restates.
 *
 * Grid: periodic box, n[0] x n[1] x n[2] nodes (x fastest), spacing h_d = L[d] / n[d],
 * arrays indexed [z][y][x].  Scalar type real_t is double, or double complex when built
 * with -DOR_COMPLEX (complex-step differentiation; branches then use real parts).
 */
#ifndef TG_ORACLE_H
#define TG_ORACLE_H
#include <stdint.h>

#ifdef OR_COMPLEX
#include <complex.h>
typedef double complex real_t;
#else
typedef double real_t;
#endif

typedef struct { int32_t n[3]; double L[3]; } or_grid;

/* Parameter block, Table t:setup.  Species order of E, nu, eta: tumor (p+i+n), gray matter,
 * white matter, CSF, background. */
typedef struct {
  real_t k_g, k_w, k_f, k_scale;          /* Eq. e:diffusion_tensor                       */
  real_t rho_g, rho_w, rho_i_frac;        /* Eq. e:reaction_op, e:gog_reac_inv_op         */
  real_t alpha0, beta0, gamma, sigma_b;   /* Eq. e:alpha, e:beta, e:death                 */
  real_t o_hyp, o_inv, o_heal;            /* Eq. e:death, e:gog_reac_op, e:o              */
  real_t delta_s, delta_p, eps_H;         /* Eq. e:ox; smoothed Heaviside width           */
  real_t E[5], nu[5], eta[5];             /* Eq. e:lame, e:screening                      */
  real_t E_scale, zeta;                   /* E multiplier; Eq. e:forcingfunction          */
  real_t delta_e, delta_half, delta_l;    /* Eq. e:edema                                  */
  double rtol_diff, rtol_elas;            /* Krylov stopping: |r| <= rtol |rhs|           */
  int32_t maxit_diff, maxit_elas;
  int32_t precond_elas;                   /* 0 Jacobi, 1 spectral (Section 3)             */
  int32_t model;                          /* 0 multispecies, 1 single species (Eq. e:rd)  */
} or_params;

typedef struct {
  real_t *p, *i, *n, *g, *w, *f, *o, *l, *bg;   /* species and materials               */
  real_t *u[3], *v[3];                           /* displacement, velocity              */
  /* optional history of the elasticity solve's starting guess: the velocity at the start of
   * the previous step (vprev[0] == NULL: none kept); vprev_valid says whether it holds one.
   * or_init clears vprev_valid, or_step uses and then refreshes it. */
  real_t *vprev[3];
  int32_t vprev_valid;
} or_state;

typedef struct {
  int32_t it_diff[3];      /* CG iterations of the i, o, l Crank-Nicolson solves          */
  int32_t it_elas;         /* CG iterations of the elasticity solve                       */
  double relres_diff[3];   /* final |r| / |rhs|                                           */
  double relres_elas;
} or_stats;

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_NOCONV = 3, OR_ERR_NONFINITE = 4 };

/* Full step and initialisation (Section 3, multispecies splitting). */
int or_init(const or_grid*, const or_params*, or_state*, or_stats*);
int or_step(const or_grid*, const or_params*, double dt, or_state*, or_stats*);

/* Building blocks, exported for the pins. */
void or_diffusion_node_K(const or_grid*, const or_params*, const real_t* g, const real_t* w,
                         const real_t* f, real_t* K);
void or_diffusion_faces(const or_grid*, const real_t* K, real_t* Kface0, real_t* Kface1,
                        real_t* Kface2);
void or_diffusion_apply(const or_grid*, const real_t* Kf0, const real_t* Kf1, const real_t* Kf2,
                        const real_t* c, real_t* out);
int or_cn_solve(const or_grid*, const real_t* Kf0, const real_t* Kf1, const real_t* Kf2,
                double dt, const real_t* c_in, real_t* c_out, double rtol, int32_t maxit,
                int32_t* iters, double* relres);
void or_lame(const or_grid*, const or_params*, const real_t* p, const real_t* i, const real_t* n,
             const real_t* g, const real_t* w, const real_t* f, const real_t* bg, real_t* mu,
             real_t* lam, real_t* eta);
void or_force(const or_grid*, const or_params*, const real_t* p, const real_t* n, real_t* bx,
              real_t* by, real_t* bz);
void or_elasticity_apply(const or_grid*, const real_t* mu, const real_t* lam, const real_t* eta,
                         const real_t* u3, real_t* out3);
int or_elasticity_solve(const or_grid*, const real_t* mu, const real_t* lam, const real_t* eta,
                        const real_t* rhs3, real_t* u3, double rtol, int32_t maxit,
                        int32_t precond, int32_t* iters, double* relres);
void or_dft3(const or_grid*, double* re, double* im, int sgn);
void or_elasticity_spectral(const or_grid*, double mu0, double lam0, double eta0,
                            const double* r3, double* z3);
/* Preconditioner 2: z = s * A0^{-1} (s * r), s = (D0 / D)^{1/2} (diagonals of A0 and A);
 * real build only */
void or_elasticity_scaled_spectral(const or_grid*, const double* mu, const double* lam,
                                   const double* eta, const double* r3, double* z3);
real_t or_interp(const or_grid*, const real_t* q, real_t X, real_t Y, real_t Z);
void or_divergence(const or_grid*, const real_t* vx, const real_t* vy, const real_t* vz,
                   real_t* div);
void or_sl_advect(const or_grid*, double dt, const real_t* vx, const real_t* vy, const real_t* vz,
                  real_t* const* q_in, real_t* const* q_out);
real_t or_heaviside(const or_params*, real_t x);
void or_react(const or_grid*, const or_params*, double dt, const real_t* rho, real_t* p,
              real_t* i, real_t* n, real_t* g, real_t* w, real_t* o, real_t* l);
void or_react_single(const or_grid*, double dt, const real_t* rho, real_t* c, real_t* g,
                     real_t* w);
/* Mass-effect diagnostics (Section 3): trace of the stress T = lambda tr(E) I + 2 mu E
 * (Eq. e:hook), the in-plane maximum shear stress of Eq. e:princ_stress and
 * J = det(I + grad u) (Eq. e:jacobian), with centred differences for grad u. */
void or_diagnostics(const or_grid*, const real_t* mu, const real_t* lam, const real_t* u3,
                    real_t* trace, real_t* tau, real_t* jac);
/* largest periodic distance from the point seed of a node with |u| >= thr (0 if none) */
double or_displacement_extent(const or_grid*, const real_t* u3, const double seed[3],
                              double thr);
#endif
