/* oracle.c -- plain CPU restatement of the operator-split multispecies step (FP64).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA library is checked against.  Loops are
 * written out literally, one formula per line, without blocking or fusion, so that each can
 * be read against the paper.  Reductions are summed over fixed 4096-element blocks and then
 * in block order, so the result does not depend on the OpenMP thread count.
 *
 * Readings of the paper that this file follows (the paper leaves these open):
 *  - spatial operators are second-order finite differences on the periodic box, not the
 *    paper's pseudo-spectral ones (Section 3);
 *  - the split is the sequence of Section 3 applied once per step (first-order Lie);
 *  - the elasticity solve is (eta I - L_h) u = -b, i.e. Eq. e:screening moved to SPD form;
 *    it is symmetric, so CG replaces the paper's GMRES; it is preconditioned either by
 *    Jacobi or, as in Section 3, by the exact inverse of the constant-coefficient operator
 *    with the domain means of mu, lambda and eta -- for the finite-difference operator that
 *    inverse is diagonal in the discrete Fourier basis (one 3x3 system per wave vector);
 *    the diffusion solves use Jacobi;
 *  - the diffusion face coefficient is the harmonic mean of the two node values (zero when
 *    both are zero), node K clamped at zero;
 *  - the unqualified "D" in the g, w equations (Eq. e:gm_wm, e:w) is D i: the Crank-Nicolson
 *    increment of i is taken from g and w in proportion g/(g+w) (zero where g+w <= 0);
 *  - smoothed Heaviside H(x) = (1 + tanh(x / eps_H)) / 2 (evaluated as a logistic);
 *  - "explicit" reaction sub-steps are one Heun (RK2) step each; p, i, n, g, w use the
 *    post-diffusion oxygen and the proliferation field of the step's start;
 *  - diffusion coefficients and rho come from the step's start; Lame, eta and the force
 *    from the post-reaction state;
 *  - semi-Lagrangian interpolation is tricubic Lagrange on the 4^3 nodes floor(X)-1..+2,
 *    coordinates in index units, periodic wrap; the conservative source is -q div v with
 *    div v from centred differences.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef OR_COMPLEX
#define RE(x) creal(x)
#define TANH(x) ctanh(x)
#define EXP(x) cexp(x)
#define SQRT_RE(x) sqrt(creal(x))
#else
#define RE(x) (x)
#define TANH(x) tanh(x)
#define EXP(x) exp(x)
#define SQRT_RE(x) sqrt(x)
#endif

/* ---------------------------------------------------------------- grid helpers */

static int64_t nvox(const or_grid* G) { return (int64_t)G->n[0] * G->n[1] * G->n[2]; }
static double hd(const or_grid* G, int d) { return G->L[d] / G->n[d]; }

static int64_t wrapi(int64_t a, int64_t n) {
  int64_t r = a % n;
  return r < 0 ? r + n : r;
}

/* linear index of node c + s1 e_d1 + s2 e_d2 (periodic); d = -1 means no shift */
static int64_t at(const or_grid* G, const int64_t c[3], int d1, int s1, int d2, int s2) {
  int64_t q[3] = {c[0], c[1], c[2]};
  if (d1 >= 0) q[d1] += s1;
  if (d2 >= 0) q[d2] += s2;
  return (wrapi(q[2], G->n[2]) * G->n[1] + wrapi(q[1], G->n[1])) * G->n[0] + wrapi(q[0], G->n[0]);
}

static void coords(const or_grid* G, int64_t lin, int64_t c[3]) {
  c[0] = lin % G->n[0];
  c[1] = (lin / G->n[0]) % G->n[1];
  c[2] = lin / ((int64_t)G->n[0] * G->n[1]);
}

/* ---------------------------------------------------------------- reductions */

#define RBLK 4096
static real_t dot(int64_t m, const real_t* x, const real_t* y) {
  int64_t nb = (m + RBLK - 1) / RBLK;
  real_t* part = (real_t*)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(real_t));
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nb; ++b) {
    real_t s = 0;
    int64_t e1 = (b + 1) * RBLK < m ? (b + 1) * RBLK : m;
    for (int64_t e = b * RBLK; e < e1; ++e) s += x[e] * y[e];
    part[b] = s;
  }
  real_t s = 0;
  for (int64_t b = 0; b < nb; ++b) s += part[b];
  free(part);
  return s;
}

/* ---------------------------------------------------------------- PCG
 * Solves A x = b from the given x with preconditioner z = M(r); stops when
 * |r|_2 <= rtol |b|_2 (Section 3: CG for the diffusion solve, a Krylov method for the
 * elasticity solve). */
typedef void (*apply_fn)(const void* ctx, const real_t* x, real_t* y);
typedef void (*prec_fn)(const void* ctx, int64_t m, const real_t* r, real_t* z);

/* Jacobi: z = D^{-1} r, ctx the array of inverse diagonal entries */
static void jacobi_prec(const void* ctx, int64_t m, const real_t* r, real_t* z) {
  const real_t* dinv = (const real_t*)ctx;
  for (int64_t e = 0; e < m; ++e) z[e] = dinv[e] * r[e];
}

static int pcg(int64_t m, apply_fn A, const void* ctx, prec_fn M, const void* mctx,
               const real_t* b, real_t* x, double rtol, int32_t maxit, int32_t* iters,
               double* relres) {
  real_t* r = (real_t*)malloc((size_t)m * sizeof(real_t));
  real_t* z = (real_t*)malloc((size_t)m * sizeof(real_t));
  real_t* p = (real_t*)malloc((size_t)m * sizeof(real_t));
  real_t* q = (real_t*)malloc((size_t)m * sizeof(real_t));
  int status = OR_OK;
  int32_t it = 0;
  double bnorm = SQRT_RE(dot(m, b, b));
  double rnorm = 0.0;
  if (bnorm == 0.0) {
    for (int64_t e = 0; e < m; ++e) x[e] = 0;
    goto done;
  }
  A(ctx, x, q);
  for (int64_t e = 0; e < m; ++e) r[e] = b[e] - q[e];
  M(mctx, m, r, z);
  for (int64_t e = 0; e < m; ++e) p[e] = z[e];
  real_t rz = dot(m, r, z);
  rnorm = SQRT_RE(dot(m, r, r));
  while (rnorm > rtol * bnorm) {
    if (!isfinite(rnorm)) { status = OR_ERR_NONFINITE; break; }
    if (it >= maxit) { status = OR_ERR_NOCONV; break; }
    A(ctx, p, q);
    real_t alpha = rz / dot(m, p, q);
    for (int64_t e = 0; e < m; ++e) x[e] += alpha * p[e];
    for (int64_t e = 0; e < m; ++e) r[e] -= alpha * q[e];
    M(mctx, m, r, z);
    real_t rz_new = dot(m, r, z);
    rnorm = SQRT_RE(dot(m, r, r));
    real_t beta = rz_new / rz;
    rz = rz_new;
    for (int64_t e = 0; e < m; ++e) p[e] = z[e] + beta * p[e];
    ++it;
  }
  if (status == OR_OK && !isfinite(rnorm)) status = OR_ERR_NONFINITE;
done:
  if (iters) *iters = it;
  if (relres) *relres = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  free(r); free(z); free(p); free(q);
  return status;
}

/* ---------------------------------------------------------------- diffusion
 * Eq. e:diffusion_op / e:diffusion_tensor:  D c = div(K grad c),  K = k_g g + k_w w (+ k_f f),
 * all scaled by k_scale.  Discretely
 *   (D_h c)_j = sum_d [ K_{j+1/2 e_d} (c_{j+e_d} - c_j) - K_{j-1/2 e_d} (c_j - c_{j-e_d}) ] / h_d^2. */
void or_diffusion_node_K(const or_grid* G, const or_params* P, const real_t* g, const real_t* w,
                         const real_t* f, real_t* K) {
  int64_t m = nvox(G);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    real_t k = P->k_scale * (P->k_g * g[e] + P->k_w * w[e] + P->k_f * f[e]);
    K[e] = RE(k) > 0.0 ? k : 0.0;
  }
}

/* face between node j and j + e_d: harmonic mean 2 K_a K_b / (K_a + K_b), 0 if both are 0 */
void or_diffusion_faces(const or_grid* G, const real_t* K, real_t* Kf0, real_t* Kf1, real_t* Kf2) {
  real_t* Kf[3] = {Kf0, Kf1, Kf2};
  int64_t m = nvox(G);
  for (int d = 0; d < 3; ++d) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
      int64_t c[3];
      coords(G, e, c);
      real_t a = K[e], b = K[at(G, c, d, +1, -1, 0)];
      Kf[d][e] = RE(a + b) > 0.0 ? 2.0 * a * b / (a + b) : 0.0;
    }
  }
}

void or_diffusion_apply(const or_grid* G, const real_t* Kf0, const real_t* Kf1, const real_t* Kf2,
                        const real_t* c, real_t* out) {
  const real_t* Kf[3] = {Kf0, Kf1, Kf2};
  int64_t m = nvox(G);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int64_t q[3];
    coords(G, e, q);
    real_t s = 0;
    for (int d = 0; d < 3; ++d) {
      int64_t jp = at(G, q, d, +1, -1, 0), jm = at(G, q, d, -1, -1, 0);
      double h = hd(G, d);
      s += (Kf[d][e] * (c[jp] - c[e]) - Kf[d][jm] * (c[e] - c[jm])) / (h * h);
    }
    out[e] = s;
  }
}

typedef struct { const or_grid* G; const real_t* Kf[3]; double dt; real_t* tmp; } cn_ctx;

/* Crank-Nicolson left operator (1 - dt/2 D) x (Section 3, diffusion sub-step) */
static void cn_apply(const void* vctx, const real_t* x, real_t* y) {
  const cn_ctx* C = (const cn_ctx*)vctx;
  or_diffusion_apply(C->G, C->Kf[0], C->Kf[1], C->Kf[2], x, C->tmp);
  int64_t m = nvox(C->G);
  for (int64_t e = 0; e < m; ++e) y[e] = x[e] - 0.5 * C->dt * C->tmp[e];
}

/* (1 - dt/2 D) c_out = (1 + dt/2 D) c_in, CG from c_out = c_in (Section 3) */
int or_cn_solve(const or_grid* G, const real_t* Kf0, const real_t* Kf1, const real_t* Kf2,
                double dt, const real_t* c_in, real_t* c_out, double rtol, int32_t maxit,
                int32_t* iters, double* relres) {
  int64_t m = nvox(G);
  real_t* rhs = (real_t*)malloc((size_t)m * sizeof(real_t));
  real_t* dinv = (real_t*)malloc((size_t)m * sizeof(real_t));
  real_t* tmp = (real_t*)malloc((size_t)m * sizeof(real_t));
  const real_t* Kf[3] = {Kf0, Kf1, Kf2};
  or_diffusion_apply(G, Kf0, Kf1, Kf2, c_in, tmp);
  for (int64_t e = 0; e < m; ++e) rhs[e] = c_in[e] + 0.5 * dt * tmp[e];
  for (int64_t e = 0; e < m; ++e) {
    int64_t q[3];
    coords(G, e, q);
    real_t diag = 1.0;
    for (int d = 0; d < 3; ++d) {
      double h = hd(G, d);
      diag += 0.5 * dt * (Kf[d][e] + Kf[d][at(G, q, d, -1, -1, 0)]) / (h * h);
    }
    dinv[e] = 1.0 / diag;
  }
  if (c_out != c_in) memcpy(c_out, c_in, (size_t)m * sizeof(real_t));
  cn_ctx C = {G, {Kf0, Kf1, Kf2}, dt, tmp};
  int st = pcg(m, cn_apply, &C, jacobi_prec, dinv, rhs, c_out, rtol, maxit, iters, relres);
  free(rhs); free(dinv); free(tmp);
  return st;
}

/* ---------------------------------------------------------------- elasticity
 * Eq. e:lame: mu = sum_s E_s / (2 (1 + nu_s)) iota_s,
 *             lambda = sum_s nu_s E_s / ((1 - 2 nu_s)(1 + nu_s)) iota_s,
 * species iota = (p + i + n, g, w, f, bg), each E_s scaled by E_scale; the screening
 * coefficient (Eq. e:screening) is mixed the same way, eta = sum_s eta_s iota_s. */
void or_lame(const or_grid* G, const or_params* P, const real_t* p, const real_t* i, const real_t* n,
             const real_t* g, const real_t* w, const real_t* f, const real_t* bg, real_t* mu,
             real_t* lam, real_t* eta) {
  int64_t m = nvox(G);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    real_t iota[5] = {p[e] + i[e] + n[e], g[e], w[e], f[e], bg[e]};
    real_t smu = 0, slam = 0, seta = 0;
    for (int s = 0; s < 5; ++s) {
      real_t E = P->E_scale * P->E[s], nu = P->nu[s];
      smu += E / (2.0 * (1.0 + nu)) * iota[s];
      slam += nu * E / ((1.0 - 2.0 * nu) * (1.0 + nu)) * iota[s];
      seta += P->eta[s] * iota[s];
    }
    mu[e] = smu;
    lam[e] = slam;
    eta[e] = seta;
  }
}

/* Eq. e:forcingfunction: b = zeta tanh(p + n) grad(p + n), centred differences */
void or_force(const or_grid* G, const or_params* P, const real_t* p, const real_t* n, real_t* bx,
              real_t* by, real_t* bz) {
  real_t* b[3] = {bx, by, bz};
  int64_t m = nvox(G);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int64_t q[3];
    coords(G, e, q);
    real_t s = p[e] + n[e];
    for (int d = 0; d < 3; ++d) {
      int64_t jp = at(G, q, d, +1, -1, 0), jm = at(G, q, d, -1, -1, 0);
      real_t grad = ((p[jp] + n[jp]) - (p[jm] + n[jm])) / (2.0 * hd(G, d));
      b[d][e] = P->zeta * TANH(s) * grad;
    }
  }
}

/* face value of the coefficient multiplying d_d u_a in component a:
 * lambda + 2 mu when d == a, mu otherwise; arithmetic mean of the two nodes */
static real_t elas_face(int a, int d, const real_t* mu, const real_t* lam, int64_t j0, int64_t j1) {
  real_t mf = 0.5 * (mu[j0] + mu[j1]);
  if (a == d) return 0.5 * (lam[j0] + lam[j1]) + 2.0 * mf;
  return mf;
}

/* Eq. e:variable_elasticity / e:screening:
 *   (L u)_a = sum_d d_d( C^{ad} d_d u_a ) + sum_{d != a} [ d_d(mu d_a u_d) + d_a(lambda d_d u_d) ]
 * with compact face differences for the first sum and centred differences for the mixed
 * terms; out = eta u - L u.  u3/out3 hold the three components one after another. */
void or_elasticity_apply(const or_grid* G, const real_t* mu, const real_t* lam, const real_t* eta,
                         const real_t* u3, real_t* out3) {
  int64_t m = nvox(G);
  const real_t* u[3] = {u3, u3 + m, u3 + 2 * m};
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int64_t c[3];
    coords(G, e, c);
    for (int a = 0; a < 3; ++a) {
      real_t Lu = 0;
      for (int d = 0; d < 3; ++d) {
        int64_t jp = at(G, c, d, +1, -1, 0), jm = at(G, c, d, -1, -1, 0);
        double h = hd(G, d);
        real_t Cp = elas_face(a, d, mu, lam, e, jp);
        real_t Cm = elas_face(a, d, mu, lam, jm, e);
        Lu += (Cp * (u[a][jp] - u[a][e]) - Cm * (u[a][e] - u[a][jm])) / (h * h);
      }
      for (int d = 0; d < 3; ++d) {
        if (d == a) continue;
        double ha = hd(G, a), hdd = hd(G, d);
        /* d_d( mu d_a u_d ): d_a u_d evaluated at c +/- e_d */
        real_t gp = (u[d][at(G, c, d, +1, a, +1)] - u[d][at(G, c, d, +1, a, -1)]) / (2.0 * ha);
        real_t gm = (u[d][at(G, c, d, -1, a, +1)] - u[d][at(G, c, d, -1, a, -1)]) / (2.0 * ha);
        Lu += (mu[at(G, c, d, +1, -1, 0)] * gp - mu[at(G, c, d, -1, -1, 0)] * gm) / (2.0 * hdd);
        /* d_a( lambda d_d u_d ): d_d u_d evaluated at c +/- e_a */
        real_t qp = (u[d][at(G, c, a, +1, d, +1)] - u[d][at(G, c, a, +1, d, -1)]) / (2.0 * hdd);
        real_t qm = (u[d][at(G, c, a, -1, d, +1)] - u[d][at(G, c, a, -1, d, -1)]) / (2.0 * hdd);
        Lu += (lam[at(G, c, a, +1, -1, 0)] * qp - lam[at(G, c, a, -1, -1, 0)] * qm) / (2.0 * ha);
      }
      out3[a * m + e] = eta[e] * u[a][e] - Lu;
    }
  }
}

typedef struct { const or_grid* G; const real_t *mu, *lam, *eta; } el_ctx;

static void el_apply(const void* vctx, const real_t* x, real_t* y) {
  const el_ctx* C = (const el_ctx*)vctx;
  or_elasticity_apply(C->G, C->mu, C->lam, C->eta, x, y);
}

/* ---------------------------------------------------------------- discrete Fourier transform
 * Unnormalised DFT of one line, X[k] = sum_j x[j] exp(sgn 2 pi i j k / n), sgn = -1 forward,
 * +1 inverse.  Lengths that are powers of two use the textbook radix-2 Cooley-Tukey scheme
 * in its iterative form (bit-reversed reordering, then rounds of butterflies on blocks of
 * length 2, 4, ..., n); other lengths evaluate the definition term by term. */
static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* wr[k] + i wi[k] = exp(sgn 2 pi i k / n), k = 0 .. n-1 */
static void dft_roots(int n, int sgn, double* wr, double* wi) {
  for (int k = 0; k < n; ++k) {
    double a = sgn * 2.0 * M_PI * (double)k / (double)n;
    wr[k] = cos(a);
    wi[k] = sin(a);
  }
}

static void dft_line(int n, double* re, double* im, const double* wr, const double* wi,
                     double* tr, double* ti) {
  if (is_pow2(n)) {
    for (int a = 1, b = 0; a < n; ++a) {       /* bit-reversal permutation */
      int bit = n >> 1;
      for (; b & bit; bit >>= 1) b ^= bit;
      b ^= bit;
      if (a < b) {
        double t = re[a]; re[a] = re[b]; re[b] = t;
        t = im[a]; im[a] = im[b]; im[b] = t;
      }
    }
    for (int len = 2; len <= n; len <<= 1) {
      int half = len / 2, step = n / len;
      for (int s0 = 0; s0 < n; s0 += len)
        for (int k = 0; k < half; ++k) {
          double c = wr[k * step], sn = wi[k * step];
          int lo = s0 + k, hi = s0 + k + half;
          double vr = re[hi] * c - im[hi] * sn;
          double vi = re[hi] * sn + im[hi] * c;
          re[hi] = re[lo] - vr;
          im[hi] = im[lo] - vi;
          re[lo] += vr;
          im[lo] += vi;
        }
    }
  } else {
    for (int k = 0; k < n; ++k) {
      double sr = 0.0, si = 0.0;
      for (int j = 0; j < n; ++j) {
        int q = (int)(((int64_t)j * k) % n);
        sr += re[j] * wr[q] - im[j] * wi[q];
        si += re[j] * wi[q] + im[j] * wr[q];
      }
      tr[k] = sr;
      ti[k] = si;
    }
    memcpy(re, tr, (size_t)n * sizeof(double));
    memcpy(im, ti, (size_t)n * sizeof(double));
  }
}

/* 3-D DFT of re + i im over the grid (x fastest), axis by axis; sgn as in dft_line */
void or_dft3(const or_grid* G, double* re, double* im, int sgn) {
  int64_t m = nvox(G);
  for (int d = 0; d < 3; ++d) {
    int n = G->n[d];
    int64_t stride = d == 0 ? 1 : (d == 1 ? G->n[0] : (int64_t)G->n[0] * G->n[1]);
    double* wr = (double*)malloc((size_t)n * sizeof(double));
    double* wi = (double*)malloc((size_t)n * sizeof(double));
    dft_roots(n, sgn, wr, wi);
    int64_t nlines = m / n;
#pragma omp parallel
    {
      double* buf = (double*)malloc((size_t)(4 * n) * sizeof(double));
#pragma omp for schedule(static)
      for (int64_t l = 0; l < nlines; ++l) {
        /* first node of line l: all coordinates but axis d enumerate the lines */
        int64_t base = (l / stride) * stride * n + (l % stride);
        for (int j = 0; j < n; ++j) {
          buf[j] = re[base + j * stride];
          buf[n + j] = im[base + j * stride];
        }
        dft_line(n, buf, buf + n, wr, wi, buf + 2 * n, buf + 3 * n);
        for (int j = 0; j < n; ++j) {
          re[base + j * stride] = buf[j];
          im[base + j * stride] = buf[n + j];
        }
      }
      free(buf);
    }
    free(wr);
    free(wi);
  }
}

/* Section 3 elasticity preconditioner: z = A0^{-1} r, A0 = eta0 I - L_h with constant
 * mu0, lam0, eta0.  On a grid mode exp(i theta . j), theta_d = 2 pi k_d / n_d, the compact
 * second difference gives -S_d, S_d = (2 - 2 cos theta_d) / h_d^2, and the centred first
 * difference gives i T_d, T_d = sin theta_d / h_d.  A0 therefore maps the mode's amplitude
 * vector by the real symmetric matrix
 *   M_aa = eta0 + mu0 (S_0 + S_1 + S_2) + (lam0 + mu0) S_a,
 *   M_ab = (lam0 + mu0) T_a T_b   (a != b),
 * solved here by Cramer's rule for every mode.  A singular M (only the mean mode when
 * eta0 = 0) maps to zero.  r3, z3: three real components, one after another. */
void or_elasticity_spectral(const or_grid* G, double mu0, double lam0, double eta0,
                            const double* r3, double* z3) {
  int64_t m = nvox(G);
  double* re = (double*)malloc((size_t)(3 * m) * sizeof(double));
  double* im = (double*)calloc((size_t)(3 * m), sizeof(double));
  memcpy(re, r3, (size_t)(3 * m) * sizeof(double));
  for (int a = 0; a < 3; ++a) or_dft3(G, re + a * m, im + a * m, -1);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int64_t c[3];
    coords(G, e, c);
    double S[3], T[3];
    for (int d = 0; d < 3; ++d) {
      double th = 2.0 * M_PI * (double)c[d] / (double)G->n[d];
      double h = hd(G, d);
      S[d] = (2.0 - 2.0 * cos(th)) / (h * h);
      T[d] = sin(th) / h;
    }
    double M[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        M[a][b] = (a == b) ? eta0 + mu0 * (S[0] + S[1] + S[2]) + (lam0 + mu0) * S[a]
                           : (lam0 + mu0) * T[a] * T[b];
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
               - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
               + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    double xr[3], xi[3];
    for (int a = 0; a < 3; ++a) {
      /* Cramer: replace column a of M by the right-hand side */
      double Mr[3][3], Mi[3][3];
      for (int q = 0; q < 3; ++q)
        for (int b = 0; b < 3; ++b) {
          Mr[q][b] = (b == a) ? re[q * m + e] : M[q][b];
          Mi[q][b] = (b == a) ? im[q * m + e] : M[q][b];
        }
      double dr = Mr[0][0] * (Mr[1][1] * Mr[2][2] - Mr[1][2] * Mr[2][1])
                - Mr[0][1] * (Mr[1][0] * Mr[2][2] - Mr[1][2] * Mr[2][0])
                + Mr[0][2] * (Mr[1][0] * Mr[2][1] - Mr[1][1] * Mr[2][0]);
      double di = Mi[0][0] * (Mi[1][1] * Mi[2][2] - Mi[1][2] * Mi[2][1])
                - Mi[0][1] * (Mi[1][0] * Mi[2][2] - Mi[1][2] * Mi[2][0])
                + Mi[0][2] * (Mi[1][0] * Mi[2][1] - Mi[1][1] * Mi[2][0]);
      xr[a] = det != 0.0 ? dr / det : 0.0;
      xi[a] = det != 0.0 ? di / det : 0.0;
    }
    for (int a = 0; a < 3; ++a) {
      re[a * m + e] = xr[a];
      im[a * m + e] = xi[a];
    }
  }
  for (int a = 0; a < 3; ++a) or_dft3(G, re + a * m, im + a * m, +1);
  for (int64_t e = 0; e < 3 * m; ++e) z3[e] = re[e] / (double)m;
  free(re);
  free(im);
}

typedef struct { const or_grid* G; double mu0, lam0, eta0; } sp_ctx;

/* the spectral preconditioner on the real and (complex-step) imaginary parts separately:
 * it is a fixed real linear map, independent of the perturbation */
static void spectral_prec(const void* vctx, int64_t m3, const real_t* r, real_t* z) {
  const sp_ctx* C = (const sp_ctx*)vctx;
  double* a = (double*)malloc((size_t)m3 * sizeof(double));
  double* b = (double*)malloc((size_t)m3 * sizeof(double));
  for (int64_t e = 0; e < m3; ++e) a[e] = RE(r[e]);
  or_elasticity_spectral(C->G, C->mu0, C->lam0, C->eta0, a, b);
#ifdef OR_COMPLEX
  double* c = (double*)malloc((size_t)m3 * sizeof(double));
  for (int64_t e = 0; e < m3; ++e) a[e] = cimag(r[e]);
  or_elasticity_spectral(C->G, C->mu0, C->lam0, C->eta0, a, c);
  for (int64_t e = 0; e < m3; ++e) z[e] = b[e] + I * c[e];
  free(c);
#else
  for (int64_t e = 0; e < m3; ++e) z[e] = b[e];
#endif
  free(a);
  free(b);
}

/* Diagonal of A = eta I - L_h for component a at every node: eta plus the two faces of the
 * second difference in each direction (the centred mixed terms do not touch the diagonal). */
static void elas_diag(const or_grid* G, const real_t* mu, const real_t* lam, const real_t* eta,
                      real_t* diag3) {
  int64_t m = nvox(G);
  for (int a = 0; a < 3; ++a) {
    for (int64_t e = 0; e < m; ++e) {
      int64_t c[3];
      coords(G, e, c);
      real_t diag = eta[e];
      for (int d = 0; d < 3; ++d) {
        int64_t jp = at(G, c, d, +1, -1, 0), jm = at(G, c, d, -1, -1, 0);
        double h = hd(G, d);
        diag += (elas_face(a, d, mu, lam, e, jp) + elas_face(a, d, mu, lam, jm, e)) / (h * h);
      }
      diag3[a * m + e] = diag;
    }
  }
}

/* Preconditioner 2 (this library's, not the paper's): the spectral inverse between two
 * diagonal scalings, z = s * A0^{-1} (s * r) with s = (D0 / D)^{1/2} per component and node,
 * D the diagonal of A and D0 that of A0 (D0_a = eta0 + sum_d 2 c_ad / h_d^2 with
 * c_aa = lam0 + 2 mu0 and c_ad = mu0 otherwise).  It is symmetric positive definite, equals
 * A0^{-1} where the coefficients are the means, and equals A^{-1} when A is diagonal
 * (mu = lambda = 0).  Real parts of the coefficients in complex-step mode. */
static void scaled_spectral_scale(const or_grid* G, const real_t* mu, const real_t* lam,
                                  const real_t* eta, double mu0, double lam0, double eta0,
                                  double* s3) {
  int64_t m = nvox(G);
  real_t* diag3 = (real_t*)malloc((size_t)(3 * m) * sizeof(real_t));
  elas_diag(G, mu, lam, eta, diag3);
  for (int a = 0; a < 3; ++a) {
    double d0 = eta0;
    for (int d = 0; d < 3; ++d) {
      double h = hd(G, d);
      d0 += 2.0 * (d == a ? lam0 + 2.0 * mu0 : mu0) / (h * h);
    }
    for (int64_t e = 0; e < m; ++e) s3[a * m + e] = sqrt(d0 / RE(diag3[a * m + e]));
  }
  free(diag3);
}

static void domain_means(int64_t m, const real_t* mu, const real_t* lam, const real_t* eta,
                         double* mu0, double* lam0, double* eta0) {
  *mu0 = *lam0 = *eta0 = 0.0;
  for (int64_t e = 0; e < m; ++e) {
    *mu0 += RE(mu[e]);
    *lam0 += RE(lam[e]);
    *eta0 += RE(eta[e]);
  }
  *mu0 /= (double)m;
  *lam0 /= (double)m;
  *eta0 /= (double)m;
}

#ifndef OR_COMPLEX
/* z = s * A0^{-1} (s * r) for the given coefficients (the map preconditioner 2 applies) */
void or_elasticity_scaled_spectral(const or_grid* G, const double* mu, const double* lam,
                                   const double* eta, const double* r3, double* z3) {
  int64_t m = nvox(G);
  double mu0, lam0, eta0;
  domain_means(m, mu, lam, eta, &mu0, &lam0, &eta0);
  double* s3 = (double*)malloc((size_t)(3 * m) * sizeof(double));
  double* a = (double*)malloc((size_t)(3 * m) * sizeof(double));
  scaled_spectral_scale(G, mu, lam, eta, mu0, lam0, eta0, s3);
  for (int64_t e = 0; e < 3 * m; ++e) a[e] = s3[e] * r3[e];
  or_elasticity_spectral(G, mu0, lam0, eta0, a, z3);
  for (int64_t e = 0; e < 3 * m; ++e) z3[e] = s3[e] * z3[e];
  free(s3);
  free(a);
}
#endif

typedef struct { sp_ctx sp; const double* s3; } ssp_ctx;

static void scaled_spectral_prec(const void* vctx, int64_t m3, const real_t* r, real_t* z) {
  const ssp_ctx* C = (const ssp_ctx*)vctx;
  real_t* t = (real_t*)malloc((size_t)m3 * sizeof(real_t));
  for (int64_t e = 0; e < m3; ++e) t[e] = C->s3[e] * r[e];
  spectral_prec(&C->sp, m3, t, z);
  for (int64_t e = 0; e < m3; ++e) z[e] = C->s3[e] * z[e];
  free(t);
}

/* (eta I - L_h) u = rhs by PCG from the given u (Section 3, elasticity sub-step);
 * precond 0: Jacobi, 1: the constant-coefficient spectral inverse with the domain means of
 * mu, lambda, eta (real parts in complex-step mode), 2: that inverse between the diagonal
 * scalings above */
int or_elasticity_solve(const or_grid* G, const real_t* mu, const real_t* lam, const real_t* eta,
                        const real_t* rhs3, real_t* u3, double rtol, int32_t maxit,
                        int32_t precond, int32_t* iters, double* relres) {
  int64_t m = nvox(G);
  el_ctx C = {G, mu, lam, eta};
  if (precond == 1 || precond == 2) {
    sp_ctx S = {G, 0.0, 0.0, 0.0};
    domain_means(m, mu, lam, eta, &S.mu0, &S.lam0, &S.eta0);
    if (precond == 1)
      return pcg(3 * m, el_apply, &C, spectral_prec, &S, rhs3, u3, rtol, maxit, iters, relres);
    double* s3 = (double*)malloc((size_t)(3 * m) * sizeof(double));
    scaled_spectral_scale(G, mu, lam, eta, S.mu0, S.lam0, S.eta0, s3);
    ssp_ctx SS = {S, s3};
    int st = pcg(3 * m, el_apply, &C, scaled_spectral_prec, &SS, rhs3, u3, rtol, maxit, iters,
                 relres);
    free(s3);
    return st;
  }
  if (precond != 0) return OR_ERR_ARG;
  real_t* dinv = (real_t*)malloc((size_t)(3 * m) * sizeof(real_t));
  elas_diag(G, mu, lam, eta, dinv);
  for (int64_t e = 0; e < 3 * m; ++e) dinv[e] = 1.0 / dinv[e];
  int st = pcg(3 * m, el_apply, &C, jacobi_prec, dinv, rhs3, u3, rtol, maxit, iters, relres);
  free(dinv);
  return st;
}

/* ---------------------------------------------------------------- semi-Lagrangian
 * Section 3: X* = x - dt u_t(x), X = x - dt/2 (u_t(x) + u_t(X*)), cubic interpolation. */

/* cubic Lagrange weights for nodes -1, 0, 1, 2 at fractional position t */
static void lagrange4(real_t t, real_t wgt[4]) {
  wgt[0] = -t * (t - 1.0) * (t - 2.0) / 6.0;
  wgt[1] = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
  wgt[2] = -(t + 1.0) * t * (t - 2.0) / 2.0;
  wgt[3] = (t + 1.0) * t * (t - 1.0) / 6.0;
}

/* tricubic interpolation of a periodic field at index-space point (X, Y, Z) */
real_t or_interp(const or_grid* G, const real_t* q, real_t X, real_t Y, real_t Z) {
  real_t pos[3] = {X, Y, Z};
  int64_t base[3];
  real_t wgt[3][4];
  for (int d = 0; d < 3; ++d) {
    double fl = floor(RE(pos[d]));
    base[d] = (int64_t)fl;
    lagrange4(pos[d] - fl, wgt[d]);
  }
  real_t s = 0;
  for (int cz = 0; cz < 4; ++cz)
    for (int cy = 0; cy < 4; ++cy)
      for (int cx = 0; cx < 4; ++cx) {
        int64_t iz = wrapi(base[2] - 1 + cz, G->n[2]);
        int64_t iy = wrapi(base[1] - 1 + cy, G->n[1]);
        int64_t ix = wrapi(base[0] - 1 + cx, G->n[0]);
        s += wgt[2][cz] * wgt[1][cy] * wgt[0][cx] * q[(iz * G->n[1] + iy) * G->n[0] + ix];
      }
  return s;
}

/* centred-difference divergence of v */
void or_divergence(const or_grid* G, const real_t* vx, const real_t* vy, const real_t* vz,
                   real_t* div) {
  const real_t* v[3] = {vx, vy, vz};
  int64_t m = nvox(G);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int64_t c[3];
    coords(G, e, c);
    real_t s = 0;
    for (int d = 0; d < 3; ++d)
      s += (v[d][at(G, c, d, +1, -1, 0)] - v[d][at(G, c, d, -1, -1, 0)]) / (2.0 * hd(G, d));
    div[e] = s;
  }
}

/* Advect q_in[0..4] = (p, i, n, g, w) in conservative form d_t q + div(q v) = 0, i.e. along
 * characteristics dq/dt = -q div v, with the RK2 source update of Section 3:
 *   q* = q(X) + dt g(q(X), X),  q_new = q(X) + dt/2 (g(q(X), X) + g(q*, x)),  g(q, x) = -q div v(x);
 * and q_in[5] = f without source (Eq. for f: d_t f + grad f . v = 0). */
void or_sl_advect(const or_grid* G, double dt, const real_t* vx, const real_t* vy, const real_t* vz,
                  real_t* const* q_in, real_t* const* q_out) {
  int64_t m = nvox(G);
  const real_t* v[3] = {vx, vy, vz};
  real_t* div = (real_t*)malloc((size_t)m * sizeof(real_t));
  or_divergence(G, vx, vy, vz, div);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int64_t c[3];
    coords(G, e, c);
    real_t Xs[3], X[3];
    for (int d = 0; d < 3; ++d) Xs[d] = (double)c[d] - dt * v[d][e] / hd(G, d);
    for (int d = 0; d < 3; ++d) {
      real_t v_star = or_interp(G, v[d], Xs[0], Xs[1], Xs[2]);
      X[d] = (double)c[d] - 0.5 * dt * (v[d][e] + v_star) / hd(G, d);
    }
    real_t divX = or_interp(G, div, X[0], X[1], X[2]);
    for (int s = 0; s < 5; ++s) {
      real_t qX = or_interp(G, q_in[s], X[0], X[1], X[2]);
      real_t gX = -qX * divX;
      real_t q_star = qX + dt * gX;
      real_t g_star = -q_star * div[e];
      q_out[s][e] = qX + 0.5 * dt * (gX + g_star);
    }
    q_out[5][e] = or_interp(G, q_in[5], X[0], X[1], X[2]);
  }
  free(div);
}

/* ---------------------------------------------------------------- reactions */

/* smoothed Heaviside (1 + tanh(x / eps_H)) / 2, evaluated in the equal logistic form
 * 1 / (1 + exp(-2 x / eps_H)), which keeps full relative accuracy for x << 0 */
real_t or_heaviside(const or_params* P, real_t x) { return 1.0 / (1.0 + EXP(-2.0 * x / P->eps_H)); }
static real_t heaviside(const or_params* P, real_t x) { return or_heaviside(P, x); }

/* oxygen factor of Eq. e:gog_reac_op / e:gog_reac_inv_op, o_mit = (o_hyp + o_inv) / 2 */
static real_t mitosis_factor(const or_params* P, real_t o) {
  real_t o_mit = 0.5 * (P->o_hyp + P->o_inv);
  if (RE(o) > RE(P->o_inv)) return 1.0;
  if (RE(o) >= RE(o_mit)) return (o - o_mit) / (P->o_inv - o_mit);
  return 0.0;
}

/* source terms of Eq. e:p, e:i, e:n, e:gm_wm, e:w (diffusion and transport excluded) */
static void species_rates(const or_params* P, real_t rho, real_t o, const real_t y[5], real_t dy[5]) {
  real_t p = y[0], i = y[1], g = y[3], w = y[4];
  real_t h = P->gamma * heaviside(P, P->o_hyp - o);                   /* Eq. e:death */
  real_t alpha = P->alpha0 * heaviside(P, P->o_inv - o);              /* Eq. e:alpha */
  real_t beta = P->beta0 * heaviside(P, P->sigma_b - p - i) * o;      /* Eq. e:beta  */
  real_t mf = mitosis_factor(P, o);
  real_t R = rho * p * (1.0 - p) * mf;                                /* Eq. e:gog_reac_op     */
  real_t Rt = P->rho_i_frac * rho * i * (1.0 - i) * mf;               /* Eq. e:gog_reac_inv_op */
  real_t gw = g + w;
  real_t fg = RE(gw) > 0.0 ? g / gw : 0.0;
  real_t fw = RE(gw) > 0.0 ? w / gw : 0.0;
  dy[0] = R - alpha * p + beta * i - h * p;
  dy[1] = Rt + alpha * p - beta * i - h * i;
  dy[2] = h * (p + i + g + w);
  dy[3] = -fg * (R + Rt) - h * g;
  dy[4] = -fw * (R + Rt) - h * w;
}

/* Section 3 reaction sub-steps, one Heun step each:
 *  (p, i, n, g, w) with o = o_dagger and the frozen rho;  then oxygen (Eq. e:ox) from
 *  o_dagger with the new p, g, w;  then edema (Eq. e:edema, reaction part) with the new i. */
void or_react(const or_grid* G, const or_params* P, double dt, const real_t* rho, real_t* p,
              real_t* i, real_t* n, real_t* g, real_t* w, real_t* o, real_t* l) {
  int64_t m = nvox(G);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    real_t y[5] = {p[e], i[e], n[e], g[e], w[e]};
    real_t k1[5], k2[5], ys[5];
    species_rates(P, rho[e], o[e], y, k1);
    for (int s = 0; s < 5; ++s) ys[s] = y[s] + dt * k1[s];
    species_rates(P, rho[e], o[e], ys, k2);
    for (int s = 0; s < 5; ++s) y[s] = y[s] + 0.5 * dt * (k1[s] + k2[s]);
    p[e] = y[0]; i[e] = y[1]; n[e] = y[2]; g[e] = y[3]; w[e] = y[4];

    /* oxygen: d_t o = -delta_p p + delta_s (o_heal - o)(g + w) */
    real_t o0 = o[e];
    real_t ko1 = -P->delta_p * p[e] + P->delta_s * (P->o_heal - o0) * (g[e] + w[e]);
    real_t os = o0 + dt * ko1;
    real_t ko2 = -P->delta_p * p[e] + P->delta_s * (P->o_heal - os) * (g[e] + w[e]);
    o[e] = o0 + 0.5 * dt * (ko1 + ko2);

    /* edema: d_t l = delta_e i / (i + delta_half) (1 - i) - delta_l l */
    real_t l0 = l[e];
    real_t src = P->delta_e * i[e] / (i[e] + P->delta_half) * (1.0 - i[e]);
    real_t kl1 = src - P->delta_l * l0;
    real_t ls = l0 + dt * kl1;
    real_t kl2 = src - P->delta_l * ls;
    l[e] = l0 + 0.5 * dt * (kl1 + kl2);
  }
}

/* Single-species model (Eq. e:rd): one Heun step of the reaction part,
 *   d_t c = R,  d_t g = -g/(g+w) R,  d_t w = -w/(g+w) R,  R = rho c (1 - c)  (Eq. e:reac_op),
 * rho frozen at the step's start (reading 10); the ratio is 0 where g + w <= 0. */
static void single_rates(real_t rho, const real_t y[3], real_t dy[3]) {
  real_t R = rho * y[0] * (1.0 - y[0]);
  real_t gw = y[1] + y[2];
  real_t fg = RE(gw) > 0.0 ? y[1] / gw : 0.0;
  real_t fw = RE(gw) > 0.0 ? y[2] / gw : 0.0;
  dy[0] = R;
  dy[1] = -fg * R;
  dy[2] = -fw * R;
}

void or_react_single(const or_grid* G, double dt, const real_t* rho, real_t* c, real_t* g,
                     real_t* w) {
  int64_t m = nvox(G);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    real_t y[3] = {c[e], g[e], w[e]};
    real_t k1[3], k2[3], ys[3];
    single_rates(rho[e], y, k1);
    for (int s = 0; s < 3; ++s) ys[s] = y[s] + dt * k1[s];
    single_rates(rho[e], ys, k2);
    for (int s = 0; s < 3; ++s) y[s] = y[s] + 0.5 * dt * (k1[s] + k2[s]);
    c[e] = y[0]; g[e] = y[1]; w[e] = y[2];
  }
}

/* ---------------------------------------------------------------- diagnostics */

void or_diagnostics(const or_grid* G, const real_t* mu, const real_t* lam, const real_t* u3,
                    real_t* trace, real_t* tau, real_t* jac) {
  int64_t m = nvox(G);
  const real_t* u[3] = {u3, u3 + m, u3 + 2 * m};
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int64_t c[3];
    coords(G, e, c);
    real_t D[3][3];                       /* D[a][d] = d u_a / d x_d, centred */
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d)
        D[a][d] = (u[a][at(G, c, d, +1, -1, 0)] - u[a][at(G, c, d, -1, -1, 0)]) / (2.0 * hd(G, d));
    real_t E[3][3], T[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) E[a][b] = 0.5 * (D[a][b] + D[b][a]);
    real_t trE = E[0][0] + E[1][1] + E[2][2];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) T[a][b] = (a == b ? lam[e] * trE : 0.0) + 2.0 * mu[e] * E[a][b];
    trace[e] = T[0][0] + T[1][1] + T[2][2];
    real_t hx = 0.5 * (T[0][0] - T[1][1]);
    tau[e] = SQRT_RE(hx * hx + T[0][1] * T[0][1]);
    real_t F[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) F[a][b] = (a == b ? 1.0 : 0.0) + D[a][b];
    jac[e] = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1])
           - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0])
           + F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
  }
}

double or_displacement_extent(const or_grid* G, const real_t* u3, const double seed[3],
                              double thr) {
  int64_t m = nvox(G);
  double best = 0.0;
  for (int64_t e = 0; e < m; ++e) {
    double uu = 0.0;
    for (int a = 0; a < 3; ++a) uu += RE(u3[a * m + e]) * RE(u3[a * m + e]);
    if (sqrt(uu) < thr) continue;
    int64_t c[3];
    coords(G, e, c);
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      double x = c[d] * hd(G, d) - seed[d];
      x -= G->L[d] * floor(x / G->L[d] + 0.5);   /* nearest periodic image */
      r2 += x * x;
    }
    if (sqrt(r2) > best) best = sqrt(r2);
  }
  return best;
}

/* ---------------------------------------------------------------- step */

static real_t* alloc_field(int64_t m) { return (real_t*)calloc((size_t)m, sizeof(real_t)); }

static int valid_grid(const or_grid* G) {
  for (int d = 0; d < 3; ++d)
    if (G->n[d] < 4 || !(G->L[d] > 0.0)) return 0;
  return 1;
}

/* Elasticity sub-step: Lame, eta and force from the current state, solve
 * (eta I - L_h) u = -b from the current u. */
static int elasticity_substep(const or_grid* G, const or_params* P, or_state* S, int32_t* iters,
                              double* relres) {
  int64_t m = nvox(G);
  real_t* mu = alloc_field(m);
  real_t* lam = alloc_field(m);
  real_t* eta = alloc_field(m);
  real_t* rhs = alloc_field(3 * m);
  real_t* u3 = alloc_field(3 * m);
  or_lame(G, P, S->p, S->i, S->n, S->g, S->w, S->f, S->bg, mu, lam, eta);
  or_force(G, P, S->p, S->n, rhs, rhs + m, rhs + 2 * m);
  for (int64_t e = 0; e < 3 * m; ++e) rhs[e] = -rhs[e];
  for (int a = 0; a < 3; ++a) memcpy(u3 + a * m, S->u[a], (size_t)m * sizeof(real_t));
  int st = or_elasticity_solve(G, mu, lam, eta, rhs, u3, P->rtol_elas, P->maxit_elas,
                               P->precond_elas, iters, relres);
  for (int a = 0; a < 3; ++a) memcpy(S->u[a], u3 + a * m, (size_t)m * sizeof(real_t));
  free(mu); free(lam); free(eta); free(rhs); free(u3);
  return st;
}

/* Initial displacement u^0 from the initial state (from u = 0), v^0 = 0. */
int or_init(const or_grid* G, const or_params* P, or_state* S, or_stats* stats) {
  if (!valid_grid(G)) return OR_ERR_ARG;
  int64_t m = nvox(G);
  for (int a = 0; a < 3; ++a) {
    memset(S->u[a], 0, (size_t)m * sizeof(real_t));
    memset(S->v[a], 0, (size_t)m * sizeof(real_t));
  }
  S->vprev_valid = 0;
  int32_t it = 0;
  double rr = 0.0;
  int st = elasticity_substep(G, P, S, &it, &rr);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->it_elas = it;
    stats->relres_elas = rr;
  }
  return st;
}

/* One step of the multispecies splitting (Section 3), or of the single-species one for
 * P->model == 1 (Section 3's list for Eq. e:rd: c in p; S2 diffuses c alone and S3 is the
 * logistic reaction of c with its loss from g and w; i and n, zero for that model, are only
 * advected; o and l are left alone):
 *  S0  K (faces) and rho from the state at the step's start;
 *  S1  semi-Lagrangian advection of p, i, n, g, w (conservative) and f with v^n;
 *  S2  Crank-Nicolson diffusion of i, o and edema l; the increment of i leaves g and w;
 *  S3  reaction of p, i, n, g, w;  S4 oxygen reaction;  S5 edema reaction;
 *  S6  elasticity solve for u^{n+1}, started from the extrapolation of u in time: quadratic,
 *      u^n + dt v^n + dt (v^n - v^{n-1}), when the previous step's velocity is kept
 *      (S->vprev), else linear, u^n + dt v^n;
 *  S7  v^{n+1} = (u^{n+1} - u^n) / dt. */
int or_step(const or_grid* G, const or_params* P, double dt, or_state* S, or_stats* stats) {
  if (!valid_grid(G) || !(dt > 0.0)) return OR_ERR_ARG;
  int64_t m = nvox(G);
  int st = OR_OK;
  or_stats local;
  memset(&local, 0, sizeof(local));

  /* S0 */
  real_t* K = alloc_field(m);
  real_t* Kf[3] = {alloc_field(m), alloc_field(m), alloc_field(m)};
  real_t* rho = alloc_field(m);
  or_diffusion_node_K(G, P, S->g, S->w, S->f, K);
  or_diffusion_faces(G, K, Kf[0], Kf[1], Kf[2]);
  for (int64_t e = 0; e < m; ++e) rho[e] = P->rho_g * S->g[e] + P->rho_w * S->w[e];

  /* S1 */
  real_t* qout[6];
  for (int s = 0; s < 6; ++s) qout[s] = alloc_field(m);
  real_t* qin[6] = {S->p, S->i, S->n, S->g, S->w, S->f};
  or_sl_advect(G, dt, S->v[0], S->v[1], S->v[2], qin, qout);
  for (int s = 0; s < 6; ++s) memcpy(qin[s], qout[s], (size_t)m * sizeof(real_t));

  /* S2: the diffusing fields are i, o, l (multispecies) or c, kept in p (single species,
   * Section 3's list for Eq. e:rd); the increment of the first leaves g and w */
  const int single = P->model == 1;
  real_t* dif = single ? S->p : S->i;
  real_t* i_old = qout[0];            /* reuse as scratch: the field after advection */
  memcpy(i_old, dif, (size_t)m * sizeof(real_t));
  real_t* fields[3] = {dif, S->o, S->l};
  for (int c = 0; c < (single ? 1 : 3) && st == OR_OK; ++c)
    st = or_cn_solve(G, Kf[0], Kf[1], Kf[2], dt, fields[c], fields[c], P->rtol_diff,
                     P->maxit_diff, &local.it_diff[c], &local.relres_diff[c]);
  if (st == OR_OK) {
    for (int64_t e = 0; e < m; ++e) {
      real_t di = dif[e] - i_old[e];
      real_t g = S->g[e], w = S->w[e], gw = g + w;
      real_t fg = RE(gw) > 0.0 ? g / gw : 0.0;
      real_t fw = RE(gw) > 0.0 ? w / gw : 0.0;
      S->g[e] = g - di * fg;
      S->w[e] = w - di * fw;
    }
    /* S3 - S5 (single species: the logistic reaction of c with the g, w losses) */
    if (single)
      or_react_single(G, dt, rho, S->p, S->g, S->w);
    else
      or_react(G, P, dt, rho, S->p, S->i, S->n, S->g, S->w, S->o, S->l);
    /* S6 - S7 */
    real_t* u_old[3] = {qout[1], qout[2], qout[3]};
    for (int a = 0; a < 3; ++a) memcpy(u_old[a], S->u[a], (size_t)m * sizeof(real_t));
    /* the solve starts from the extrapolation of u through u^n, u^{n-1} (and u^{n-2}):
     * d = dt v^n is the linear increment (u^n + d = 2 u^n - u^{n-1}); with the previous
     * step's velocity, q = dt (v^n - v^{n-1}) makes it quadratic
     * (u^n + d + q = 3 u^n - 3 u^{n-1} + u^{n-2}) */
    const int quad = S->vprev[0] != NULL && S->vprev_valid;
    for (int a = 0; a < 3; ++a)
      for (int64_t e = 0; e < m; ++e) {
        real_t s = dt * S->v[a][e];
        if (quad) s = s + dt * (S->v[a][e] - S->vprev[a][e]);
        S->u[a][e] = S->u[a][e] + s;
      }
    st = elasticity_substep(G, P, S, &local.it_elas, &local.relres_elas);
    for (int a = 0; a < 3; ++a) {
      if (S->vprev[0] != NULL) memcpy(S->vprev[a], S->v[a], (size_t)m * sizeof(real_t));
      for (int64_t e = 0; e < m; ++e) S->v[a][e] = (S->u[a][e] - u_old[a][e]) / dt;
    }
    if (S->vprev[0] != NULL) S->vprev_valid = 1;
  }
  if (stats) *stats = local;
  free(K); free(Kf[0]); free(Kf[1]); free(Kf[2]); free(rho);
  for (int s = 0; s < 6; ++s) free(qout[s]);
  return st;
}
