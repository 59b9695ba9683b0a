// tg_adjoint.cu -- discrete adjoint of one operator-split step (FP64), for gradients of a
// misfit with respect to theta = (k_scale, rho, o_hyp, o_inv, E_scale).
//
// The paper names adjoint-based parameter estimation as its next goal (Section 5); this file
// differentiates the discretised step S0-S7 exactly, treating each linear solve as its exact
// inverse.  Given lambda^{n+1} (the sensitivity of the misfit to the state after the step) the
// kernels below produce lambda^n and add the step's contribution to dJ/dtheta.  Reverse order:
//   S7^T  v = (u+ - u^n)/dt
//   S6^T  adjoint elasticity solve M psi = lambda_u, then the sensitivities of M (through mu,
//         lambda, eta of Eq. e:lame) and of the force b (Eq. e:forcingfunction)
//   S5^T, S4^T, S3^T  reverse Heun steps of the edema, oxygen and species reactions
//   S2^T  fix-up of g, w; adjoint Crank-Nicolson solves A phi = lambda_out, lambda_in = B phi,
//         and the sensitivity of the diffusion faces (harmonic means of K)
//   S1^T  transpose of the semi-Lagrangian interpolation (scatter with FP64 atomics), the
//         dependence of the departure points on v, and the transpose of div_h
//   S0^T  rho and K of the step's start back to g, w, f.
#include "tg_internal.cuh"

namespace tg {
namespace {

constexpr int GK = 0, GRHO = 1, GOHYP = 2, GOINV = 3, GE = 4;   // theta slots

// add a block's partial sums of theta components to grad[] (last block, one atomic per slot)
template <int NV>
__device__ void add_theta(double (&v)[NV], const int (&slot)[NV], const AdjView& A) {
  double out[NV];
  if (reduce_last_block<NV>(v, A.partial, A.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) A.grad[slot[q]] += out[q];
  }
}

// ------------------------------------------------------------------------------ S7^T, setup
// rhs = lambda_u + lambda_v / dt (for S6^T), lambda_u^n = -lambda_v / dt; copy the incoming
// lambdas of the reacted species and of f+ to scratch.
__global__ void __launch_bounds__(NT) k_adj_prep(long long n, AdjView A, double inv_dt) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double lv = A.lam.v[a][c];
      A.rhs[a][c] = A.lam.u[a][c] + lv * inv_dt;
      A.lam.u[a][c] = -lv * inv_dt;
    }
    A.LQ[0][c] = A.lam.p[c];
    A.LQ[1][c] = A.lam.i[c];
    A.LQ[2][c] = A.lam.n[c];
    A.LQ[3][c] = A.lam.g[c];
    A.LQ[4][c] = A.lam.w[c];
    A.LQ[5][c] = A.lam.o[c];
    A.LQ[6][c] = A.lam.l[c];
    A.LF[c] = A.lam.f[c];
  }
}

// ------------------------------------------------------------------------------ S6^T
// With psi solving M psi = lambda_u and u = u+:  dJ = -psi^T dM u, M = eta I - L_h(mu, lambda).
// Summation by parts of psi^T L_h u gives, at node j,
//   dJ/dmu_j     = -sum_a sum_d w_ad (G_ad(j+1/2) + G_ad(j-1/2)) - sum_{a!=d} (D_d psi_a)(D_a u_d)
//   dJ/dlambda_j = -sum_a 1/2 (G_aa(j+1/2) + G_aa(j-1/2))    - sum_{a!=d} (D_a psi_a)(D_d u_d)
//   dJ/deta_j    = -sum_a psi_a u_a
// where G_ad is the face product of compact differences of psi_a and u_a along d over h_d^2
// and w_ad = 1 (d == a), 1/2 (d != a).  The force b = zeta tanh(s) D s, s = p + n, gets
// lambda_b = -psi.  When `species` is set the results flow to the species lambdas.
__global__ void __launch_bounds__(NT) k_adj_elas_coef(Geo G, DevParams P, AdjView A,
                                                      const double* __restrict__ mu,
                                                      const double* __restrict__ lam,
                                                      const double* __restrict__ p,
                                                      const double* __restrict__ nn,
                                                      double inv_Escale, int species) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  double acc[1] = {0.0};
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      const long long np[3] = {nb.at(1, 0, 0), nb.at(0, 1, 0), nb.at(0, 0, 1)};
      const long long nm[3] = {nb.at(-1, 0, 0), nb.at(0, -1, 0), nb.at(0, 0, -1)};
      double lmu = 0.0, lla = 0.0, leta = 0.0;
      double Dpsi[3][3], Du[3][3];   // [component][direction], centred differences
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double* ps = A.psi[a];
        const double* uu = A.up[a];
        const double pc = ps[c], uc = uu[c];
        leta -= pc * uc;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const double pp = ps[np[d]], pm = ps[nm[d]], up = uu[np[d]], um = uu[nm[d]];
          const double Gsum = ((pp - pc) * (up - uc) + (pc - pm) * (uc - um)) * G.ih2[d];
          lmu -= (d == a ? 1.0 : 0.5) * Gsum;
          if (d == a) lla -= 0.5 * Gsum;
          Dpsi[a][d] = (pp - pm) * G.inv2h[d];
          Du[a][d] = (up - um) * G.inv2h[d];
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d)
          if (d != a) {
            lmu -= Dpsi[a][d] * Du[d][a];
            lla -= Dpsi[a][a] * Du[d][d];
          }
      acc[0] += (lmu * mu[c] + lla * lam[c]) * inv_Escale;
      if (species) {
        double li[5];
#pragma unroll
        for (int s = 0; s < 5; ++s) li[s] = P.cmu[s] * lmu + P.clam[s] * lla + P.eta[s] * leta;
        // force: lambda_b = -psi;  s = p + n
        const double sc = p[c] + nn[c];
        const double th = tanh(sc);
        double ls = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const double Ds = ((p[np[d]] + nn[np[d]]) - (p[nm[d]] + nn[nm[d]])) * G.inv2h[d];
          ls += P.zeta * (1.0 - th * th) * (-A.psi[d][c]) * Ds;
          // - D_d( zeta tanh(s) lambda_b_d )
          const double fp = P.zeta * tanh(p[np[d]] + nn[np[d]]) * (-A.psi[d][np[d]]);
          const double fm = P.zeta * tanh(p[nm[d]] + nn[nm[d]]) * (-A.psi[d][nm[d]]);
          ls -= (fp - fm) * G.inv2h[d];
        }
        A.LQ[0][c] += li[0] + ls;
        A.LQ[1][c] += li[0];
        A.LQ[2][c] += li[0] + ls;
        A.LQ[3][c] += li[1];
        A.LQ[4][c] += li[2];
        A.LF[c] += li[3];
      }
    }
  }
  const int slot[1] = {GE};
  add_theta<1>(acc, slot, A);
}

// ------------------------------------------------------------------------------ S5^T S4^T S3^T
__device__ __forceinline__ double heav(const DevParams& P, double x) {
  return 1.0 / (1.0 + exp(-2.0 * x * P.inv_eps_H));
}
// dH/dx of the logistic form: (2 / eps_H) H (1 - H)
__device__ __forceinline__ double dheav(const DevParams& P, double x) {
  const double h = heav(P, x);
  return 2.0 * P.inv_eps_H * h * (1.0 - h);
}

struct Ox {          // oxygen-dependent factors and their derivatives
  double h, alpha, mf;
  double h_o, alpha_o, mf_o;            // d/do
  double h_hyp, mf_hyp;                  // d/do_hyp
  double alpha_inv, mf_inv;              // d/do_inv
};

__device__ __forceinline__ Ox oxygen_factors(const DevParams& P, double o) {
  Ox X;
  X.h = P.gamma * heav(P, P.o_hyp - o);
  X.alpha = P.alpha0 * heav(P, P.o_inv - o);
  const double Hh = dheav(P, P.o_hyp - o), Hi = dheav(P, P.o_inv - o);
  X.h_o = -P.gamma * Hh;
  X.h_hyp = P.gamma * Hh;
  X.alpha_o = -P.alpha0 * Hi;
  X.alpha_inv = P.alpha0 * Hi;
  const double D = P.o_inv - P.o_mit;
  if (o > P.o_inv) {
    X.mf = 1.0;
    X.mf_o = X.mf_hyp = X.mf_inv = 0.0;
  } else if (o >= P.o_mit) {
    X.mf = (o - P.o_mit) / D;
    X.mf_o = 1.0 / D;
    X.mf_hyp = 0.5 * (o - P.o_inv) / (D * D);
    X.mf_inv = -0.5 * (o - P.o_hyp) / (D * D);
  } else {
    X.mf = 0.0;
    X.mf_o = X.mf_hyp = X.mf_inv = 0.0;
  }
  return X;
}

// Adjoint of the species source F(y; o, rho) at y: adds J^T a to ly and the parameter and
// oxygen sensitivities to lo, lrho, lhyp, linv.
__device__ __forceinline__ void species_rates_adj(const DevParams& P, double rho, double o,
                                                  const Ox& X, const double y[5],
                                                  const double a[5], double ly[5], double& lo,
                                                  double& lrho, double& lhyp, double& linv) {
  const double p = y[0], i = y[1], g = y[3], w = y[4];
  const double Hb = heav(P, P.sigma_b - p - i);
  const double beta = P.beta0 * Hb * o;
  const double beta_pi = -P.beta0 * dheav(P, P.sigma_b - p - i) * o;   // d beta / dp = d / di
  const double beta_o = P.beta0 * Hb;
  const double rhoi = P.rho_i_frac * rho;
  const double lp = p * (1.0 - p), li = i * (1.0 - i);
  const double R = rho * lp * X.mf, Rt = rhoi * li * X.mf, T = R + Rt;
  const double Rp = rho * (1.0 - 2.0 * p) * X.mf, Rti = rhoi * (1.0 - 2.0 * i) * X.mf;
  const double gw = g + w;
  const bool pos = gw > 0.0;
  const double fg = pos ? g / gw : 0.0, fw = pos ? w / gw : 0.0;
  const double ig2 = pos ? 1.0 / (gw * gw) : 0.0;
  const double h = X.h, al = X.alpha;
  const double ap = a[0], ai = a[1], an = a[2], ag = a[3], aw = a[4];
  const double agw = -(ag * fg + aw * fw);        // multiplies dT
  // d/dp
  ly[0] += ap * (Rp - al + beta_pi * i - h) + ai * (al - beta_pi * i) + an * h + agw * Rp;
  // d/di
  ly[1] += ap * (beta_pi * i + beta) + ai * (Rti - beta_pi * i - beta - h) + an * h + agw * Rti;
  // d/dg, d/dw (fractions g/(g+w), w/(g+w))
  ly[3] += an * h + ag * (-w * ig2 * T - h) + aw * (w * ig2 * T);
  ly[4] += an * h + ag * (g * ig2 * T) + aw * (-g * ig2 * T - h);
  // d/do
  {
    const double Ro = rho * lp * X.mf_o, Rto = rhoi * li * X.mf_o;
    lo += ap * (Ro - X.alpha_o * p + beta_o * i - X.h_o * p) +
          ai * (Rto + X.alpha_o * p - beta_o * i - X.h_o * i) + an * X.h_o * (p + i + g + w) +
          ag * (-fg * (Ro + Rto) - X.h_o * g) + aw * (-fw * (Ro + Rto) - X.h_o * w);
  }
  // d/drho (field)
  {
    const double Rr = lp * X.mf, Rtr = P.rho_i_frac * li * X.mf;
    lrho += ap * Rr + ai * Rtr + agw * (Rr + Rtr);
  }
  // d/do_hyp
  {
    const double Rh = rho * lp * X.mf_hyp, Rth = rhoi * li * X.mf_hyp;
    lhyp += ap * (Rh - X.h_hyp * p) + ai * (Rth - X.h_hyp * i) + an * X.h_hyp * (p + i + g + w) +
            ag * (-fg * (Rh + Rth) - X.h_hyp * g) + aw * (-fw * (Rh + Rth) - X.h_hyp * w);
  }
  // d/do_inv
  {
    const double Rv = rho * lp * X.mf_inv, Rtv = rhoi * li * X.mf_inv;
    linv += ap * (Rv - X.alpha_inv * p) + ai * (Rtv + X.alpha_inv * p) + agw * (Rv + Rtv);
  }
}

// forward source (same formulas as the reaction kernel) for the recomputation
__device__ __forceinline__ void species_rates_f(const DevParams& P, double rho, double o,
                                                const Ox& X, const double y[5], double dy[5]) {
  const double p = y[0], i = y[1], g = y[3], w = y[4];
  const double beta = P.beta0 * heav(P, P.sigma_b - p - i) * o;
  const double R = rho * p * (1.0 - p) * X.mf;
  const double Rt = P.rho_i_frac * rho * i * (1.0 - i) * X.mf;
  const double gw = g + w;
  const double fg = gw > 0.0 ? g / gw : 0.0, fw = gw > 0.0 ? w / gw : 0.0;
  dy[0] = R - X.alpha * p + beta * i - X.h * p;
  dy[1] = Rt + X.alpha * p - beta * i - X.h * i;
  dy[2] = X.h * (p + i + g + w);
  dy[3] = -fg * (R + Rt) - X.h * g;
  dy[4] = -fw * (R + Rt) - X.h * w;
}

__global__ void __launch_bounds__(NT) k_adj_react(Geo G, DevParams P, double dt, AdjView A,
                                                  TapeView T, const double* __restrict__ rho) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  double acc[3] = {0.0, 0.0, 0.0};   // rho, o_hyp, o_inv
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const long long c = ((long long)k * G.ny + j) * G.nx + i;
      // ---- forward recomputation: fix-up, species Heun, oxygen and edema inputs
      const double id = T.idag[c], idd = T.iddag[c];
      const double g0 = T.gdag[c], w0 = T.wdag[c];
      const double di = idd - id, gw0 = g0 + w0;
      const bool pos0 = gw0 > 0.0;
      const double fg0 = pos0 ? g0 / gw0 : 0.0, fw0 = pos0 ? w0 / gw0 : 0.0;
      double y[5] = {T.pdag[c], idd, T.ndag[c], g0 - di * fg0, w0 - di * fw0};
      const double od = T.odag[c], ld = T.ldag[c], r = rho[c];
      const Ox X = oxygen_factors(P, od);
      double k1v[5], ys[5], k2v[5], yp[5];
      species_rates_f(P, r, od, X, y, k1v);
#pragma unroll
      for (int s = 0; s < 5; ++s) ys[s] = y[s] + dt * k1v[s];
      species_rates_f(P, r, od, X, ys, k2v);
#pragma unroll
      for (int s = 0; s < 5; ++s) yp[s] = y[s] + 0.5 * dt * (k1v[s] + k2v[s]);
      const double gwp = yp[3] + yp[4];
      // ---- S5^T: edema l+ = Heun(l_dag) with source S(i+)
      double lyp[5] = {A.LQ[0][c], A.LQ[1][c], A.LQ[2][c], A.LQ[3][c], A.LQ[4][c]};
      const double lo_p = A.LQ[5][c], ll_p = A.LQ[6][c];
      double l_ld;
      {
        const double lk1 = 0.5 * dt * ll_p, lk2 = 0.5 * dt * ll_p;
        double lS = lk2;
        const double lls = -P.delta_l * lk2;
        double lld = ll_p + lls;
        const double lk1t = lk1 + dt * lls;
        lS += lk1t;
        lld += -P.delta_l * lk1t;
        l_ld = lld;
        const double ip = yp[1], den = ip + P.delta_half;
        const double dS = P.delta_e * (P.delta_half / (den * den) * (1.0 - ip) - ip / den);
        lyp[1] += lS * dS;
      }
      // ---- S4^T: oxygen o+ = Heun(o_dag) with p+, g+ + w+
      double l_od;
      {
        const double k1o = -P.delta_p * yp[0] + P.delta_s * (P.o_heal - od) * gwp;
        const double os = od + dt * k1o;
        const double lk1 = 0.5 * dt * lo_p, lk2 = 0.5 * dt * lo_p;
        double lod = lo_p;
        // k2 = F(os)
        const double los = -P.delta_s * gwp * lk2;
        lyp[0] += -P.delta_p * lk2;
        double lgw = P.delta_s * (P.o_heal - os) * lk2;
        lod += los;
        const double lk1t = lk1 + dt * los;
        lod += -P.delta_s * gwp * lk1t;
        lyp[0] += -P.delta_p * lk1t;
        lgw += P.delta_s * (P.o_heal - od) * lk1t;
        lyp[3] += lgw;
        lyp[4] += lgw;
        l_od = lod;
      }
      // ---- S3^T: y+ = y + dt/2 (F(y) + F(ys)), ys = y + dt F(y)
      double ly[5], lys[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      double a2[5], lo = 0.0, lr = 0.0, lh = 0.0, lv = 0.0;
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        ly[s] = lyp[s];
        a2[s] = 0.5 * dt * lyp[s];
      }
      species_rates_adj(P, r, od, X, ys, a2, lys, lo, lr, lh, lv);
      double a1[5];
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        ly[s] += lys[s];
        a1[s] = 0.5 * dt * lyp[s] + dt * lys[s];
      }
      species_rates_adj(P, r, od, X, y, a1, ly, lo, lr, lh, lv);
      l_od += lo;
      // ---- fix-up^T: g~ = g - di g/(g+w), w~ = w - di w/(g+w), di = i_dd - i_d
      double lg0 = ly[3], lw0 = ly[4], ldi = 0.0;
      if (pos0) {
        ldi = -(ly[3] * fg0 + ly[4] * fw0);
        const double ig2 = 1.0 / (gw0 * gw0);
        lg0 = ly[3] - di * w0 * (ly[3] - ly[4]) * ig2;
        lw0 = ly[4] + di * g0 * (ly[3] - ly[4]) * ig2;
      }
      A.LD[0][c] = ly[0];          // p_dag
      A.LD[1][c] = -ldi;           // i_dag (direct part; the CN part is added later)
      A.LD[2][c] = ly[2];          // n_dag
      A.LD[3][c] = lg0;            // g_dag
      A.LD[4][c] = lw0;            // w_dag
      A.LCN[0][c] = ly[1] + ldi;   // i_ddag
      A.LCN[1][c] = l_od;          // o_dag
      A.LCN[2][c] = l_ld;          // l_dag
      A.LRHO[c] = lr;
      acc[0] += lr * (T.g[c] + T.w[c]);   // rho = rho_g g + rho_w w with rho_g = rho_w = theta
      acc[1] += lh;
      acc[2] += lv;
    }
  }
  const int slot[3] = {GRHO, GOHYP, GOINV};
  add_theta<3>(acc, slot, A);
}

// ------------------------------------------------------------------------------ S2^T, S0^T
__device__ __forceinline__ double nodeK_raw(const DevParams& P, double g, double w, double f) {
  return P.k_scale * (P.k_g * g + P.k_w * w + P.k_f * f);
}

// After the adjoint CN solves A phi_c = lambda_out_c:
//   lambda_in_c = B phi_c = phi_c + S(phi_c) with S = dt/2 D_h (faces a_d);
//   lambda of face a_d(j+1/2) = -sum_c (phi_c(j+e_d) - phi_c(j)) (cs_c(j+e_d) - cs_c(j)),
//   cs_c = in_c + out_c;  faces are dt/(2 h_d^2) x harmonic(K_j, K_{j+e_d}), K from g, w, f.
// Writes lambda_o^n, lambda_l^n, adds B phi_i to lambda_i_dag, and initialises the step-start
// lambdas of g, w, f with the K and rho sensitivities (p, i, n start at zero) before the
// transport adjoint scatters into them.
__global__ void __launch_bounds__(NT) k_adj_cn_post(Geo G, DevParams P, double half_dt, AdjView A,
                                                    TapeView T) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  double acc[1] = {0.0};
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    const double* in[3] = {T.idag, T.o, T.l};
    const double* out[3] = {T.iddag, T.odag, T.ldag};
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      const long long np[3] = {nb.at(1, 0, 0), nb.at(0, 1, 0), nb.at(0, 0, 1)};
      const long long nm[3] = {nb.at(-1, 0, 0), nb.at(0, -1, 0), nb.at(0, 0, -1)};
      auto K = [&](long long e) {
        const double kr = nodeK_raw(P, T.g[e], T.w[e], T.f[e]);
        return kr > 0.0 ? kr : 0.0;
      };
      const double Kc = K(c);
      double lK = 0.0;
      double Bphi[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) Bphi[q] = A.phi[q][c];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double sd = half_dt * G.ih2[d];
        const double Kp = K(np[d]), Km = K(nm[d]);
        const double sp = Kc + Kp, sm = Km + Kc;
        const double ap = sp > 0.0 ? sd * 2.0 * Kc * Kp / sp : 0.0;   // face j+1/2
        const double am = sm > 0.0 ? sd * 2.0 * Km * Kc / sm : 0.0;   // face j-1/2
        double lap = 0.0, lam = 0.0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const double* ph = A.phi[q];
          const double pc = ph[c], pp = ph[np[d]], pm = ph[nm[d]];
          Bphi[q] += ap * (pp - pc) - am * (pc - pm);
          const double cc = in[q][c] + out[q][c];
          const double cp = in[q][np[d]] + out[q][np[d]];
          const double cm = in[q][nm[d]] + out[q][nm[d]];
          lap -= (pp - pc) * (cp - cc);
          lam -= (pc - pm) * (cc - cm);
        }
        // d(face j+1/2)/dK_j = sd 2 Kp^2 / sp^2 ;  d(face j-1/2)/dK_j = sd 2 Km^2 / sm^2
        if (sp > 0.0) lK += lap * sd * 2.0 * Kp * Kp / (sp * sp);
        if (sm > 0.0) lK += lam * sd * 2.0 * Km * Km / (sm * sm);
      }
      A.LD[1][c] += Bphi[0];
      A.lam.o[c] = Bphi[1];
      A.lam.l[c] = Bphi[2];
      const double kr = nodeK_raw(P, T.g[c], T.w[c], T.f[c]);
      const double lKr = kr > 0.0 ? lK : 0.0;
      const double lr = A.LRHO[c];
      A.lam.g[c] = P.k_scale * P.k_g * lKr + P.rho_g * lr;
      A.lam.w[c] = P.k_scale * P.k_w * lKr + P.rho_w * lr;
      A.lam.f[c] = P.k_scale * P.k_f * lKr;
      A.lam.p[c] = 0.0;
      A.lam.i[c] = 0.0;
      A.lam.n[c] = 0.0;
      acc[0] += lKr * (P.k_g * T.g[c] + P.k_w * T.w[c] + P.k_f * T.f[c]);   // dK/dk_scale
    }
  }
  const int slot[1] = {GK};
  add_theta<1>(acc, slot, A);
}

// CN adjoint solve start: x = 0, r = rhs, p = D^{-1} r
__global__ void __launch_bounds__(NT) k_cn_init_rhs(Geo G, Cn3 C, AdjView A) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  double acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const long long c = ((long long)k * G.ny + j) * G.nx + i;
      const double di = C.dinv[c];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const double b = A.LCN[r][c];
        const double z = di * b;
        C.x[r][c] = 0.0;
        C.r[r][c] = b;
        C.p[r][c] = z;
        acc[3 * r + 0] += b * b;
        acc[3 * r + 1] += b * b;
        acc[3 * r + 2] += b * z;
      }
    }
  }
  double out[9];
  if (reduce_last_block<9>(acc, C.partial, C.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) cg_after_init(C.S[r], out[3 * r], out[3 * r + 1], out[3 * r + 2]);
  }
}

// ------------------------------------------------------------------------------ S1^T
struct Cub {
  long long xo[4], yo[4], zo[4];
  double wx[4], wy[4], wz[4];
  double dx[4], dy[4], dz[4];   // derivatives of the weights (index units)
};

__device__ __forceinline__ void axis_w(double X, int n, long long stride, long long o[4], double w[4],
                                       double dw[4]) {
  const double fl = floor(X);
  long long m = ((long long)fl - 1) % n;
  if (m < 0) m += n;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    o[a] = m * stride;
    m = (m + 1 == n) ? 0 : m + 1;
  }
  const double t = X - fl, tm1 = t - 1.0, tm2 = t - 2.0, tp1 = t + 1.0;
  w[0] = -t * tm1 * tm2 * (1.0 / 6.0);
  w[1] = tp1 * tm1 * tm2 * 0.5;
  w[2] = -tp1 * t * tm2 * 0.5;
  w[3] = tp1 * t * tm1 * (1.0 / 6.0);
  dw[0] = -(3.0 * t * t - 6.0 * t + 2.0) * (1.0 / 6.0);
  dw[1] = (3.0 * t * t - 4.0 * t - 1.0) * 0.5;
  dw[2] = -(3.0 * t * t - 2.0 * t - 2.0) * 0.5;
  dw[3] = (3.0 * t * t - 1.0) * (1.0 / 6.0);
}

__device__ __forceinline__ void cub_setup(Cub& C, const Geo& G, double X, double Y, double Z) {
  axis_w(X, G.nx, 1, C.xo, C.wx, C.dx);
  axis_w(Y, G.ny, G.nx, C.yo, C.wy, C.dy);
  axis_w(Z, G.nz, G.nxy, C.zo, C.wz, C.dz);
}

// value and index-space gradient of the tricubic interpolant of q
__device__ __forceinline__ double cub_eval(const Cub& C, const double* __restrict__ q, double gr[3]) {
  double s = 0.0;
  gr[0] = gr[1] = gr[2] = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const double* row = q + C.zo[c] + C.yo[b];
      double sx = 0.0, sdx = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double v = __ldg(row + C.xo[a]);
        sx += C.wx[a] * v;
        sdx += C.dx[a] * v;
      }
      s += C.wz[c] * C.wy[b] * sx;
      gr[0] += C.wz[c] * C.wy[b] * sdx;
      gr[1] += C.wz[c] * C.dy[b] * sx;
      gr[2] += C.dz[c] * C.wy[b] * sx;
    }
  return s;
}

__device__ __forceinline__ double cub_value(const Cub& C, const double* __restrict__ q) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const double* row = q + C.zo[c] + C.yo[b];
      s += C.wz[c] * C.wy[b] *
           (C.wx[0] * __ldg(row + C.xo[0]) + C.wx[1] * __ldg(row + C.xo[1]) +
            C.wx[2] * __ldg(row + C.xo[2]) + C.wx[3] * __ldg(row + C.xo[3]));
    }
  return s;
}

// transpose of interpolation: target[node] += weight * val, for up to 7 fields at once
__device__ __forceinline__ void cub_scatter(const Cub& C, double* const* tgt, const double* val,
                                            int nf) {
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const long long row = C.zo[c] + C.yo[b];
      const double wzy = C.wz[c] * C.wy[b];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double w = wzy * C.wx[a];
        const long long e = row + C.xo[a];
        for (int f = 0; f < nf; ++f) atomicAdd(tgt[f] + e, w * val[f]);
      }
    }
}

__global__ void __launch_bounds__(NT) k_adj_sl(Geo G, double dt, double3 dt_h, AdjView A,
                                               TapeView T, const double* __restrict__ div) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  const double* q[6] = {T.p, T.i, T.n, T.g, T.w, T.f};
  double* tq[7] = {A.lam.p, A.lam.i, A.lam.n, A.lam.g, A.lam.w, A.lam.f, A.LDEL};
  double* tv[3] = {A.LV[0], A.LV[1], A.LV[2]};
  const double dth[3] = {dt_h.x, dt_h.y, dt_h.z};
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    const double v0[3] = {T.v[0][c], T.v[1][c], T.v[2][c]};
    Cub Cs, Cx;
    cub_setup(Cs, G, i - v0[0] * dth[0], j - v0[1] * dth[1], k - v0[2] * dth[2]);
    double vs[3], gvs[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) vs[d] = cub_eval(Cs, T.v[d], gvs[d]);
    const double X[3] = {i - 0.5 * (v0[0] + vs[0]) * dth[0], j - 0.5 * (v0[1] + vs[1]) * dth[1],
                         k - 0.5 * (v0[2] + vs[2]) * dth[2]};
    cub_setup(Cx, G, X[0], X[1], X[2]);
    double gd[3];
    const double dX = cub_eval(Cx, div, gd);
    const double dx = div[c];
    const double m = 1.0 - 0.5 * dt * dX - 0.5 * dt * dx + 0.5 * dt * dt * dX * dx;
    const double lq[6] = {A.LD[0][c], A.LD[1][c], A.LD[2][c], A.LD[3][c], A.LD[4][c], A.LF[c]};
    double val[7];
    double lX[3] = {0.0, 0.0, 0.0};
    double lm = 0.0;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      double gq[3];
      const double qX = cub_eval(Cx, q[s], gq);
      const double lqX = (s < 5) ? m * lq[s] : lq[s];
      if (s < 5) lm += qX * lq[s];
      val[s] = lqX;
#pragma unroll
      for (int d = 0; d < 3; ++d) lX[d] += lqX * gq[d];
    }
    const double ldX = lm * (-0.5 * dt + 0.5 * dt * dt * dx);
    const double ldx = lm * (-0.5 * dt + 0.5 * dt * dt * dX);
    val[6] = ldX;
#pragma unroll
    for (int d = 0; d < 3; ++d) lX[d] += ldX * gd[d];
    cub_scatter(Cx, tq, val, 7);
    atomicAdd(A.LDEL + c, ldx);
    // X = x - dt/(2h) (v0 + vs):  lambda_v0 and lambda_vs
    double lv0[3], lvs[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lv0[d] = -0.5 * dth[d] * lX[d];
      lvs[d] = -0.5 * dth[d] * lX[d];
    }
    cub_scatter(Cs, tv, lvs, 3);
    // vs_d = I[v_d](X*):  lambda_X* = sum_d lvs_d grad I[v_d];  X* = x - dt v0 / h
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      double lXs = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) lXs += lvs[d] * gvs[d][e];
      lv0[e] += -dth[e] * lXs;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) atomicAdd(tv[d] + c, lv0[d]);
  }
}

// lambda_v^n = (scattered part) + div_h^T lambda_delta = LV - D lambda_delta
__global__ void __launch_bounds__(NT) k_adj_div(Geo G, AdjView A) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    const long long c = nb.at(0, 0, 0);
    A.lam.v[0][c] = A.LV[0][c] - (A.LDEL[nb.at(1, 0, 0)] - A.LDEL[nb.at(-1, 0, 0)]) * G.inv2h[0];
    A.lam.v[1][c] = A.LV[1][c] - (A.LDEL[nb.at(0, 1, 0)] - A.LDEL[nb.at(0, -1, 0)]) * G.inv2h[1];
    A.lam.v[2][c] = A.LV[2][c] - (A.LDEL[nb.at(0, 0, 1)] - A.LDEL[nb.at(0, 0, -1)]) * G.inv2h[2];
  }
}

int flat_blocks(long long n) {
  long long b = (n + NT - 1) / NT;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_adj_prep(const Geo& G, const AdjView& A, double inv_dt, cudaStream_t st) {
  k_adj_prep<<<flat_blocks(G.nvox), NT, 0, st>>>(G.nvox, A, inv_dt);
  return cudaGetLastError();
}

cudaError_t launch_adj_elas_coef(const Geo& G, const DevParams& P, const AdjView& A,
                                 const double* mu, const double* lam, const double* p,
                                 const double* n, double inv_Escale, bool species,
                                 cudaStream_t st) {
  k_adj_elas_coef<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, A, mu, lam, p, n, inv_Escale,
                                                   species ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_adj_react(const Geo& G, const DevParams& P, double dt, const AdjView& A,
                             const TapeView& T, const double* rho, cudaStream_t st) {
  k_adj_react<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, dt, A, T, rho);
  return cudaGetLastError();
}

cudaError_t launch_cn_init_rhs(const Geo& G, const Cn3& C, const AdjView& A, cudaStream_t st) {
  k_cn_init_rhs<<<G.grid, dim3(BX, BY), 0, st>>>(G, C, A);
  return cudaGetLastError();
}

cudaError_t launch_adj_cn_post(const Geo& G, const DevParams& P, double dt, const AdjView& A,
                               const TapeView& T, cudaStream_t st) {
  k_adj_cn_post<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, 0.5 * dt, A, T);
  return cudaGetLastError();
}

cudaError_t launch_adj_sl(const Geo& G, double dt, const AdjView& A, const TapeView& T,
                          const double* div, cudaStream_t st) {
  const double3 dth = make_double3(dt / G.h[0], dt / G.h[1], dt / G.h[2]);
  k_adj_sl<<<G.grid, dim3(BX, BY), 0, st>>>(G, dt, dth, A, T, div);
  return cudaGetLastError();
}

cudaError_t launch_adj_div(const Geo& G, const AdjView& A, cudaStream_t st) {
  k_adj_div<<<G.grid, dim3(BX, BY), 0, st>>>(G, A);
  return cudaGetLastError();
}

}  // namespace tg
