// tg_elasticity.cu -- the screened Navier-Lame solve of S6 (and of tg_init / tg_solve_elasticity).
//
// Eq. e:screening with Eq. e:variable_elasticity: -eta u + L u = b, solved in the SPD form
// (eta I - L_h) u = -b.  Component a of L_h u is
//   sum_d d_d( C^{ad} d_d u_a ) + sum_{d != a} [ d_d(mu d_a u_d) + d_a(lambda d_d u_d) ]
// with C^{aa} = lambda + 2 mu and C^{ad} = mu (d != a): compact face differences (face value
// = mean of the two nodes) for the first sum, centred differences for the mixed terms.  The
// stencil touches the 6 face and 12 edge neighbours of a node (19 of the 3x3x3 box).
//
// Per-step precomputation trades bytes for FP64 arithmetic: face coefficients already
// divided by h_d^2 and the Jacobi diagonal are stored, so a matrix-vector product needs
// 1 multiply and 6 fused multiply-adds per component for the face part.
#include "tg_internal.cuh"

namespace tg {
namespace {

__global__ void __launch_bounds__(NT) k_elas_coef(Geo G, DevParams P, Elas E,
                                                  const double* __restrict__ p,
                                                  const double* __restrict__ n, int force) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    const long long c = nb.at(0, 0, 0);
    const double muc = E.mu[c], lac = E.lam[c];
    double mfp[3], mfm[3], lfp[3], lfm[3];
    long long np[3] = {nb.at(1, 0, 0), nb.at(0, 1, 0), nb.at(0, 0, 1)};
    long long nm[3] = {nb.at(-1, 0, 0), nb.at(0, -1, 0), nb.at(0, 0, -1)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      mfp[d] = 0.5 * (muc + E.mu[np[d]]);
      mfm[d] = 0.5 * (E.mu[nm[d]] + muc);
      lfp[d] = 0.5 * (lac + E.lam[np[d]]);
      lfm[d] = 0.5 * (E.lam[nm[d]] + lac);
      const double fv = (lfp[d] + 2.0 * mfp[d]) * G.ih2[d], gv = mfp[d] * G.ih2[d];
      if (E.df) {   // (hi, lo) pairs for the double-FP32 residual
        reinterpret_cast<float2*>(E.F[d])[c] = df_pack(fv);
        reinterpret_cast<float2*>(E.G[d])[c] = df_pack(gv);
      } else {
        E.F[d][c] = fv;
        E.G[d][c] = gv;
      }
    }
    const double et = E.eta[c];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double s = et;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double cp = (d == a) ? lfp[d] + 2.0 * mfp[d] : mfp[d];
        const double cm = (d == a) ? lfm[d] + 2.0 * mfm[d] : mfm[d];
        s += (cp + cm) * G.ih2[d];
      }
      if (E.df)
        reinterpret_cast<float2*>(E.dsum[a])[c] = df_pack(s);
      else
        E.dsum[a][c] = s;
      if (E.jacobi) E.dinv[a][c] = 1.0 / s;
    }
    if (force) {
      const double sc = p[c] + n[c];
      const double th = P.zeta * tanh(sc);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double bv = th * (((p[np[d]] + n[np[d]]) - (p[nm[d]] + n[nm[d]])) * G.inv2h[d]);
        if (E.df)
          reinterpret_cast<float2*>(E.b[d])[c] = df_pack(bv);
        else
          E.b[d][c] = bv;
      }
    }
  }
}

// The coefficient build of the double-FP32 residual (mixed precision): faces, diagonal and
// force as (hi, lo) pairs, all in double-FP32 arithmetic on the FP32 units (no FP64
// operation).  The faces are formed from the pairs of the node mu and lambda, the force
// b = zeta tanh(s) grad_h s from the pairs of s = p + n (both written first by k_lame_df),
// with the double-FP32 tanh.  With Jacobi preconditioning this also writes the inner solves'
// FP32 inverse diagonal.
__global__ void __launch_bounds__(NT, 4) k_elas_coef_df(Geo G, DevParams P, Elas E, Elas32 I,
                                                     const float2* __restrict__ sdf, int force) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  Df ih2[3], i2h[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ih2[d] = df_split(G.ih2[d]);
    i2h[d] = df_split(G.inv2h[d]);
  }
  const Df zeta = df_split(P.zeta);
  auto half = [](Df x) { return Df{0.5f * x.hi, 0.5f * x.lo}; };    // exact
  auto twice = [](Df x) { return Df{2.0f * x.hi, 2.0f * x.lo}; };   // exact
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    const long long c = nb.at(0, 0, 0);
    const long long np[3] = {nb.at(1, 0, 0), nb.at(0, 1, 0), nb.at(0, 0, 1)};
    const long long nm[3] = {nb.at(-1, 0, 0), nb.at(0, -1, 0), nb.at(0, 0, -1)};
    const Df muc = df_of(E.mudf[c]), lac = df_of(E.lamdf[c]);
    Df Fp[3], Fm[3], Gp[3], Gm[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const Df mp = half(df_add_pos(muc, df_of(E.mudf[np[d]])));
      const Df mm = half(df_add_pos(df_of(E.mudf[nm[d]]), muc));
      const Df lp = half(df_add_pos(lac, df_of(E.lamdf[np[d]])));
      const Df lm = half(df_add_pos(df_of(E.lamdf[nm[d]]), lac));
      Gp[d] = df_mul(mp, ih2[d]);
      Gm[d] = df_mul(mm, ih2[d]);
      Fp[d] = df_mul(df_add_pos(lp, twice(mp)), ih2[d]);
      Fm[d] = df_mul(df_add_pos(lm, twice(mm)), ih2[d]);
      reinterpret_cast<float2*>(E.F[d])[c] = make_float2(Fp[d].hi, Fp[d].lo);
      reinterpret_cast<float2*>(E.G[d])[c] = make_float2(Gp[d].hi, Gp[d].lo);
    }
    const Df et = df_split(E.eta[c]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Df s = et;
#pragma unroll
      for (int d = 0; d < 3; ++d)
        s = df_add_pos(s, d == a ? df_add_pos(Fp[d], Fm[d]) : df_add_pos(Gp[d], Gm[d]));
      reinterpret_cast<float2*>(E.dsum[a])[c] = make_float2(s.hi, s.lo);
      if (E.jacobi) I.dinv[a][c] = 1.0f / __fadd_rn(s.hi, s.lo);
    }
    if (force) {   // the FP64 path's order: zeta tanh(s), then th ((s+ - s-) / (2 h))
      const Df th = df_mul(zeta, df_tanh(df_of(sdf[c])));
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const Df bv = df_mul(th, df_mul(df_sub(df_of(sdf[np[d]]), df_of(sdf[nm[d]])), i2h[d]));
        reinterpret_cast<float2*>(E.b[d])[c] = make_float2(bv.hi, bv.lo);
      }
    }
  }
}

// r = rhs - A u, du = 0, p = D^{-1} r;  rhs = -b (force) or the caller's b.  With SPEC the
// preconditioner runs in separate kernels afterwards: only r, du and the norms here.
template <bool SPEC>
__global__ void __launch_bounds__(NT) k_elas_init(Geo G, Elas E, int minus_b) {
  const double* const u[3] = {E.u[0], E.u[1], E.u[2]};
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const bool on = (i < G.nx) && (j < G.ny);
  double acc[3] = {0.0, 0.0, 0.0};
  if (on) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      double Au[3];
      Au[0] = elas_row64<0>(G, nb, c, E, u);
      Au[1] = elas_row64<1>(G, nb, c, E, u);
      Au[2] = elas_row64<2>(G, nb, c, E, u);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double rhs = minus_b ? -E.b[a][c] : E.b[a][c];
        const double res = rhs - Au[a];
        E.r[a][c] = res;
        E.du[a][c] = 0.0;
        acc[0] += rhs * rhs;
        acc[1] += res * res;
        if (!SPEC) {
          const double z = E.dinv[a][c] * res;
          E.p[a][c] = z;
          acc[2] += res * z;
        }
      }
    }
  }
  double out[3];
  if (reduce_last_block<3>(acc, E.partial, E.counter, out) && threadIdx.x == 0 && threadIdx.y == 0)
    cg_after_init(*E.S, out[0], out[1], out[2]);
}

__global__ void __launch_bounds__(NT) k_elas_matvec(Geo G, Elas E) {
  if (E.S->status != CG_RUNNING) return;
  const double* const p[3] = {E.p[0], E.p[1], E.p[2]};
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const bool on = (i < G.nx) && (j < G.ny);
  double acc[1] = {0.0};
  if (on) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      const double q0 = elas_row64<0>(G, nb, c, E, p);
      const double q1 = elas_row64<1>(G, nb, c, E, p);
      const double q2 = elas_row64<2>(G, nb, c, E, p);
      E.q[0][c] = q0;
      E.q[1][c] = q1;
      E.q[2][c] = q2;
      acc[0] += p[0][c] * q0 + p[1][c] * q1 + p[2][c] * q2;
    }
  }
  double out[1];
  if (reduce_last_block<1>(acc, E.partial, E.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
    E.S->pq = out[0];
    E.S->alpha = E.S->rz / out[0];
  }
}

template <bool SPEC>
__global__ void __launch_bounds__(NT) k_elas_update(Geo G, Elas E) {
  if (E.S->status != CG_RUNNING) return;
  const double alpha = E.S->alpha;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const bool on = (i < G.nx) && (j < G.ny);
  double acc[2] = {0.0, 0.0};
  if (on) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const long long c = ((long long)k * G.ny + j) * G.nx + i;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        E.du[a][c] += alpha * E.p[a][c];
        const double res = E.r[a][c] - alpha * E.q[a][c];
        E.r[a][c] = res;
        if (!SPEC) acc[0] += res * (E.dinv[a][c] * res);
        acc[1] += res * res;
      }
    }
  }
  double out[2];
  if (reduce_last_block<2>(acc, E.partial, E.counter, out) && threadIdx.x == 0 &&
      threadIdx.y == 0) {
    if (SPEC)
      cg_after_update_rr(*E.S, out[1]);
    else
      cg_after_update(*E.S, out[0], out[1]);
  }
}

__global__ void __launch_bounds__(NT) k_elas_pupdate(Geo G, Elas E) {
  if (E.S->status != CG_RUNNING) return;
  const double beta = E.S->beta;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) E.p[a][c] = E.dinv[a][c] * E.r[a][c] + beta * E.p[a][c];
  }
}

// p = z + beta p with z from the spectral preconditioner (p = z on the first iteration)
__global__ void __launch_bounds__(NT) k_elas_pupdate_spec(Geo G, Elas E) {
  if (E.S->status != CG_RUNNING) return;
  const double beta = E.S->beta;
  const bool first = E.S->it == 0;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) E.p[a][c] = first ? E.z[a][c] : E.z[a][c] + beta * E.p[a][c];
  }
}

// u += du (du = -u when the right-hand side vanished, i.e. u = 0), v = vo + du / dt with vo
// the velocity of the starting guess: v^n for the linear extrapolation (extrap == 1),
// v^n + (v^n - v^{n-1}) for the quadratic one (extrap == 2), 0 without (extrap == 0).  A step
// keeps v^n in vp before writing v^{n+1}.
__global__ void __launch_bounds__(NT) k_elas_finish(Geo G, Elas E, double inv_dt, int zero_rhs,
                                                    int extrap) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double uo = E.u[a][c];
      const double du = zero_rhs ? -uo : E.du[a][c];
      E.u[a][c] = zero_rhs ? 0.0 : uo + du;
      if (inv_dt > 0.0) {
        const double vn = E.v[a][c];
        const double vo = extrap == 0 ? 0.0 : (extrap == 1 ? vn : vn + (vn - E.vp[a][c]));
        if (E.vp[a]) E.vp[a][c] = vn;
        E.v[a][c] = vo + du * inv_dt;
      }
    }
  }
}

}  // namespace

cudaError_t launch_elas_coef_df(const Geo& G, const DevParams& P, const Elas& E,
                                const Elas32& I, const float2* sdf, bool force, cudaStream_t st) {
  TG_TIMED(K_ELAS_COEF_DF, st,
           k_elas_coef_df<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, E, I, sdf, force ? 1 : 0));
  return cudaGetLastError();
}

cudaError_t launch_elas_coef(const Geo& G, const DevParams& P, const Elas& E, const double* p,
                             const double* n, bool force, cudaStream_t st) {
  TG_TIMED(K_ELAS_COEF, st,
           k_elas_coef<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, E, p, n, force ? 1 : 0));
  return cudaGetLastError();
}

cudaError_t launch_elas_init(const Geo& G, const Elas& E, bool minus_b, cudaStream_t st) {
  TG_TIMED(K_ELAS_INIT, st,
           k_elas_init<false><<<G.grid, dim3(BX, BY), 0, st>>>(G, E, minus_b ? 1 : 0));
  return cudaGetLastError();
}

cudaError_t launch_elas_init_spec(const Geo& G, const Elas& E, bool minus_b, cudaStream_t st) {
  TG_TIMED(K_ELAS_INIT_SPEC, st,
           k_elas_init<true><<<G.grid, dim3(BX, BY), 0, st>>>(G, E, minus_b ? 1 : 0));
  return cudaGetLastError();
}

cudaError_t launch_elas_matvec(const Geo& G, const Elas& E, cudaStream_t st) {
  TG_TIMED(K_ELAS_MATVEC, st, k_elas_matvec<<<G.grid, dim3(BX, BY), 0, st>>>(G, E));
  return cudaGetLastError();
}

cudaError_t launch_elas_update(const Geo& G, const Elas& E, cudaStream_t st) {
  TG_TIMED(K_ELAS_UPDATE, st, k_elas_update<false><<<G.grid, dim3(BX, BY), 0, st>>>(G, E));
  TG_TIMED(K_ELAS_PUPDATE, st, k_elas_pupdate<<<G.grid, dim3(BX, BY), 0, st>>>(G, E));
  return cudaGetLastError();
}

cudaError_t launch_elas_update_spec(const Geo& G, const Elas& E, cudaStream_t st) {
  TG_TIMED(K_ELAS_UPDATE_SPEC, st, k_elas_update<true><<<G.grid, dim3(BX, BY), 0, st>>>(G, E));
  return cudaGetLastError();
}

cudaError_t launch_elas_pupdate_spec(const Geo& G, const Elas& E, cudaStream_t st) {
  TG_TIMED(K_ELAS_PUPDATE_SPEC, st, k_elas_pupdate_spec<<<G.grid, dim3(BX, BY), 0, st>>>(G, E));
  return cudaGetLastError();
}

cudaError_t launch_elas_finish(const Geo& G, const Elas& E, double inv_dt, bool zero_rhs,
                               int extrap, cudaStream_t st) {
  TG_TIMED(K_ELAS_FINISH, st,
           k_elas_finish<<<G.grid, dim3(BX, BY), 0, st>>>(G, E, inv_dt, zero_rhs ? 1 : 0,
                                                          extrap));
  return cudaGetLastError();
}

}  // namespace tg
