// tg_mixed.cu -- the TG_MIXED precision: FP32 stencils and interpolation, FP64 residuals,
// reductions and state.
//
// Elasticity (S6) is solved by iterative refinement: the outer loop evaluates the residual
// r = rhs - A u of the FP64 operator in FP64 and stops at |r| <= rtol |rhs| (the same test as
// the FP64 path); each sweep solves A e = r approximately with Jacobi-PCG in FP32 and adds e
// to u in FP64.  The FP32 operator rebuilds its face coefficients on the fly from node
// values of mu, lambda and eta (FP32 arithmetic is cheap on this part, bytes are not), so a
// matrix-vector product streams 6 FP32 arrays instead of 17 FP64 ones.  Dot products form
// FP32 products per voxel, sum a thread's few voxels in FP32 and accumulate across threads
// and blocks in FP64.
//
// Transport (S1) gathers from FP32 copies of v, div v and the six transported fields.  The
// departure point is kept as (node index, FP32 sub-cell offset), so FP32 loses no precision
// on the coordinate itself; the result is written to the FP64 state.
#include "tg_internal.cuh"

namespace tg {
namespace {

// ------------------------------------------------------------------------------ conversions

__global__ void __launch_bounds__(NT) k_to_f32(long long n, F32Copy c) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
#pragma unroll 1
    for (int a = 0; a < c.count; ++a) c.dst[a][e] = (float)c.src[a][e];
  }
}

// FP32 node coefficients and Jacobi inverse diagonal from the FP64 ones
__global__ void __launch_bounds__(NT) k_elas32_coef(long long n, const double* __restrict__ mu,
                                                    const double* __restrict__ lam,
                                                    const double* __restrict__ eta,
                                                    const double* __restrict__ d0,
                                                    const double* __restrict__ d1,
                                                    const double* __restrict__ d2, Elas32 I) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    I.mu[e] = (float)mu[e];
    I.lam[e] = (float)lam[e];
    I.eta[e] = (float)eta[e];
    I.dinv[0][e] = (float)d0[e];
    I.dinv[1][e] = (float)d1[e];
    I.dinv[2][e] = (float)d2[e];
  }
}

// ------------------------------------------------------------------------------ FP32 operator

struct Fac32 {
  float Fp[3], Fm[3];   // (lambda + 2 mu) faces / h_d^2 at +e_d and -e_d
  float Gp[3], Gm[3];   // mu faces / h_d^2
  float mup[3], mum[3]; // node mu at c +/- e_d
  float lap[3], lam[3]; // node lambda at c +/- e_d
  float eta;
};

__device__ __forceinline__ void load_fac32(const Geo& G, const float ih2[3], const Nbr& nb,
                                           long long c, const float* __restrict__ mu,
                                           const float* __restrict__ la,
                                           const float* __restrict__ eta, Fac32& f) {
  const float muc = __ldg(mu + c), lac = __ldg(la + c);
  f.eta = __ldg(eta + c);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const long long jp = nb.at(d == 0, d == 1, d == 2), jm = nb.at(-(d == 0), -(d == 1), -(d == 2));
    f.mup[d] = __ldg(mu + jp);
    f.mum[d] = __ldg(mu + jm);
    f.lap[d] = __ldg(la + jp);
    f.lam[d] = __ldg(la + jm);
    const float gp = 0.5f * (muc + f.mup[d]), gm = 0.5f * (f.mum[d] + muc);
    const float lp = 0.5f * (lac + f.lap[d]), lm = 0.5f * (f.lam[d] + lac);
    f.Gp[d] = gp * ih2[d];
    f.Gm[d] = gm * ih2[d];
    f.Fp[d] = (lp + 2.0f * gp) * ih2[d];
    f.Fm[d] = (lm + 2.0f * gm) * ih2[d];
  }
}

template <int A, int D>
__device__ __forceinline__ float mixed32(const Nbr& nb, const float* __restrict__ xd,
                                         const Fac32& f) {
  const float epp = __ldg(xd + at2<A, D>(nb, +1, +1));
  const float epm = __ldg(xd + at2<A, D>(nb, -1, +1));
  const float emp = __ldg(xd + at2<A, D>(nb, +1, -1));
  const float emm = __ldg(xd + at2<A, D>(nb, -1, -1));
  return f.mup[D] * (epp - epm) - f.mum[D] * (emp - emm) + f.lap[A] * (epp - emp) -
         f.lam[A] * (epm - emm);
}

template <int A>
__device__ __forceinline__ float row32(const Nbr& nb, long long c, const Fac32& f,
                                       const float* const x[3], const float sc[3][3]) {
  constexpr int D1 = (A + 1) % 3, D2 = (A + 2) % 3;
  const float* __restrict__ xa = x[A];
  float diag = f.eta;
  float off = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float cp = (d == A) ? f.Fp[d] : f.Gp[d];
    const float cm = (d == A) ? f.Fm[d] : f.Gm[d];
    diag += cp + cm;
    off += cp * __ldg(xa + nb.at(d == 0, d == 1, d == 2)) +
           cm * __ldg(xa + nb.at(-(d == 0), -(d == 1), -(d == 2)));
  }
  float v = diag * __ldg(xa + c) - off;
  v -= sc[A][D1] * mixed32<A, D1>(nb, x[D1], f);
  v -= sc[A][D2] * mixed32<A, D2>(nb, x[D2], f);
  return v;
}

struct Consts32 {
  float ih2[3];
  float sc[3][3];
};

__device__ __forceinline__ bool running(const CgScal* S) { return S->status == CG_RUNNING; }

__global__ void __launch_bounds__(NT) k_elas32_matvec(Geo G, Consts32 K, Elas32 I) {
  if (!running(I.S)) return;
  const float* const p[3] = {I.p[0], I.p[1], I.p[2]};
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  float part = 0.0f;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      Fac32 f;
      load_fac32(G, K.ih2, nb, c, I.mu, I.lam, I.eta, f);
      const float q0 = row32<0>(nb, c, f, p, K.sc);
      const float q1 = row32<1>(nb, c, f, p, K.sc);
      const float q2 = row32<2>(nb, c, f, p, K.sc);
      I.q[0][c] = q0;
      I.q[1][c] = q1;
      I.q[2][c] = q2;
      part += __ldg(p[0] + c) * q0 + __ldg(p[1] + c) * q1 + __ldg(p[2] + c) * q2;
    }
  }
  double acc[1] = {(double)part};
  double out[1];
  if (reduce_last_block<1>(acc, I.partial, I.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
    I.S->pq = out[0];
    I.S->alpha = I.S->rz / out[0];
  }
}

__global__ void __launch_bounds__(NT) k_elas32_update(Geo G, Elas32 I) {
  if (!running(I.S)) return;
  const float alpha = (float)I.S->alpha;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  float prz = 0.0f, prr = 0.0f;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const long long c = ((long long)k * G.ny + j) * G.nx + i;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        I.e[a][c] += alpha * I.p[a][c];
        const float res = I.r[a][c] - alpha * I.q[a][c];
        I.r[a][c] = res;
        prz += res * (I.dinv[a][c] * res);
        prr += res * res;
      }
    }
  }
  double acc[2] = {(double)prz, (double)prr};
  double out[2];
  if (reduce_last_block<2>(acc, I.partial, I.counter, out) && threadIdx.x == 0 && threadIdx.y == 0)
    cg_after_update(*I.S, out[0], out[1]);
}

__global__ void __launch_bounds__(NT) k_elas32_pupdate(Geo G, Elas32 I) {
  if (!running(I.S)) return;
  const float beta = (float)I.S->beta;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) I.p[a][c] = I.dinv[a][c] * I.r[a][c] + beta * I.p[a][c];
  }
}

// ------------------------------------------------------------------------------ refinement

// FP64 residual r = rhs - A u of the current iterate; decides the outer stop and starts the
// inner FP32 solve A e = r from e = 0 with tolerance max(tau_min, rtol_safety).
__global__ void __launch_bounds__(NT) k_elas_ir_residual(Geo G, Elas E, Elas32 I, CgScal* Sout,
                                                         int minus_b, double tau_min) {
  const double* const u[3] = {E.u[0], E.u[1], E.u[2]};
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  double acc[3] = {0.0, 0.0, 0.0};
  if (i < G.nx && j < G.ny) {
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
        const float r32 = (float)res;
        const float z32 = I.dinv[a][c] * r32;
        I.r[a][c] = r32;
        I.p[a][c] = z32;
        I.e[a][c] = 0.0f;
        acc[0] += rhs * rhs;
        acc[1] += res * res;
        acc[2] += (double)r32 * (double)z32;
      }
    }
  }
  double out[3];
  if (reduce_last_block<3>(acc, E.partial, E.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
    CgScal& O = *Sout;
    CgScal& S = *I.S;
    const double bb = out[0], rr = out[1], rz = out[2];
    O.bb = bb;
    O.rr = rr;
    O.it += 1;
    if (bb == 0.0) {
      O.status = CG_ZERO_RHS;
    } else if (!isfinite(rr)) {
      O.status = CG_NONFINITE;
    } else if (sqrt(rr) <= O.rtol * sqrt(bb)) {
      O.status = CG_CONVERGED;
    } else {
      O.status = CG_RUNNING;
    }
    // inner solve: rhs r, relative target max(tau_min, half of what the outer still needs)
    S.bb = rr;
    S.rr = rr;
    S.rz = rz;
    S.it = 0;
    S.maxit = O.maxit;
    S.alpha = 0.0;
    S.beta = 0.0;
    S.rtol = (rr > 0.0) ? fmax(tau_min, 0.5 * O.rtol * sqrt(bb / rr)) : 1.0;
    S.status = (O.status == CG_RUNNING) ? CG_RUNNING : CG_CONVERGED;
  }
}

// u += e, du += e (FP64 accumulation of the FP32 correction)
__global__ void __launch_bounds__(NT) k_elas_ir_correct(long long n, Elas E, Elas32 I) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double e = (double)I.e[a][c];
      E.u[a][c] += e;
      E.du[a][c] += e;
    }
  }
}

// v = du / dt; a vanishing right-hand side means u = 0
__global__ void __launch_bounds__(NT) k_elas_ir_finish(long long n, Elas E, double inv_dt,
                                                       int zero_rhs) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double du = E.du[a][c];
      if (zero_rhs) {
        du -= E.u[a][c];
        E.u[a][c] = 0.0;
      }
      if (inv_dt > 0.0) E.v[a][c] = du * inv_dt;
    }
  }
}

// ------------------------------------------------------------------------------ FP32 transport

struct Cubic32 {
  long long xo[4], yo[4], zo[4];
  float wx[4], wy[4], wz[4];
};

__device__ __forceinline__ void lagrange4f(float t, float w[4]) {
  const float tm1 = t - 1.0f, tm2 = t - 2.0f, tp1 = t + 1.0f;
  w[0] = -t * tm1 * tm2 * (1.0f / 6.0f);
  w[1] = tp1 * tm1 * tm2 * 0.5f;
  w[2] = -tp1 * t * tm2 * 0.5f;
  w[3] = tp1 * t * tm1 * (1.0f / 6.0f);
}

// node j plus sub-cell offset d (FP32): base node j + floor(d), fraction d - floor(d)
__device__ __forceinline__ void axis32(int j, float d, int n, long long stride, long long o[4],
                                       float w[4]) {
  const float fl = floorf(d);
  long long m = ((long long)j + (long long)fl - 1) % n;
  if (m < 0) m += n;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    o[a] = m * stride;
    m = (m + 1 == n) ? 0 : m + 1;
  }
  lagrange4f(d - fl, w);
}

__device__ __forceinline__ float eval32(const Cubic32& T, const float* __restrict__ q) {
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float sy = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float* row = q + T.zo[c] + T.yo[b];
      const float sx = T.wx[0] * __ldg(row + T.xo[0]) + T.wx[1] * __ldg(row + T.xo[1]) +
                       T.wx[2] * __ldg(row + T.xo[2]) + T.wx[3] * __ldg(row + T.xo[3]);
      sy += T.wy[b] * sx;
    }
    s += T.wz[c] * sy;
  }
  return s;
}

__global__ void __launch_bounds__(NT) k_sl32(Geo G, float dt, float3 dt_h, Sl32 S) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    const float v0x = S.v[0][c], v0y = S.v[1][c], v0z = S.v[2][c];
    Cubic32 T;
    axis32(i, -v0x * dt_h.x, G.nx, 1, T.xo, T.wx);
    axis32(j, -v0y * dt_h.y, G.ny, G.nx, T.yo, T.wy);
    axis32(k, -v0z * dt_h.z, G.nz, G.nxy, T.zo, T.wz);
    const float vsx = eval32(T, S.v[0]), vsy = eval32(T, S.v[1]), vsz = eval32(T, S.v[2]);
    axis32(i, -0.5f * (v0x + vsx) * dt_h.x, G.nx, 1, T.xo, T.wx);
    axis32(j, -0.5f * (v0y + vsy) * dt_h.y, G.ny, G.nx, T.yo, T.wy);
    axis32(k, -0.5f * (v0z + vsz) * dt_h.z, G.nz, G.nxy, T.zo, T.wz);
    const float dX = eval32(T, S.div);
    const float dx = S.div[c];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const float qX = eval32(T, S.q[s]);
      const float gX = -qX * dX;
      const float qs = qX + dt * gX;
      const float gs = -qs * dx;
      S.out[s][c] = (double)(qX + 0.5f * dt * (gX + gs));
    }
    S.out[5][c] = (double)eval32(T, S.q[5]);
  }
}

int stream_blocks(long long n) {
  long long b = (n + NT - 1) / NT;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_to_f32(long long n, const F32Copy& c, cudaStream_t st) {
  k_to_f32<<<stream_blocks(n), NT, 0, st>>>(n, c);
  return cudaGetLastError();
}

cudaError_t launch_elas32_coef(const Geo& G, const Elas& E, const Elas32& I, cudaStream_t st) {
  k_elas32_coef<<<stream_blocks(G.nvox), NT, 0, st>>>(G.nvox, E.mu, E.lam, E.eta, E.dinv[0],
                                                      E.dinv[1], E.dinv[2], I);
  return cudaGetLastError();
}

static Consts32 consts32(const Geo& G) {
  Consts32 K;
  for (int d = 0; d < 3; ++d) K.ih2[d] = (float)G.ih2[d];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) K.sc[a][d] = (float)G.s_cross[a][d];
  return K;
}

cudaError_t launch_elas_ir_residual(const Geo& G, const Elas& E, const Elas32& I, CgScal* Sout,
                                    bool minus_b, double tau_min, cudaStream_t st) {
  k_elas_ir_residual<<<G.grid, dim3(BX, BY), 0, st>>>(G, E, I, Sout, minus_b ? 1 : 0, tau_min);
  return cudaGetLastError();
}

cudaError_t launch_elas32_matvec(const Geo& G, const Elas32& I, cudaStream_t st) {
  k_elas32_matvec<<<G.grid, dim3(BX, BY), 0, st>>>(G, consts32(G), I);
  return cudaGetLastError();
}

cudaError_t launch_elas32_update(const Geo& G, const Elas32& I, cudaStream_t st) {
  k_elas32_update<<<G.grid, dim3(BX, BY), 0, st>>>(G, I);
  k_elas32_pupdate<<<G.grid, dim3(BX, BY), 0, st>>>(G, I);
  return cudaGetLastError();
}

cudaError_t launch_elas_ir_correct(const Geo& G, const Elas& E, const Elas32& I, cudaStream_t st) {
  k_elas_ir_correct<<<stream_blocks(G.nvox), NT, 0, st>>>(G.nvox, E, I);
  return cudaGetLastError();
}

cudaError_t launch_elas_ir_finish(const Geo& G, const Elas& E, double inv_dt, bool zero_rhs,
                                  cudaStream_t st) {
  k_elas_ir_finish<<<stream_blocks(G.nvox), NT, 0, st>>>(G.nvox, E, inv_dt, zero_rhs ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_sl32(const Geo& G, double dt, const Sl32& S, cudaStream_t st) {
  const float3 dth = make_float3((float)(dt / G.h[0]), (float)(dt / G.h[1]), (float)(dt / G.h[2]));
  k_sl32<<<G.grid, dim3(BX, BY), 0, st>>>(G, (float)dt, dth, S);
  return cudaGetLastError();
}

}  // namespace tg
