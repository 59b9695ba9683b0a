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
#include "tg_tiles.cuh"

namespace tg {
namespace {

// ------------------------------------------------------------------------------ conversions

__global__ void __launch_bounds__(NT) k_to_f32(long long n, F32Copy c) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
#pragma unroll 1
    for (int a = 0; a < c.count; ++a) c.dst[a][e] = f32_of(c.src[a][e]);
  }
}

// FP32 node coefficients and Jacobi inverse diagonal from the FP64 ones; with the double-FP32
// residual also the (hi, lo) pairs of mu, lambda and the starting u.  parts selects
// ELAS32_NODES (mu, lambda, eta and their pairs), ELAS32_DINV, ELAS32_U.
__global__ void __launch_bounds__(NT) k_elas32_coef(long long n, Elas E, Elas32 I, int parts) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    if (parts & ELAS32_NODES) {
      const Df mu = df_split(E.mu[e]), lam = df_split(E.lam[e]);   // hi = fl32(value)
      I.mu[e] = mu.hi;
      I.lam[e] = lam.hi;
      I.eta[e] = f32_of(E.eta[e]);
      if (E.df) {
        E.mudf[e] = make_float2(mu.hi, mu.lo);
        E.lamdf[e] = make_float2(lam.hi, lam.lo);
      }
    }
    if ((parts & ELAS32_DINV) && E.jacobi) {
      I.dinv[0][e] = f32_of(E.dinv[0][e]);
      I.dinv[1][e] = f32_of(E.dinv[1][e]);
      I.dinv[2][e] = f32_of(E.dinv[2][e]);
    }
    if ((parts & ELAS32_U) && E.df) {
#pragma unroll
      for (int a = 0; a < 3; ++a) E.udf[a][e] = df_pack(E.u[a][e]);
    }
  }
}

// an external right-hand side into the (hi, lo) pairs the double-FP32 residual reads
__global__ void __launch_bounds__(NT) k_df_pack3(long long n, const double* b0, const double* b1,
                                                 const double* b2, double* o0, double* o1,
                                                 double* o2) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    reinterpret_cast<float2*>(o0)[e] = df_pack(b0[e]);
    reinterpret_cast<float2*>(o1)[e] = df_pack(b1[e]);
    reinterpret_cast<float2*>(o2)[e] = df_pack(b2[e]);
  }
}

// ------------------------------------------------------------------------------ FP32 operator

// ------------------------------------------------------------------------------ FP32 inner CG

__global__ void __launch_bounds__(NT) k_elas32_matvec(Geo G, Consts32 K, Elas32 I) {
  if (!running(I.S)) return;
  __shared__ Tile32 T;
  const float part = elas32_matvec_tile<false>(G, K, I, I.S->it, I.S->beta, blockIdx.x, blockIdx.y,
                                        blockIdx.z, T);
  double acc[1] = {(double)part};
  double out[1];
  if (reduce_last_block<1>(acc, I.partial, I.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
    I.S->pq = out[0];
    I.S->alpha = I.S->rz / out[0];
  }
}

__global__ void __launch_bounds__(NT) k_elas32_update(long long n, Elas32 I) {
  if (!running(I.S)) return;
  const float alpha = (float)I.S->alpha;
  const int pb = (I.S->it & 1) ^ 1;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double drz = 0.0, drr = 0.0;
  elas32_update_range<false>(I, n, t0, n / 4, stride, alpha, pb, blockIdx.x == 0, drz, drr);
  double acc[2] = {drz, drr};
  double out[2];
  if (reduce_last_block<2>(acc, I.partial, I.counter, out) && threadIdx.x == 0 && threadIdx.y == 0)
    cg_after_update(*I.S, out[0], out[1]);
}

// the same with the spectral preconditioner: the preconditioner's last pass already wrote
// p = z + beta p_old, so the operator only stages p; the update decides convergence from
// <r, r>
__global__ void __launch_bounds__(NT) k_elas32_matvec_spec(Geo G, Consts32 K, Elas32 I) {
  if (!running(I.S)) return;
  __shared__ Tile32 T;
  const float part = elas32_matvec_tile_spec(G, K, I, I.S->it, blockIdx.x, blockIdx.y,
                                             blockIdx.z, T);
  double acc[1] = {(double)part};
  double out[1];
  if (reduce_last_block<1>(acc, I.partial, I.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
    I.S->pq = out[0];
    I.S->alpha = I.S->rz / out[0];
  }
}

__global__ void __launch_bounds__(NT) k_elas32_update_spec(long long n, Elas32 I) {
  if (!running(I.S)) return;
  const float alpha = (float)I.S->alpha;
  const int pb = (I.S->it & 1) ^ 1;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double drz = 0.0, drr = 0.0;
  elas32_update_range<false, true>(I, n, t0, n / 4, stride, alpha, pb, blockIdx.x == 0, drz,
                                   drr);
  double acc[1] = {drr};
  double out[1];
  if (reduce_last_block<1>(acc, I.partial, I.counter, out) && threadIdx.x == 0 && threadIdx.y == 0)
    cg_after_update_rr(*I.S, out[0]);
}

// ------------------------------------------------------------------------------ refinement

// FP64 residual of the current iterate, outer stopping test and start of the inner solve
template <bool DF>
__global__ void __launch_bounds__(NT, DF ? 3 : 1) k_elas_ir_residual(Geo G, Elas E, Elas32 I, CgScal* Sout,
                                                            int minus_b, double tau_min,
                                                            int max_sweeps, ScDf scd) {
  double acc[3] = {0.0, 0.0, 0.0};
  if (DF)
    elas_ir_residual_tile_df(G, E, I, minus_b, blockIdx.x, blockIdx.y, blockIdx.z, scd, acc);
  else
    elas_ir_residual_tile(G, E, I, minus_b, blockIdx.x, blockIdx.y, blockIdx.z, acc);
  double out[3];
  if (reduce_last_block<3>(acc, E.partial, E.counter, out) && threadIdx.x == 0 && threadIdx.y == 0)
    elas_ir_residual_finalize(*Sout, *I.S, out[0], out[1], out[2], tau_min, max_sweeps, true);
}

// r *= scale (the inner solve's right-hand side normalisation, a power of two: exact)
__global__ void __launch_bounds__(NT) k_elas32_scale_r(long long n, Elas32 I) {
  if (!running(I.S)) return;
  const float s = (float)I.S->scale;
  if (s == 1.0f) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int a = 0; a < 3; ++a) I.r[a][c] *= s;
  }
}

// u += e, du += e (FP64 accumulation of the FP32 correction)
__global__ void __launch_bounds__(NT) k_elas_ir_correct(long long n, Elas E, Elas32 I) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  elas_ir_correct_range(E, I, (long long)blockIdx.x * blockDim.x + threadIdx.x, n, stride,
                        1.0 / I.S->scale);
}

// Starting guess of a step's solve, extrapolation in time.  Linear: the increment
// s = dt v^n gives u^n + s = 2 u^n - u^{n-1}.  Quadratic (the previous step's velocity kept in
// vp): s = dt v^n + dt (v^n - v^{n-1}) gives 3 u^n - 3 u^{n-1} + u^{n-2}.  u = u^n + s and
// du = s, so that v^{n+1} = du / dt still measures u^{n+1} - u^n.  Each operation is rounded
// on its own (no contraction), in the oracle's order.
__global__ void __launch_bounds__(NT) k_elas_extrapolate(long long n, Elas E, double dt,
                                                         int quadratic) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (E.df) {   // mixed precision: s in double-FP32, two FP64 additions per component
    const Df dtd = df_split(dt);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const Df v = df_split(E.v[a][c]);
        const Df w = quadratic ? df_add(v, df_sub(v, df_split(E.vp[a][c]))) : v;
        const double s = df_value(df_mul(dtd, w));
        const double un = E.u[a][c] + s;
        E.u[a][c] = un;
        E.du[a][c] = s;
        E.udf[a][c] = df_pack(un);   // the pairs the double-FP32 residual reads
      }
    }
    return;
  }
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double v = E.v[a][c];
      double s = __dmul_rn(dt, v);
      if (quadratic) s = __dadd_rn(s, __dmul_rn(dt, __dsub_rn(v, E.vp[a][c])));
      E.u[a][c] = __dadd_rn(E.u[a][c], s);
      E.du[a][c] = s;
    }
  }
}

// v = du / dt (a step: v^n is kept in vp first); a vanishing right-hand side means u = 0
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
      if (inv_dt > 0.0) {
        if (E.vp[a]) E.vp[a][c] = E.v[a][c];
        E.v[a][c] = du * inv_dt;
      }
    }
  }
}

// ------------------------------------------------------------------------------ FP32 transport

struct Species6 {   // p, i, n, g, w, f
  const double* a[6];
};

// Taps of one tricubic interpolation: 32-bit voxel offsets of the four x, y, z nodes and
// their Lagrange weights.
struct Cubic32 {
  int xo[4], yo[4], zo[4];
  float wx[4], wy[4], wz[4];
};

__device__ __forceinline__ void lagrange4f(float t, float w[4]) {
  const float tm1 = t - 1.0f, tm2 = t - 2.0f, tp1 = t + 1.0f;
  w[0] = -t * tm1 * tm2 * (1.0f / 6.0f);
  w[1] = tp1 * tm1 * tm2 * 0.5f;
  w[2] = -tp1 * t * tm2 * 0.5f;
  w[3] = tp1 * t * tm1 * (1.0f / 6.0f);
}

// node j plus sub-cell offset d (FP32): base node j + floor(d), fraction d - floor(d); the
// periodic wrap takes a division only when the first node leaves [0, n)
__device__ __forceinline__ void axis32(int j, float d, int n, int stride, int o[4], float w[4]) {
  const float fl = floorf(d);
  int m = (int)((unsigned)j + (unsigned)(int)fl - 1u);
  if ((unsigned)m >= (unsigned)n) {
    long long mm = ((long long)j + (long long)fl - 1) % n;
    if (mm < 0) mm += n;
    m = (int)mm;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    o[a] = m * stride;
    m = (m + 1 == n) ? 0 : m + 1;
  }
  lagrange4f(d - fl, w);
}

// the interpolant of the four interleaved fields of q: x first, then y, then z
__device__ __forceinline__ float4 eval32x4(const Cubic32& T, const float4* __restrict__ q) {
  float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float4 sy = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float4* row = q + (T.zo[c] + T.yo[b]);
      const float4 a0 = __ldg(row + T.xo[0]), a1 = __ldg(row + T.xo[1]);
      const float4 a2 = __ldg(row + T.xo[2]), a3 = __ldg(row + T.xo[3]);
      sy.x += T.wy[b] * (T.wx[0] * a0.x + T.wx[1] * a1.x + T.wx[2] * a2.x + T.wx[3] * a3.x);
      sy.y += T.wy[b] * (T.wx[0] * a0.y + T.wx[1] * a1.y + T.wx[2] * a2.y + T.wx[3] * a3.y);
      sy.z += T.wy[b] * (T.wx[0] * a0.z + T.wx[1] * a1.z + T.wx[2] * a2.z + T.wx[3] * a3.z);
      sy.w += T.wy[b] * (T.wx[0] * a0.w + T.wx[1] * a1.w + T.wx[2] * a2.w + T.wx[3] * a3.w);
    }
    s.x += T.wz[c] * sy.x;
    s.y += T.wz[c] * sy.y;
    s.z += T.wz[c] * sy.z;
    s.w += T.wz[c] * sy.w;
  }
  return s;
}

// the velocity interpolant: the first three components only
__device__ __forceinline__ float3 eval32x3(const Cubic32& T, const float4* __restrict__ q) {
  float3 s = make_float3(0.0f, 0.0f, 0.0f);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float3 sy = make_float3(0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float4* row = q + (T.zo[c] + T.yo[b]);
      const float4 a0 = __ldg(row + T.xo[0]), a1 = __ldg(row + T.xo[1]);
      const float4 a2 = __ldg(row + T.xo[2]), a3 = __ldg(row + T.xo[3]);
      sy.x += T.wy[b] * (T.wx[0] * a0.x + T.wx[1] * a1.x + T.wx[2] * a2.x + T.wx[3] * a3.x);
      sy.y += T.wy[b] * (T.wx[0] * a0.y + T.wx[1] * a1.y + T.wx[2] * a2.y + T.wx[3] * a3.y);
      sy.z += T.wy[b] * (T.wx[0] * a0.z + T.wx[1] * a1.z + T.wx[2] * a2.z + T.wx[3] * a3.z);
    }
    s.x += T.wz[c] * sy.x;
    s.y += T.wz[c] * sy.y;
    s.z += T.wz[c] * sy.z;
  }
  return s;
}

// The interleaved FP32 inputs of S1: the velocity, div_h v by central differences and the six
// transported species.  Each difference v(+) - v(-) is taken from the split FP64 values,
// (hi+ - hi-) + (lo+ - lo-) in FP32, so that it keeps FP32's relative precision where the
// neighbours nearly cancel, without FP64 arithmetic.
__global__ void __launch_bounds__(NT) k_sl32_pack(Geo G, const double* __restrict__ vx,
                                                  const double* __restrict__ vy,
                                                  const double* __restrict__ vz, Species6 q, Sl32 S) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const float i2h[3] = {f32_of(G.inv2h[0]), f32_of(G.inv2h[1]), f32_of(G.inv2h[2])};
  auto diff = [](double a, double b) {
    const Df x = df_split(a), y = df_split(b);
    return (x.hi - y.hi) + (x.lo - y.lo);
  };
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    const long long c = nb.at(0, 0, 0);
    const float div = diff(vx[nb.at(1, 0, 0)], vx[nb.at(-1, 0, 0)]) * i2h[0] +
                      diff(vy[nb.at(0, 1, 0)], vy[nb.at(0, -1, 0)]) * i2h[1] +
                      diff(vz[nb.at(0, 0, 1)], vz[nb.at(0, 0, -1)]) * i2h[2];
    S.v4[c] = make_float4(f32_of(vx[c]), f32_of(vy[c]), f32_of(vz[c]), 0.0f);
    S.qa[c] = make_float4(f32_of(q.a[0][c]), f32_of(q.a[1][c]), f32_of(q.a[2][c]), div);
    S.qb[c] = make_float4(f32_of(q.a[3][c]), f32_of(q.a[4][c]), f32_of(q.a[5][c]), 0.0f);
  }
}

// Semi-Lagrangian step S1 in FP32 arithmetic (FP64 state): the departure point by the
// two-stage rule of the FP64 path, tricubic interpolation of the species and div_h v there,
// and the compression source -q div v by Heun's rule along the characteristic.
__global__ void __launch_bounds__(NT, 3) k_sl32(Geo G, float dt, float3 dt_h, Sl32 S) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int nxy = G.nx * G.ny;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const int c = (k * G.ny + j) * G.nx + i;
    const float4 v0 = __ldg(S.v4 + c);
    Cubic32 T;
    axis32(i, -v0.x * dt_h.x, G.nx, 1, T.xo, T.wx);
    axis32(j, -v0.y * dt_h.y, G.ny, G.nx, T.yo, T.wy);
    axis32(k, -v0.z * dt_h.z, G.nz, nxy, T.zo, T.wz);
    const float3 vs = eval32x3(T, S.v4);
    axis32(i, -0.5f * (v0.x + vs.x) * dt_h.x, G.nx, 1, T.xo, T.wx);
    axis32(j, -0.5f * (v0.y + vs.y) * dt_h.y, G.ny, G.nx, T.yo, T.wy);
    axis32(k, -0.5f * (v0.z + vs.z) * dt_h.z, G.nz, nxy, T.zo, T.wz);
    const float4 a = eval32x4(T, S.qa);   // p, i, n, div v at the departure point
    const float4 b = eval32x4(T, S.qb);   // g, w, f
    const float dX = a.w;
    const float dx = __ldg(S.qa + c).w;
    const float qX[5] = {a.x, a.y, a.z, b.x, b.y};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const float gX = -qX[s] * dX;
      const float qs = qX[s] + dt * gX;
      const float gs = -qs * dx;
      S.out[s][c] = f64_of(qX[s] + 0.5f * dt * (gX + gs));
    }
    S.out[5][c] = f64_of(b.z);
  }
}

int stream_blocks(long long n) {
  long long b = (n + NT - 1) / NT;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_to_f32(long long n, const F32Copy& c, cudaStream_t st) {
  TG_TIMED(K_TO_F32, st, k_to_f32<<<stream_blocks(n), NT, 0, st>>>(n, c));
  return cudaGetLastError();
}

cudaError_t launch_elas32_coef(const Geo& G, const Elas& E, const Elas32& I, cudaStream_t st,
                              int parts) {
  TG_TIMED(K_ELAS32_COEF, st,
           k_elas32_coef<<<stream_blocks(G.nvox), NT, 0, st>>>(G.nvox, E, I, parts));
  return cudaGetLastError();
}

cudaError_t launch_df_pack3(const Geo& G, const double* const b[3], double* const out[3],
                            cudaStream_t st) {
  TG_TIMED(K_DF_PACK3, st,
           k_df_pack3<<<stream_blocks(G.nvox), NT, 0, st>>>(G.nvox, b[0], b[1], b[2], out[0], out[1],
                                                            out[2]));
  return cudaGetLastError();
}



cudaError_t launch_elas_ir_residual(const Geo& G, const Elas& E, const Elas32& I, CgScal* Sout,
                                    bool minus_b, double tau_min, cudaStream_t st) {
  if (E.df)
    TG_TIMED(K_ELAS_IR_RESIDUAL_DF, st,
             k_elas_ir_residual<true><<<G.grid, dim3(BX, BY), 0, st>>>(G, E, I, Sout, minus_b ? 1 : 0,
                                                                       tau_min, 1 << 30,
                                                                       sc_df_host(G)));
  else
    TG_TIMED(K_ELAS_IR_RESIDUAL, st,
             k_elas_ir_residual<false><<<G.grid, dim3(BX, BY), 0, st>>>(G, E, I, Sout, minus_b ? 1 : 0,
                                                                        tau_min, 1 << 30,
                                                                        ScDf{}));
  return cudaGetLastError();
}

cudaError_t launch_elas32_matvec(const Geo& G, const Elas32& I, cudaStream_t st) {
  TG_TIMED(K_ELAS32_MATVEC, st,
           k_elas32_matvec<<<G.grid, dim3(BX, BY), 0, st>>>(G, make_consts32(G), I));
  return cudaGetLastError();
}

// flat launches that reduce: never more blocks than the partial-sum buffer holds
static int reduce_blocks(const Geo& G, long long items) {
  long long b = (items + NT - 1) / NT;
  b = b < 8LL * 152 ? b : 8LL * 152;
  b = b < G.nblocks ? b : G.nblocks;
  return (int)(b > 0 ? b : 1);
}

cudaError_t launch_elas32_update(const Geo& G, const Elas32& I, cudaStream_t st) {
  TG_TIMED(K_ELAS32_UPDATE, st,
           k_elas32_update<<<reduce_blocks(G, (G.nvox + 3) / 4), NT, 0, st>>>(G.nvox, I));
  return cudaGetLastError();
}

cudaError_t launch_elas32_scale_r(const Geo& G, const Elas32& I, cudaStream_t st) {
  TG_TIMED(K_ELAS32_SCALE_R, st, k_elas32_scale_r<<<stream_blocks(G.nvox), NT, 0, st>>>(G.nvox, I));
  return cudaGetLastError();
}

cudaError_t launch_elas32_matvec_spec(const Geo& G, const Elas32& I, cudaStream_t st) {
  TG_TIMED(K_ELAS32_MATVEC_SPEC, st,
           k_elas32_matvec_spec<<<G.grid, dim3(BX, BY), 0, st>>>(G, make_consts32(G), I));
  return cudaGetLastError();
}

cudaError_t launch_elas32_update_spec(const Geo& G, const Elas32& I, cudaStream_t st) {
  TG_TIMED(K_ELAS32_UPDATE_SPEC, st,
           k_elas32_update_spec<<<reduce_blocks(G, (G.nvox + 3) / 4), NT, 0, st>>>(G.nvox, I));
  return cudaGetLastError();
}

cudaError_t launch_elas_ir_correct(const Geo& G, const Elas& E, const Elas32& I, cudaStream_t st) {
  TG_TIMED(K_ELAS_IR_CORRECT, st,
           k_elas_ir_correct<<<stream_blocks(G.nvox), NT, 0, st>>>(G.nvox, E, I));
  return cudaGetLastError();
}

cudaError_t launch_elas_extrapolate(const Geo& G, const Elas& E, double dt, bool quadratic,
                                    cudaStream_t st) {
  TG_TIMED(K_ELAS_EXTRAPOLATE, st,
           k_elas_extrapolate<<<stream_blocks(G.nvox), NT, 0, st>>>(G.nvox, E, dt,
                                                                    quadratic ? 1 : 0));
  return cudaGetLastError();
}

cudaError_t launch_elas_ir_finish(const Geo& G, const Elas& E, double inv_dt, bool zero_rhs,
                                  cudaStream_t st) {
  TG_TIMED(K_ELAS_IR_FINISH, st,
           k_elas_ir_finish<<<stream_blocks(G.nvox), NT, 0, st>>>(G.nvox, E, inv_dt, zero_rhs ? 1 : 0));
  return cudaGetLastError();
}

cudaError_t launch_sl32_pack(const Geo& G, const double* const v[3], const double* const q[6],
                             const Sl32& S, cudaStream_t st) {
  if (G.nvox >= (1LL << 31)) return cudaErrorInvalidValue;
  Species6 qs;
  for (int s = 0; s < 6; ++s) qs.a[s] = q[s];
  TG_TIMED(K_SL32_PACK, st,
           k_sl32_pack<<<G.grid, dim3(BX, BY), 0, st>>>(G, v[0], v[1], v[2], qs, S));
  return cudaGetLastError();
}

cudaError_t launch_sl32(const Geo& G, double dt, const Sl32& S, cudaStream_t st) {
  if (G.nvox >= (1LL << 31)) return cudaErrorInvalidValue;
  const float3 dth = make_float3((float)(dt / G.h[0]), (float)(dt / G.h[1]), (float)(dt / G.h[2]));
  TG_TIMED(K_SL32, st, k_sl32<<<G.grid, dim3(BX, BY), 0, st>>>(G, (float)dt, dth, S));
  return cudaGetLastError();
}

}  // namespace tg
