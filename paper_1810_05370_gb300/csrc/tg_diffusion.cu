// tg_diffusion.cu -- S0 coefficients and the Crank-Nicolson diffusion solves (S2).
//
// Section 3: (1 - dt/2 D) c^{+} = (1 + dt/2 D) c, solved by CG, for c in {i, o, l}, with
// D c = div(K grad c), K = k_scale (k_g g + k_w w + k_f f) (Eq. e:diffusion_op,
// e:diffusion_tensor).  Discretely, with face coefficients a_d = dt/(2 h_d^2) K_{j+1/2 e_d}
// (harmonic mean of the two nodes, zero when both vanish),
//   (A c)_j = c_j + sum_d [ a_d,j (c_j - c_{j+e_d}) + a_d,j-e_d (c_j - c_{j-e_d}) ].
// The three right-hand sides share the coefficient reads: every kernel below streams the
// six face values of a node once and applies them to all active solves.
#include "tg_tiles.cuh"

namespace tg {
namespace {

__device__ __forceinline__ double node_K(const DevParams& P, double g, double w, double f) {
  double k = P.k_scale * (P.k_g * g + P.k_w * w + P.k_f * f);
  return k > 0.0 ? k : 0.0;
}

__device__ __forceinline__ double harmonic(double a, double b) {
  return (a + b) > 0.0 ? 2.0 * a * b / (a + b) : 0.0;
}

// S0 in two passes.  FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU, so each face
// (one division) is formed once, by the node below it, instead of by both of its nodes:
// k_diff_faces writes a_d,j for the faces j + e_d/2 and rho; k_diff_diag then adds the faces
// below each node from the neighbours' entries.
__global__ void __launch_bounds__(NT) k_diff_faces(Geo G, DevParams P, double half_dt,
                                                   const double* __restrict__ g,
                                                   const double* __restrict__ w,
                                                   const double* __restrict__ f, double* Kfx,
                                                   double* Kfy, double* Kfz, double* rho,
                                                   float2* dfx, float2* dfy, float2* dfz) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  const double sx = half_dt * G.ih2[0], sy = half_dt * G.ih2[1], sz = half_dt * G.ih2[2];
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    auto K = [&](long long e) { return node_K(P, g[e], w[e], f[e]); };
    const long long c = nb.at(0, 0, 0);
    const double kc = K(c);
    const double fx = sx * harmonic(kc, K(nb.at(1, 0, 0)));
    const double fy = sy * harmonic(kc, K(nb.at(0, 1, 0)));
    const double fz = sz * harmonic(kc, K(nb.at(0, 0, 1)));
    Kfx[c] = fx;
    Kfy[c] = fy;
    Kfz[c] = fz;
    if (dfx) {   // (hi, lo) pairs for the mixed precision's double-FP32 residual
      dfx[c] = df_pack(fx);
      dfy[c] = df_pack(fy);
      dfz[c] = df_pack(fz);
    }
    rho[c] = P.rho_g * g[c] + P.rho_w * w[c];
  }
}

// The same S0 for the mixed precision with double-FP32 residuals, whose solves need the faces
// only as (hi, lo) pairs (double-FP32 residuals and oxygen solve) and as FP32 values (inner
// solves), with the FP32 inverse diagonal.  Pass 1 forms each node's K once in double-FP32
// from the split FP64 fields and keeps it as a pair, with rho (one FP64 addition, for its
// FP64 output); pass 2 forms each node's six faces as harmonic means in double-FP32
// arithmetic on the FP32 units (the quotient as a product with the double-FP32 reciprocal),
// so no FP64 division is left.
__global__ void __launch_bounds__(NT) k_diff_node_df(Geo G, DevParams P,
                                                     const double* __restrict__ g,
                                                     const double* __restrict__ w,
                                                     const double* __restrict__ f, float2* Kn,
                                                     double* rho) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const Df kg = df_split(P.k_g), kw = df_split(P.k_w), kf = df_split(P.k_f);
  const Df ks = df_split(P.k_scale), rg = df_split(P.rho_g), rw = df_split(P.rho_w);
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    const Df gc = df_split(g[c]), wc = df_split(w[c]);
    // node_K's order: k_scale ((k_g g + k_w w) + k_f f), clamped at 0
    Df K = df_mul(ks, df_add(df_add(df_mul(kg, gc), df_mul(kw, wc)), df_mul(kf, df_split(f[c]))));
    if (!(K.hi > 0.0f)) K = Df{0.0f, 0.0f};
    Kn[c] = make_float2(K.hi, K.lo);
    rho[c] = df_value(df_add(df_mul(rg, gc), df_mul(rw, wc)));
  }
}

// 2 a b / (a + b), 0 if a + b = 0.  Below 1e-30 (far outside tissue, where K is an FP32
// subnormal) the face, at most 2 (a + b), is dropped: it is ~1e-30 of the CN diagonal's 1, and
// the reciprocal of a subnormal sum would overflow.
__device__ __forceinline__ Df df_harmonic(Df a, Df b) {
  const Df s = df_add(a, b);
  if (!(s.hi > 1e-30f)) return Df{0.0f, 0.0f};
  const Df y = {1.0f / s.hi, 0.0f};   // reciprocal: FP32 start, one Newton step in double-FP32
  const Df inv = df_add(y, df_mul(y, df_sub(Df{1.0f, 0.0f}, df_mul(s, y))));
  const Df ab = df_mul(a, b);
  return df_mul(Df{2.0f * ab.hi, 2.0f * ab.lo}, inv);
}

__global__ void __launch_bounds__(NT) k_diff_faces_df(Geo G, Df sx, Df sy, Df sz,
                                                      const float2* __restrict__ Kn,
                                                      float2* dfx, float2* dfy, float2* dfz,
                                                      float* f32x, float* f32y, float* f32z,
                                                      float* dinv32, float* dmax) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  float dm = 0.0f;   // the largest diagonal this thread formed
  const bool on = i < G.nx && j < G.ny;
  const int k0 = blockIdx.z * G.zc, k1 = on ? min(G.nz, k0 + G.zc) : k0;
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    const long long c = nb.at(0, 0, 0);
    auto K = [&](long long e) { return df_of(__ldg(Kn + e)); };
    const Df kc = K(c);
    const Df fxp = df_mul(sx, df_harmonic(kc, K(nb.at(1, 0, 0))));
    const Df fyp = df_mul(sy, df_harmonic(kc, K(nb.at(0, 1, 0))));
    const Df fzp = df_mul(sz, df_harmonic(kc, K(nb.at(0, 0, 1))));
    const Df fxm = df_mul(sx, df_harmonic(K(nb.at(-1, 0, 0)), kc));
    const Df fym = df_mul(sy, df_harmonic(K(nb.at(0, -1, 0)), kc));
    const Df fzm = df_mul(sz, df_harmonic(K(nb.at(0, 0, -1)), kc));
    dfx[c] = make_float2(fxp.hi, fxp.lo);
    dfy[c] = make_float2(fyp.hi, fyp.lo);
    dfz[c] = make_float2(fzp.hi, fzp.lo);
    f32x[c] = fxp.hi;
    f32y[c] = fyp.hi;
    f32z[c] = fzp.hi;
    // 1 + (xp + xm) + (yp + ym) + (zp + zm), as the FP64 diagonal
    const Df d = df_add(df_add(df_add(Df{1.0f, 0.0f}, df_add(fxp, fxm)), df_add(fyp, fym)),
                        df_add(fzp, fzm));
    dinv32[c] = 1.0f / d.hi;
    dm = fmaxf(dm, d.hi);
  }
  // the block's maximum into *dmax (positive floats order as their bit patterns)
  for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  __shared__ float wmax[NT / 32];
  const int lane = (threadIdx.y * BX + threadIdx.x) & 31, warp = (threadIdx.y * BX + threadIdx.x) >> 5;
  if (lane == 0) wmax[warp] = dm;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    float b = 0.0f;
    for (int q = 0; q < NT / 32; ++q) b = fmaxf(b, wmax[q]);
    atomicMax(reinterpret_cast<unsigned int*>(dmax), __float_as_uint(b));
  }
}

// CN diagonal 1 + sum of the six faces of each node, and its inverse
__global__ void __launch_bounds__(NT) k_diff_diag(Geo G, const double* __restrict__ Kfx,
                                                  const double* __restrict__ Kfy,
                                                  const double* __restrict__ Kfz, double* dsum,
                                                  double* dinv) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    const long long c = nb.at(0, 0, 0);
    const double d = 1.0 + (Kfx[c] + Kfx[nb.at(-1, 0, 0)]) + (Kfy[c] + Kfy[nb.at(0, -1, 0)]) +
                     (Kfz[c] + Kfz[nb.at(0, 0, -1)]);
    dsum[c] = d;
    dinv[c] = 1.0 / d;
  }
}

// mask: bit r set for the solves to start; the others are marked finished
__global__ void __launch_bounds__(NT) k_cn_init(Geo G, Cn3 C, int mask) {
  double acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  cn_init_tile(G, C, blockIdx.x, blockIdx.y, blockIdx.z, acc, mask);
  double out[9];
  if (reduce_last_block<9>(acc, C.partial, C.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if ((mask >> r) & 1)
        cg_after_init(C.S[r], out[3 * r], out[3 * r + 1], out[3 * r + 2]);
      else
        cg_skip(C.S[r]);
    }
  }
}

__global__ void __launch_bounds__(NT) k_cn_matvec(Geo G, Cn3 C) {
  bool act[3];
  bool any = false;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    act[r] = C.S[r].status == CG_RUNNING;
    any |= act[r];
  }
  if (!any) return;
  double acc[3] = {0.0, 0.0, 0.0};
  cn_matvec_tile<false>(G, C, act, blockIdx.x, blockIdx.y, blockIdx.z, acc);
  double out[3];
  if (reduce_last_block<3>(acc, C.partial, C.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
      if (act[r]) {
        C.S[r].pq = out[r];
        C.S[r].alpha = C.S[r].rz / out[r];
      }
  }
}

__global__ void __launch_bounds__(NT) k_cn_update(Geo G, Cn3 C) {
  bool act[3];
  double alpha[3];
  bool any = false;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    act[r] = C.S[r].status == CG_RUNNING;
    alpha[r] = C.S[r].alpha;
    any |= act[r];
  }
  if (!any) return;
  double acc[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) acc[q] = 0.0;
  cn_update_tile(G, C, act, alpha, blockIdx.x, blockIdx.y, blockIdx.z, acc);
  double out[6];
  if (reduce_last_block<6>(acc, C.partial, C.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
      if (act[r]) cg_after_update(C.S[r], out[2 * r], out[2 * r + 1]);
  }
}

__global__ void __launch_bounds__(NT) k_cn_pupdate(Geo G, Cn3 C) {
  bool act[3];
  double beta[3];
  bool any = false;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    act[r] = C.S[r].status == CG_RUNNING;
    beta[r] = C.S[r].beta;
    any |= act[r];
  }
  if (!any) return;
  cn_pupdate_tile(G, C, act, beta, blockIdx.x, blockIdx.y, blockIdx.z);
}

}  // namespace

cudaError_t launch_diff_coef(const Geo& G, const DevParams& P, double dt, const double* g,
                             const double* w, const double* f, double* const Kf[3], double* dsum,
                             double* dinv, double* rho, cudaStream_t st,
                             double* const Kfdf[3]) {
  float2* df[3] = {nullptr, nullptr, nullptr};
  if (Kfdf)
    for (int d = 0; d < 3; ++d) df[d] = reinterpret_cast<float2*>(Kfdf[d]);
  TG_TIMED(K_DIFF_FACES, st,
           k_diff_faces<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, 0.5 * dt, g, w, f, Kf[0], Kf[1], Kf[2],
                                                         rho, df[0], df[1], df[2]));
  TG_TIMED(K_DIFF_DIAG, st,
           k_diff_diag<<<G.grid, dim3(BX, BY), 0, st>>>(G, Kf[0], Kf[1], Kf[2], dsum, dinv));
  return cudaGetLastError();
}

cudaError_t launch_diff_coef_df(const Geo& G, const DevParams& P, double dt, const double* g,
                                const double* w, const double* f, float2* Kn, double* rho,
                                float2* const Kfdf[3], float* const Kf32[3], float* dinv32,
                                float* dmax, cudaStream_t st) {
  TG_TIMED(K_DIFF_NODE_DF, st,
           k_diff_node_df<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, g, w, f, Kn, rho));
  const Df sx = df_split_host(0.5 * dt * G.ih2[0]), sy = df_split_host(0.5 * dt * G.ih2[1]),
           sz = df_split_host(0.5 * dt * G.ih2[2]);
  TG_TIMED(K_DIFF_FACES_DF, st,
           k_diff_faces_df<<<G.grid, dim3(BX, BY), 0, st>>>(G, sx, sy, sz, Kn, Kfdf[0], Kfdf[1],
                                                            Kfdf[2], Kf32[0], Kf32[1], Kf32[2],
                                                            dinv32, dmax));
  return cudaGetLastError();
}

cudaError_t launch_cn_init(const Geo& G, const Cn3& C, cudaStream_t st, int mask) {
  TG_TIMED(K_CN_INIT, st, k_cn_init<<<G.grid, dim3(BX, BY), 0, st>>>(G, C, mask));
  return cudaGetLastError();
}

cudaError_t launch_cn_iter(const Geo& G, const Cn3& C, cudaStream_t st) {
  TG_TIMED(K_CN_MATVEC, st, k_cn_matvec<<<G.grid, dim3(BX, BY), 0, st>>>(G, C));
  TG_TIMED(K_CN_UPDATE, st, k_cn_update<<<G.grid, dim3(BX, BY), 0, st>>>(G, C));
  TG_TIMED(K_CN_PUPDATE, st, k_cn_pupdate<<<G.grid, dim3(BX, BY), 0, st>>>(G, C));
  return cudaGetLastError();
}

}  // namespace tg
