// tg_cn_mixed.cu -- the Crank-Nicolson solves of S2 in the TG_MIXED precision.
//
// Section 3: (1 - dt/2 D) c+ = (1 + dt/2 D) c for c in {i, o, l}, one operator for the three.
// Iterative refinement, as for the elasticity solve of the mixed precision: the FP64 residual
// r = rhs - A x of the current fields decides convergence (|r| <= rtol |rhs|, the FP64
// path's test) and each sweep solves A e = r approximately with Jacobi PCG in FP32 on FP32
// copies of the face coefficients, then x += e in FP64.  An FP32 iteration streams half the
// bytes of an FP64 one; the three right-hand sides share every face read.
#include "tg_tiles.cuh"

namespace tg {
namespace {

// FP64 residual of the three fields; with init the right-hand sides rhs = x + dt/2 D_h x are
// formed first and kept in C.p (A x = x - dt/2 D_h x, so then r = 2 dt/2 D_h x).
__global__ void __launch_bounds__(NT) k_cn_ir_residual(Geo G, Cn3 C, Cn32 I, CgScal* Sout,
                                                       int init, double tau_min,
                                                       int max_sweeps, int mask) {
  double acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      const Faces F = load_faces(C, nb, c);
      const float di = I.dinv[c];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (!((mask >> r) & 1)) continue;
        const double* x = C.x[r];
        const double xc = x[c];
        const double s = F.xp * (x[nb.at(1, 0, 0)] - xc) - F.xm * (xc - x[nb.at(-1, 0, 0)]) +
                         F.yp * (x[nb.at(0, 1, 0)] - xc) - F.ym * (xc - x[nb.at(0, -1, 0)]) +
                         F.zp * (x[nb.at(0, 0, 1)] - xc) - F.zm * (xc - x[nb.at(0, 0, -1)]);
        double rhs;
        if (init) {
          rhs = xc + s;
          C.p[r][c] = rhs;
        } else {
          rhs = C.p[r][c];
        }
        const double res = rhs - xc + s;
        const float r32 = (float)res;
        I.r[r][c] = r32;
        I.e[r][c] = 0.0f;
        acc[3 * r + 0] += rhs * rhs;
        acc[3 * r + 1] += res * res;
        acc[3 * r + 2] += (double)r32 * (double)(di * r32);
      }
    }
  }
  double out[9];
  if (reduce_last_block<9>(acc, C.partial, C.counter, out) && threadIdx.x == 0 &&
      threadIdx.y == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if ((mask >> r) & 1) {
        elas_ir_residual_finalize(Sout[r], I.S[r], out[3 * r], out[3 * r + 1], out[3 * r + 2],
                                  tau_min, max_sweeps);
      } else {
        cg_skip(Sout[r]);
        cg_skip(I.S[r]);
      }
    }
  }
}

// The same in double-FP32 arithmetic (C.df): fields, faces and right-hand sides as (hi, lo)
// pairs, s = sum over the six faces of a (x_n - x_c) with error-free sums and products on the
// FP32 units; the norms of a thread's voxels are summed in FP32, threads and blocks in FP64.
__global__ void __launch_bounds__(NT) k_cn_ir_residual_df(Geo G, Cn3 C, Cn32 I, CgScal* Sout,
                                                          int init, double tau_min,
                                                          int max_sweeps, int mask) {
  float sbb[3] = {0.0f, 0.0f, 0.0f}, srr[3] = {0.0f, 0.0f, 0.0f}, srz[3] = {0.0f, 0.0f, 0.0f};
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      const long long nbr[6] = {nb.at(1, 0, 0), nb.at(-1, 0, 0), nb.at(0, 1, 0),
                                nb.at(0, -1, 0), nb.at(0, 0, 1), nb.at(0, 0, -1)};
      const Df f[6] = {df_of(C.Kfdf[0][c]), df_of(C.Kfdf[0][nbr[1]]), df_of(C.Kfdf[1][c]),
                       df_of(C.Kfdf[1][nbr[3]]), df_of(C.Kfdf[2][c]), df_of(C.Kfdf[2][nbr[5]])};
      const float di = I.dinv[c];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (!((mask >> r) & 1)) continue;
        const float2* x = C.xdf[r];
        const Df xc = df_of(x[c]);
        Df s = df_mul(f[0], df_sub(df_of(x[nbr[0]]), xc));
#pragma unroll
        for (int q = 1; q < 6; ++q) s = df_add(s, df_mul(f[q], df_sub(df_of(x[nbr[q]]), xc)));
        float2* rhs2 = reinterpret_cast<float2*>(C.p[r]);
        Df rhs;
        if (init) {
          rhs = df_add(xc, s);
          rhs2[c] = make_float2(rhs.hi, rhs.lo);
        } else {
          rhs = df_of(rhs2[c]);
        }
        const Df res = df_add(df_sub(rhs, xc), s);
        const float r32 = __fadd_rn(res.hi, res.lo);
        I.r[r][c] = r32;
        I.e[r][c] = 0.0f;
        sbb[r] += rhs.hi * rhs.hi;
        srr[r] += r32 * r32;
        srz[r] += r32 * (di * r32);
      }
    }
  }
  double acc[9];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    acc[3 * r + 0] = (double)sbb[r];
    acc[3 * r + 1] = (double)srr[r];
    acc[3 * r + 2] = (double)srz[r];
  }
  double out[9];
  if (reduce_last_block<9>(acc, C.partial, C.counter, out) && threadIdx.x == 0 &&
      threadIdx.y == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if ((mask >> r) & 1) {
        elas_ir_residual_finalize(Sout[r], I.S[r], out[3 * r], out[3 * r + 1], out[3 * r + 2],
                                  tau_min, max_sweeps);
      } else {
        cg_skip(Sout[r]);
        cg_skip(I.S[r]);
      }
    }
  }
}

__device__ __forceinline__ bool active3(const Cn32& I, bool (&act)[3]) {
  bool any = false;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    act[r] = I.S[r].status == CG_RUNNING;
    any |= act[r];
  }
  return any;
}

// q = A p (diagonal 1 + sum of the six faces), <p, q>
__global__ void __launch_bounds__(NT) k_cn32_matvec(Geo G, Cn32 I) {
  bool act[3];
  if (!active3(I, act)) return;
  float part[3] = {0.0f, 0.0f, 0.0f};
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      const long long xp = nb.at(1, 0, 0), xm = nb.at(-1, 0, 0), yp = nb.at(0, 1, 0),
                      ym = nb.at(0, -1, 0), zp = nb.at(0, 0, 1), zm = nb.at(0, 0, -1);
      const float fxp = __ldg(I.Kf[0] + c), fxm = __ldg(I.Kf[0] + xm);
      const float fyp = __ldg(I.Kf[1] + c), fym = __ldg(I.Kf[1] + ym);
      const float fzp = __ldg(I.Kf[2] + c), fzm = __ldg(I.Kf[2] + zm);
      const float d = 1.0f + ((fxp + fxm) + (fyp + fym) + (fzp + fzm));
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (!act[r]) continue;
        const float* p = I.p[r];
        const float pc = p[c];
        const float q = d * pc - (fxp * p[xp] + fxm * p[xm] + fyp * p[yp] + fym * p[ym] +
                                  fzp * p[zp] + fzm * p[zm]);
        I.q[r][c] = q;
        part[r] += pc * q;
      }
    }
  }
  double acc[3] = {(double)part[0], (double)part[1], (double)part[2]};
  double out[3];
  if (reduce_last_block<3>(acc, I.partial, I.counter, out) && threadIdx.x == 0 &&
      threadIdx.y == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
      if (act[r]) {
        I.S[r].pq = out[r];
        I.S[r].alpha = I.S[r].rz / out[r];
      }
  }
}

// e += alpha p, r -= alpha q; <r, D^{-1} r>, <r, r>.  float4 groups g = g0, g0 + gs, ... of an
// n-voxel system plus the scalar tail n - n % 4 .. n (block 0); a group's products are summed
// in FP32, groups in FP64.
__global__ void __launch_bounds__(NT) k_cn32_update(long long n, Cn32 I) {
  bool act[3];
  if (!active3(I, act)) return;
  float alpha[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) alpha[r] = (float)I.S[r].alpha;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const long long gs = (long long)gridDim.x * blockDim.x, ng = n / 4;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < ng; v += gs) {
    const float4 d = __ldg(reinterpret_cast<const float4*>(I.dinv) + v);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!act[r]) continue;
      float4* e4 = reinterpret_cast<float4*>(I.e[r]) + v;
      float4* r4 = reinterpret_cast<float4*>(I.r[r]) + v;
      const float4 p = reinterpret_cast<const float4*>(I.p[r])[v];
      const float4 q = reinterpret_cast<const float4*>(I.q[r])[v];
      float4 e = *e4, x = *r4;
      const float a = alpha[r];
      e.x += a * p.x; e.y += a * p.y; e.z += a * p.z; e.w += a * p.w;
      x.x -= a * q.x; x.y -= a * q.y; x.z -= a * q.z; x.w -= a * q.w;
      *e4 = e;
      *r4 = x;
      acc[2 * r] += (double)(x.x * (d.x * x.x) + x.y * (d.y * x.y) + x.z * (d.z * x.z) +
                             x.w * (d.w * x.w));
      acc[2 * r + 1] += (double)(x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w);
    }
  }
  if (blockIdx.x == 0) {
    for (long long c = 4 * ng + threadIdx.x; c < n; c += blockDim.x) {
      const float di = I.dinv[c];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (!act[r]) continue;
        I.e[r][c] += alpha[r] * I.p[r][c];
        const float res = I.r[r][c] - alpha[r] * I.q[r][c];
        I.r[r][c] = res;
        acc[2 * r] += (double)(res * (di * res));
        acc[2 * r + 1] += (double)(res * res);
      }
    }
  }
  double out[6];
  if (reduce_last_block<6>(acc, I.partial, I.counter, out) && threadIdx.x == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
      if (act[r]) cg_after_update(I.S[r], out[2 * r], out[2 * r + 1]);
  }
}

// p = D^{-1} r + beta p (p = D^{-1} r on an inner solve's first iteration), float4 groups
__global__ void __launch_bounds__(NT) k_cn32_pupdate(long long n, Cn32 I) {
  bool act[3];
  if (!active3(I, act)) return;
  float beta[3];
  bool first[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    beta[r] = (float)I.S[r].beta;
    first[r] = I.S[r].it == 0;
  }
  const long long gs = (long long)gridDim.x * blockDim.x, ng = n / 4;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < ng; v += gs) {
    const float4 d = __ldg(reinterpret_cast<const float4*>(I.dinv) + v);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!act[r]) continue;
      const float4 x = reinterpret_cast<const float4*>(I.r[r])[v];
      float4* p4 = reinterpret_cast<float4*>(I.p[r]) + v;
      const float4 z = {d.x * x.x, d.y * x.y, d.z * x.z, d.w * x.w};
      if (first[r]) {
        *p4 = z;
      } else {
        const float4 p = *p4;
        const float b = beta[r];
        *p4 = float4{z.x + b * p.x, z.y + b * p.y, z.z + b * p.z, z.w + b * p.w};
      }
    }
  }
  if (blockIdx.x == 0) {
    for (long long c = 4 * ng + threadIdx.x; c < n; c += blockDim.x) {
      const float di = I.dinv[c];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (!act[r]) continue;
        const float z = di * I.r[r][c];
        I.p[r][c] = first[r] ? z : z + beta[r] * I.p[r][c];
      }
    }
  }
}

// x += e in FP64 for the solves in the mask (e = 0 for those that did not run this sweep)
__global__ void __launch_bounds__(NT) k_cn_ir_correct(long long n, Cn3 C, Cn32 I, int mask) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!((mask >> r) & 1)) continue;
      const double x = C.x[r][c] + (double)I.e[r][c];
      C.x[r][c] = x;
      if (C.df) C.xdf[r][c] = df_pack(x);   // the next residual's pairs
    }
  }
}

int flat_blocks(const Geo& G) {   // never more blocks than the partial-sum buffer holds
  long long b = (G.nvox / 4 + NT - 1) / NT;
  b = b < 8LL * 152 ? b : 8LL * 152;
  b = b < G.nblocks ? b : G.nblocks;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t launch_cn_ir_residual(const Geo& G, const Cn3& C, const Cn32& I, CgScal* Sout,
                                  bool init, double tau_min, int max_sweeps, int mask,
                                  cudaStream_t st) {
  if (C.df)
    TG_TIMED(K_CN_IR_RESIDUAL_DF, st,
             k_cn_ir_residual_df<<<G.grid, dim3(BX, BY), 0, st>>>(G, C, I, Sout, init ? 1 : 0, tau_min,
                                                                  max_sweeps, mask));
  else
    TG_TIMED(K_CN_IR_RESIDUAL, st,
             k_cn_ir_residual<<<G.grid, dim3(BX, BY), 0, st>>>(G, C, I, Sout, init ? 1 : 0, tau_min,
                                                               max_sweeps, mask));
  return cudaGetLastError();
}

// one inner iteration of the three FP32 solves: the first iteration of a sweep forms p from
// the residual before the operator
cudaError_t launch_cn32_iter(const Geo& G, const Cn32& I, cudaStream_t st) {
  TG_TIMED(K_CN32_PUPDATE, st, k_cn32_pupdate<<<flat_blocks(G), NT, 0, st>>>(G.nvox, I));
  TG_TIMED(K_CN32_MATVEC, st, k_cn32_matvec<<<G.grid, dim3(BX, BY), 0, st>>>(G, I));
  TG_TIMED(K_CN32_UPDATE, st, k_cn32_update<<<flat_blocks(G), NT, 0, st>>>(G.nvox, I));
  return cudaGetLastError();
}

cudaError_t launch_cn_ir_correct(const Geo& G, const Cn3& C, const Cn32& I, int mask,
                                 cudaStream_t st) {
  TG_TIMED(K_CN_IR_CORRECT, st, k_cn_ir_correct<<<flat_blocks(G), NT, 0, st>>>(G.nvox, C, I, mask));
  return cudaGetLastError();
}

}  // namespace tg
