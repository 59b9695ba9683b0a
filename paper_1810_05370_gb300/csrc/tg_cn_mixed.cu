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
        // s = sum over faces of a (x_n - x_c), one compensated sum of double-FP32 products
        CSum acc = {0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < 6; ++q) cs_fma(acc, f[q], df_sub_near(df_of(x[nbr[q]]), xc));
        float2* rhs2 = reinterpret_cast<float2*>(C.p[r]);
        Df rhs, res;
        if (init) {
          const Df s = cs_value(acc);
          rhs = df_add(xc, s);
          rhs2[c] = make_float2(rhs.hi, rhs.lo);
          res = df_add(df_sub(rhs, xc), s);
        } else {
          rhs = df_of(rhs2[c]);
          cs_add(acc, df_sub(rhs, xc));   // res = (rhs - x) + s
          res = cs_value(acc);
        }
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

// The operator of an inner iteration preconditioned by the polynomial, with the p-update
// fused: at iteration k, p = z + beta p_old (p = z at a solve's first iteration) is formed
// from z and the previous direction (buffer (k & 1) ? palt : p), written at the node into the
// other buffer, and q = A p, <p, q> follow (A p as in k_cn32_matvec), for the solves r0, r1
// (-1: none).  A block is MV_X x MV_Y columns marching up a chunk of zc planes: lanes
// 1 .. MV_X - 2 of rows 1 .. MV_Y - 2 are its output columns and the outer lanes and rows
// hold the neighbouring columns (periodically wrapped), so each thread forms p of its own
// column only, one plane ahead from loads issued a step earlier, and takes the x neighbours'
// p and x face from the neighbouring lanes (shuffles), the y neighbours' p and y face from the
// rows above and below through shared memory (two planes, alternating; one barrier per
// plane), and the z neighbours' from its registers.  Offsets are 32-bit (nvox < 2^31).
constexpr int MV_X = 32, MV_Y = 16, MV_OX = MV_X - 2, MV_OY = MV_Y - 2;
constexpr int MV_CELLS = MV_X * MV_Y;

__global__ void __launch_bounds__(MV_CELLS, 2) k_cn32_matvec_neu(Geo G, Cn32 I, int r0, int r1,
                                                                 int zc) {
  const bool run0 = r0 >= 0 && I.S[r0].status == CG_RUNNING;
  const bool run1 = r1 >= 0 && I.S[r1].status == CG_RUNNING;
  if (!run0 && !run1) return;
  const bool run[2] = {run0, run1};
  // a solve that does not run reads the other one's vectors (nothing of it is stored)
  const int ld[2] = {run0 ? r0 : r1, run1 ? r1 : r0};
  float beta[2];
  bool first[2];
  const float* zin[2];
  const float* pin[2];
  float* pout[2];
  float* qout[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int it = I.S[ld[q]].it;
    first[q] = it == 0;
    beta[q] = first[q] ? 0.0f : (float)I.S[ld[q]].beta;
    zin[q] = I.z[ld[q]];
    pin[q] = (it & 1) ? I.palt[ld[q]] : I.p[ld[q]];
    pout[q] = (it & 1) ? I.p[ld[q]] : I.palt[ld[q]];
    qout[q] = I.q[ld[q]];
  }
  __shared__ float sp[2][2][MV_CELLS];   // p of the step's plane: [step parity][solve][cell]
  __shared__ float sfy[2][MV_CELLS];     // the y face above each cell, same planes
  __shared__ double red[MV_CELLS / 32][2];
  __shared__ bool last;
  const int tx = threadIdx.x, ty = threadIdx.y, cell = ty * MV_X + tx;
  const int iu = blockIdx.x * MV_OX - 1 + tx, ju = blockIdx.y * MV_OY - 1 + ty;   // unwrapped
  const int gx = ((iu % G.nx) + G.nx) % G.nx, gy = ((ju % G.ny) + G.ny) % G.ny;
  const unsigned nxy = (unsigned)(G.nx * G.ny), nvox = nxy * (unsigned)G.nz;
  const unsigned col = (unsigned)(gy * G.nx + gx);
  const bool out = tx >= 1 && tx < MV_X - 1 && ty >= 1 && ty < MV_Y - 1 && iu < G.nx && ju < G.ny;
  const int cn = ty < MV_Y - 1 ? cell + MV_X : cell, cs = ty > 0 ? cell - MV_X : cell;
  const int k0 = blockIdx.z * zc, k1 = min(G.nz, k0 + zc);
  auto poff = [&](int k) {
    return (unsigned)(k < 0 ? k + G.nz : (k >= G.nz ? k - G.nz : k)) * nxy;
  };
  const float* const kfx = I.Kf[0];
  const float* const kfy = I.Kf[1];
  const float* const kfz = I.Kf[2];
  // p of the planes k0 - 1 and k0, z and p_old of plane k0 + 1, the faces of plane k0 and the
  // z face below it
  float pm[2], pc[2], nzv[2], npv[2];
  {
    const unsigned om = poff(k0 - 1) + col, o0 = poff(k0) + col, o1 = poff(k0 + 1) + col;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float zm = __ldg(zin[q] + om), z0 = __ldg(zin[q] + o0);
      pm[q] = first[q] ? zm : zm + beta[q] * __ldg(pin[q] + om);
      pc[q] = first[q] ? z0 : z0 + beta[q] * __ldg(pin[q] + o0);
      nzv[q] = __ldg(zin[q] + o1);
      npv[q] = first[q] ? 0.0f : __ldg(pin[q] + o1);
    }
  }
  float fzm = __ldg(kfz + poff(k0 - 1) + col);
  float fx = __ldg(kfx + poff(k0) + col), fy = __ldg(kfy + poff(k0) + col);
  float fz = __ldg(kfz + poff(k0) + col);
  float part[2] = {0.0f, 0.0f};
  unsigned ob = poff(k0), o1p = poff(k0 + 1), o2p = poff(k0 + 2);   // planes k, k + 1, k + 2
  int buf = 0;
  for (int k = k0; k < k1; ++k) {
    float pp[2];   // p of plane k + 1
#pragma unroll
    for (int q = 0; q < 2; ++q) pp[q] = first[q] ? nzv[q] : nzv[q] + beta[q] * npv[q];
    float nfx = 0.0f, nfy = 0.0f, nfz = 0.0f;
    if (k + 1 < k1) {   // the next step's loads: z, p_old of plane k + 2, faces of plane k + 1
      const unsigned o2 = o2p + col, o1 = o1p + col;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        nzv[q] = __ldg(zin[q] + o2);
        npv[q] = first[q] ? 0.0f : __ldg(pin[q] + o2);
      }
      nfx = __ldg(kfx + o1);
      nfy = __ldg(kfy + o1);
      nfz = __ldg(kfz + o1);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) sp[buf][q][cell] = pc[q];
    sfy[buf][cell] = fy;
    __syncthreads();
    const float fxm = __shfl_up_sync(0xffffffffu, fx, 1);
    const float fym = sfy[buf][cs];
    const float d = 1.0f + ((fx + fxm) + (fy + fym) + (fz + fzm));
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float pxp = __shfl_down_sync(0xffffffffu, pc[q], 1);
      const float pxm = __shfl_up_sync(0xffffffffu, pc[q], 1);
      const float pyp = sp[buf][q][cn], pym = sp[buf][q][cs];
      const float qv = d * pc[q] - (fx * pxp + fxm * pxm + fy * pyp + fym * pym + fz * pp[q] +
                                    fzm * pm[q]);
      if (out && run[q]) {
        pout[q][ob + col] = pc[q];
        qout[q][ob + col] = qv;
        part[q] += pc[q] * qv;
      }
      pm[q] = pc[q];
      pc[q] = pp[q];
    }
    fzm = fz;
    fx = nfx;
    fy = nfy;
    fz = nfz;
    ob = o1p;
    o1p = o2p;
    o2p += nxy;
    if (o2p == nvox) o2p = 0u;
    buf ^= 1;
  }

  // <p, q> per solve: warps, then the block's warps in order, then the blocks in order by the
  // last block to finish
  const int lane = cell & 31, warp = cell >> 5, nb = gridDim.x * gridDim.y * gridDim.z;
  const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double v = warp_sum((double)part[q]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (cell == 0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      double v = 0.0;
      for (int w = 0; w < MV_CELLS / 32; ++w) v += red[w][q];
      I.partial[2 * (size_t)b + q] = v;
    }
    __threadfence();
    last = atomicAdd(I.counter, 1u) == (unsigned int)(nb - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot[2] = {0.0, 0.0};
  for (int k = cell; k < nb; k += MV_CELLS) {
#pragma unroll
    for (int q = 0; q < 2; ++q) tot[q] += __ldcg(I.partial + 2 * (size_t)k + q);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double v = warp_sum(tot[q]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (cell == 0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      double v = 0.0;
      for (int w = 0; w < MV_CELLS / 32; ++w) v += red[w][q];
      if (run[q]) {
        I.S[ld[q]].pq = v;
        I.S[ld[q]].alpha = I.S[ld[q]].rz / v;
      }
    }
    *I.counter = 0u;
  }
}

// e += alpha p, r -= alpha q; <r, D^{-1} r>, <r, r>.  float4 groups g = g0, g0 + gs, ... of an
// n-voxel system plus the scalar tail n - n % 4 .. n (block 0); a group's products are summed
// in FP32, groups in FP64.  With the polynomial preconditioner (NEU) only <r, r> is formed:
// the next iteration's preconditioner kernel forms <r, z> and beta.
template <bool NEU>
__global__ void __launch_bounds__(NT) k_cn32_update(long long n, Cn32 I) {
  bool act[3];
  if (!active3(I, act)) return;
  float alpha[3];
  const float* pcur[3];   // the search direction this iteration's operator kernel used
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    alpha[r] = (float)I.S[r].alpha;
    pcur[r] = (NEU && !(I.S[r].it & 1)) ? I.palt[r] : I.p[r];
  }
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const long long gs = (long long)gridDim.x * blockDim.x, ng = n / 4;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < ng; v += gs) {
    const float4 d = NEU ? float4{0.0f, 0.0f, 0.0f, 0.0f}
                         : __ldg(reinterpret_cast<const float4*>(I.dinv) + v);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!act[r]) continue;
      float4* e4 = reinterpret_cast<float4*>(I.e[r]) + v;
      float4* r4 = reinterpret_cast<float4*>(I.r[r]) + v;
      const float4 p = reinterpret_cast<const float4*>(pcur[r])[v];
      const float4 q = reinterpret_cast<const float4*>(I.q[r])[v];
      float4 e = *e4, x = *r4;
      const float a = alpha[r];
      e.x += a * p.x; e.y += a * p.y; e.z += a * p.z; e.w += a * p.w;
      x.x -= a * q.x; x.y -= a * q.y; x.z -= a * q.z; x.w -= a * q.w;
      *e4 = e;
      *r4 = x;
      if (!NEU)
        acc[2 * r] += (double)(x.x * (d.x * x.x) + x.y * (d.y * x.y) + x.z * (d.z * x.z) +
                               x.w * (d.w * x.w));
      acc[2 * r + 1] += (double)(x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w);
    }
  }
  if (blockIdx.x == 0) {
    for (long long c = 4 * ng + threadIdx.x; c < n; c += blockDim.x) {
      const float di = NEU ? 0.0f : I.dinv[c];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (!act[r]) continue;
        I.e[r][c] += alpha[r] * pcur[r][c];
        const float res = I.r[r][c] - alpha[r] * I.q[r][c];
        I.r[r][c] = res;
        if (!NEU) acc[2 * r] += (double)(res * (di * res));
        acc[2 * r + 1] += (double)(res * res);
      }
    }
  }
  double out[6];
  if (reduce_last_block<6>(acc, I.partial, I.counter, out) && threadIdx.x == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!act[r]) continue;
      if (NEU)
        cg_after_update_rr(I.S[r], out[2 * r + 1]);
      else
        cg_after_update(I.S[r], out[2 * r], out[2 * r + 1]);
    }
  }
}

// p = z + beta p (p = z on an inner solve's first iteration), float4 groups; z = D^{-1} r
// (Jacobi) or the polynomial preconditioner's output I.z (NEU)
template <bool NEU>
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
    const float4 d = NEU ? float4{0.0f, 0.0f, 0.0f, 0.0f}
                         : __ldg(reinterpret_cast<const float4*>(I.dinv) + v);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!act[r]) continue;
      float4* p4 = reinterpret_cast<float4*>(I.p[r]) + v;
      float4 z;
      if (NEU) {
        z = reinterpret_cast<const float4*>(I.z[r])[v];
      } else {
        const float4 x = reinterpret_cast<const float4*>(I.r[r])[v];
        z = float4{d.x * x.x, d.y * x.y, d.z * x.z, d.w * x.w};
      }
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
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (!act[r]) continue;
        const float z = NEU ? I.z[r][c] : I.dinv[c] * I.r[r][c];
        I.p[r][c] = first[r] ? z : z + beta[r] * I.p[r][c];
      }
    }
  }
}

// ------------------------------------------------------------- polynomial preconditioner
// M r = q(N) D^{-1} r, a cubic in N = D^{-1} (D - A) (the Jacobi splitting A = D - (D - A)).
// (D - A) y at a node is the sum over its six faces of the face coefficient times y at the
// neighbour across it, so the terms y_0 = D^{-1} r, y_{j+1} = D^{-1} (D - A) y_j are three
// Jacobi sweeps, and M r = w (y_0 + y_1) + (y_2 + y_3).
//   * w = 1 is the Neumann series I + N + N^2 + N^3 of A^{-1} = (I - N)^{-1} D^{-1}.
//   * The Chebyshev choice: with B = D^{-1/2} A D^{-1/2}, whose spectrum lies in
//     [1/d_max, 2 - 1/d_max] (Gershgorin, the CN operator being I plus a positive
//     semidefinite part), the cubic q minimising max |1 - x q(x)| there satisfies
//     1 - x q(x) = T_4((1 - x)/delta) / T_4(1/delta), delta = 1 - 1/d_max; written in
//     n = 1 - x it is q = K (1 + n)(1 - delta^2 + n^2), i.e. (scale aside, which CG ignores)
//     w = 1 - delta^2 = (2 d_max - 1) / d_max^2.  It reduces x q(x)'s condition number about
//     16-fold where the Neumann series reduces it 4-fold (the first orders of T_4 and of
//     1 - (1 - x)^4 at the interval's end): 7 instead of 10 inner iterations per solve at
//     256^3 on the oracle's operator of the synthetic brain.
// Both are symmetric positive definite: M = D^{-1/2} q(B) D^{-1/2} with q > 0 on B's spectrum.
//
// The three sweeps run in one pass over memory (temporal blocking).  A block owns an
// NM_X x NM_Y tile of (x, y) columns -- the NM_OX x NM_OY output columns and a halo of
// NM_H = 3 -- and marches up a chunk of z planes: at step t it forms y_0 on plane t over the
// whole tile, y_1 on plane t - 1 one column in from the edge, y_2 on plane t - 2 two columns
// in and y_3 on plane t - 3 over the output columns, whose z = y_0 + y_1 + y_2 + y_3 it
// writes.  A warp is one row of the tile, so a term's x neighbours come from the neighbouring
// lanes (shuffles); its y neighbours from the previous step's shared-memory plane of the term
// below it (two planes per term, alternating); its z neighbours and the column's own faces
// from registers.  The registers of the last four planes form rings indexed by the plane
// modulo 4; the march is unrolled by four so that every ring index is a constant.  One
// barrier per step.  Global memory is read once per plane (r, three faces, D^{-1}) and z
// written once, plus the halo columns, which neighbouring blocks also read (mostly from L2).
// Two solves (slots) share the face reads.  <r, z> of each solve is summed for its CG scalars.
constexpr int NM_X = 32, NM_Y = 16, NM_H = 3;
constexpr int NM_OX = NM_X - 2 * NM_H, NM_OY = NM_Y - 2 * NM_H;
constexpr int NM_CELLS = NM_X * NM_Y;

struct NmTile {
  float2 y[3][2][NM_CELLS];     // terms 0..2 of the two solves: [term][plane parity][cell]
  float ay[4][NM_CELLS];        // y faces of the last four planes (index plane & 3)
  double red[NM_CELLS / 32][2];
  bool last;
};

__global__ void __launch_bounds__(NM_CELLS, 1) k_cn32_neumann(Geo G, Cn32 I, int r0, int r1,
                                                              int zc) {
  const bool run0 = r0 >= 0 && I.S[r0].status == CG_RUNNING;
  const bool run1 = r1 >= 0 && I.S[r1].status == CG_RUNNING;
  if (!run0 && !run1) return;
  // the weight of the first two terms (the last two weigh 1): the degree-3 Chebyshev
  // polynomial on the Jacobi-scaled operator's Gershgorin interval when S0 measured the
  // largest diagonal, else 1 (the Neumann series)
  float wch = 1.0f;
  if (I.dmax) {
    const float dm = *I.dmax;
    if (dm > 1.0f) wch = (2.0f * dm - 1.0f) / (dm * dm);
  }
  __shared__ NmTile T;
  const int tx = threadIdx.x, ty = threadIdx.y, cell = ty * NM_X + tx;
  const int xo = blockIdx.x * NM_OX, yo = blockIdx.y * NM_OY;
  const int gxu = xo - NM_H + tx, gyu = yo - NM_H + ty;   // unwrapped tile coordinates
  const int gx = ((gxu % G.nx) + G.nx) % G.nx, gy = ((gyu % G.ny) + G.ny) % G.ny;
  // 32-bit offsets (the launch checks nvox < 2^31)
  const unsigned nxy = (unsigned)(G.nx * G.ny), nvox = nxy * (unsigned)G.nz;
  const unsigned col = (unsigned)(gy * G.nx + gx);
  // Term j is formed on the rows j .. NM_Y - 1 - j (a warp is a row, so the test is uniform
  // over a warp and the shuffles inside it see every lane).  Its lanes tx < j and
  // tx >= NM_X - j form values from wrapped shuffles that only the same outer lanes of the
  // next term read, never an output column; likewise the terms formed in the first and last
  // steps of the march, from planes whose lower terms do not exist yet, feed only terms of
  // planes outside the output range.
  const bool row1 = ty >= 1 && ty < NM_Y - 1, row2 = ty >= 2 && ty < NM_Y - 2;
  const bool row3 = ty >= 3 && ty < NM_Y - 3;
  const bool out = row3 && tx >= NM_H && tx < NM_X - NM_H && gxu < G.nx && gyu < G.ny;
  const int k0 = blockIdx.z * zc, k1 = min(G.nz, k0 + zc);
  const bool run[2] = {run0, run1};
  // a solve that does not run reads the other one's residual (its z is neither stored nor
  // summed), so the loads need no test
  const int ld[2] = {run0 ? r0 : r1, run1 ? r1 : r0};
  const float* const rsrc[2] = {I.r[ld[0]], I.r[ld[1]]};
  float* const zdst[2] = {I.z[ld[0]], I.z[ld[1]]};
  const float* const kfx = I.Kf[0];
  const float* const kfy = I.Kf[1];
  const float* const kfz = I.Kf[2];
  const float* const dsrc = I.dinv;
  // rings over the last four planes, slot = (plane - tb) & 3 with tb = k0 - NM_H; the shared
  // planes of the terms alternate with (plane - tb) & 1, the y faces with (plane - tb) & 3
  float y0[4][2], y1[4][2], y2[4][2], rr[4][2], lz[4][2];   // lz: a_z(k-1) y_2(k-1) of plane k
  float ax[4], ay[4], az[4], di[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
#pragma unroll
    for (int q = 0; q < 2; ++q) y0[m][q] = y1[m][q] = y2[m][q] = rr[m][q] = lz[m][q] = 0.0f;
    ax[m] = ay[m] = az[m] = di[m] = 0.0f;
  }
  float acc[2] = {0.0f, 0.0f};
  // planes t + 1 and t + 2 in flight: the loads of plane t + 2 are issued at step t into the
  // set that plane t came from (set = (plane - tb) & 1)
  float pr[2][2], pax[2], pay[2], paz[2], pdi[2];
  const int tb = k0 - NM_H;
  const int nsteps = (k1 - k0 + 2 * NM_H + 3) & ~3;     // a multiple of 4
  // offsets of the next fetched plane and of the output plane (t - 3), advanced per step
  unsigned fo = (unsigned)(((tb % G.nz) + G.nz) % G.nz) * nxy;
  unsigned zo = (unsigned)k0 * nxy;   // the first output plane (k0 < nz), written at rel = 2 NM_H
  auto fetch = [&](int set) {
    const unsigned o = fo + col;
#pragma unroll
    for (int q = 0; q < 2; ++q) pr[set][q] = __ldg(rsrc[q] + o);
    pax[set] = __ldg(kfx + o);
    pay[set] = __ldg(kfy + o);
    paz[set] = __ldg(kfz + o);
    pdi[set] = __ldg(dsrc + o);
    fo += nxy;
    if (fo == nvox) fo = 0u;
  };
  fetch(0);
  fetch(1);
  // the output of plane t - 3 is kept for the steps whose offset rel = t - tb lies in
  // [2 NM_H, k1 - k0 + 2 NM_H - 1]
  const int rel_end = k1 - k0 + 2 * NM_H - 1;
  for (int m4 = 0; m4 < nsteps; m4 += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int rel = m4 + u;
      const int s0 = u, s1 = (u + 3) & 3, s2 = (u + 2) & 3, s3 = (u + 1) & 3;
      const int p0 = u & 1, p1 = (u + 1) & 1;   // parities of planes t, t - 1 (t - 2: p0, ...)
      const int ps = u & 1;
#pragma unroll
      for (int q = 0; q < 2; ++q) rr[s0][q] = pr[ps][q];
      ax[s0] = pax[ps];
      ay[s0] = pay[ps];
      az[s0] = paz[ps];
      di[s0] = pdi[ps];
      if (rel + 2 < nsteps) fetch(ps);
      // term 0 on plane t, the whole tile
#pragma unroll
      for (int q = 0; q < 2; ++q) y0[s0][q] = di[s0] * rr[s0][q];
      T.y[0][p0][cell] = make_float2(y0[s0][0], y0[s0][1]);
      T.ay[s0][cell] = ay[s0];
      // term 1 on plane t - 1
      if (row1) {
        const float axm = __shfl_up_sync(0xffffffffu, ax[s1], 1);
        float yp[2], ym[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          yp[q] = __shfl_down_sync(0xffffffffu, y0[s1][q], 1);
          ym[q] = __shfl_up_sync(0xffffffffu, y0[s1][q], 1);
        }
        const float aym = T.ay[s1][cell - NM_X];
        const float2 Yp = T.y[0][p1][cell + NM_X], Ym = T.y[0][p1][cell - NM_X];
        const float yn[2] = {Yp.x, Yp.y}, ys[2] = {Ym.x, Ym.y};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float ha = ax[s1] * yp[q] + axm * ym[q] + az[s1] * y0[s0][q];
          const float hb = ay[s1] * yn[q] + aym * ys[q] + az[s2] * y0[s2][q];
          y1[s1][q] = di[s1] * (ha + hb);
        }
        T.y[1][p1][cell] = make_float2(y1[s1][0], y1[s1][1]);
      }
      // term 2 on plane t - 2; the z-lower term a_z(k) y_2(k) of the plane above it
      if (row2) {
        const float axm = __shfl_up_sync(0xffffffffu, ax[s2], 1);
        float yp[2], ym[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          yp[q] = __shfl_down_sync(0xffffffffu, y1[s2][q], 1);
          ym[q] = __shfl_up_sync(0xffffffffu, y1[s2][q], 1);
        }
        const float aym = T.ay[s2][cell - NM_X];
        const float2 Yp = T.y[1][p0][cell + NM_X], Ym = T.y[1][p0][cell - NM_X];
        const float yn[2] = {Yp.x, Yp.y}, ys[2] = {Ym.x, Ym.y};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float ha = ax[s2] * yp[q] + axm * ym[q] + az[s2] * y1[s1][q];
          const float hb = ay[s2] * yn[q] + aym * ys[q] + az[s3] * y1[s3][q];
          y2[s2][q] = di[s2] * (ha + hb);
          lz[s1][q] = az[s2] * y2[s2][q];   // for term 3 on plane t - 1 (two steps on)
        }
        T.y[2][p0][cell] = make_float2(y2[s2][0], y2[s2][1]);
      }
      // term 3 on plane t - 3, and the output there
      if (row3) {
        const float axm = __shfl_up_sync(0xffffffffu, ax[s3], 1);
        float yp[2], ym[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          yp[q] = __shfl_down_sync(0xffffffffu, y2[s3][q], 1);
          ym[q] = __shfl_up_sync(0xffffffffu, y2[s3][q], 1);
        }
        const float aym = T.ay[s3][cell - NM_X];
        const float2 Yp = T.y[2][p1][cell + NM_X], Ym = T.y[2][p1][cell - NM_X];
        const float yn[2] = {Yp.x, Yp.y}, ys[2] = {Ym.x, Ym.y};
        if (out && rel >= 2 * NM_H && rel <= rel_end) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const float ha = ax[s3] * yp[q] + axm * ym[q] + az[s3] * y2[s2][q];
            const float hb = ay[s3] * yn[q] + aym * ys[q] + lz[s3][q];
            const float y3 = di[s3] * (ha + hb);
            const float z = wch * (y0[s3][q] + y1[s3][q]) + (y2[s3][q] + y3);
            if (run[q]) {
              zdst[q][zo + col] = z;
              acc[q] += rr[s3][q] * z;
            }
          }
        }
      }
      if (rel >= 2 * NM_H) {
        zo += nxy;
        if (zo == nvox) zo = 0u;
      }
      __syncthreads();
    }
  }

  // <r, z> per solve: warps, then the block's warps in order, then the blocks in order by the
  // last block to finish
  const int lane = cell & 31, warp = cell >> 5, nb = gridDim.x * gridDim.y * gridDim.z;
  const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double v = warp_sum((double)acc[q]);
    if (lane == 0) T.red[warp][q] = v;
  }
  __syncthreads();
  if (cell == 0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      double v = 0.0;
      for (int w = 0; w < NM_CELLS / 32; ++w) v += T.red[w][q];
      I.partial[2 * (size_t)b + q] = v;
    }
    __threadfence();
    T.last = atomicAdd(I.counter, 1u) == (unsigned int)(nb - 1);
  }
  __syncthreads();
  if (!T.last) return;
  __threadfence();
  double tot[2] = {0.0, 0.0};
  for (int k = cell; k < nb; k += NM_CELLS) {
#pragma unroll
    for (int q = 0; q < 2; ++q) tot[q] += __ldcg(I.partial + 2 * (size_t)k + q);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double v = warp_sum(tot[q]);
    if (lane == 0) T.red[warp][q] = v;
  }
  __syncthreads();
  if (cell == 0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      double v = 0.0;
      for (int w = 0; w < NM_CELLS / 32; ++w) v += T.red[w][q];
      if (run[q]) cg_after_precond(I.S[ld[q]], v);
    }
    *I.counter = 0u;
  }
}

// x += e in FP64 for the solves in the mask (e = 0 for those that did not run this sweep)
__global__ void __launch_bounds__(NT) k_cn_ir_correct(long long n, Cn3 C, Cn32 I, int mask) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!((mask >> r) & 1)) continue;
      const double x = C.x[r][c] + f64_of(I.e[r][c]);
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

// one inner iteration of the FP32 solves: the first iteration of a sweep forms p from the
// (preconditioned) residual before the operator
cudaError_t launch_cn32_iter(const Geo& G, const Cn32& I, cudaStream_t st, int r0, int r1,
                             long long partial_capacity) {
  if (I.z[0] == nullptr && I.z[1] == nullptr && I.z[2] == nullptr) {
    TG_TIMED(K_CN32_PUPDATE, st, k_cn32_pupdate<false><<<flat_blocks(G), NT, 0, st>>>(G.nvox, I));
    TG_TIMED(K_CN32_MATVEC, st, k_cn32_matvec<<<G.grid, dim3(BX, BY), 0, st>>>(G, I));
    TG_TIMED(K_CN32_UPDATE, st, k_cn32_update<false><<<flat_blocks(G), NT, 0, st>>>(G.nvox, I));
    return cudaGetLastError();
  }
  // z chunk: 32 planes, more while the blocks' two partial sums would not fit the buffer
  const long long gx = (G.nx + NM_OX - 1) / NM_OX, gy = (G.ny + NM_OY - 1) / NM_OY;
  int zc = 32;
  while (zc < G.nz && gx * gy * ((G.nz + zc - 1) / zc) * 2 > partial_capacity) zc *= 2;
  zc = zc < G.nz ? zc : G.nz;
  const long long gz = (G.nz + zc - 1) / zc;
  if (gx * gy * gz * 2 > partial_capacity || r0 < 0) return cudaErrorInvalidValue;
  if (G.nvox >= (1LL << 31)) return cudaErrorInvalidValue;   // 32-bit offsets below
  TG_TIMED(K_CN32_NEUMANN, st,
           k_cn32_neumann<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), dim3(NM_X, NM_Y), 0,
                            st>>>(G, I, r0, r1, zc));
  // the operator's grid: about as many blocks as the standard one, each block's two sums in
  // the partial buffer
  const long long mgx = (G.nx + MV_OX - 1) / MV_OX, mgy = (G.ny + MV_OY - 1) / MV_OY;
  long long mgz = (G.nblocks + mgx * mgy - 1) / (mgx * mgy);
  mgz = std::max(1LL, std::min(mgz, (long long)G.nz));
  int mzc = (int)((G.nz + mgz - 1) / mgz);
  while (mzc < G.nz && mgx * mgy * ((G.nz + mzc - 1) / mzc) * 2 > partial_capacity) mzc *= 2;
  mzc = mzc < G.nz ? mzc : G.nz;
  mgz = (G.nz + mzc - 1) / mzc;
  if (mgx * mgy * mgz * 2 > partial_capacity) return cudaErrorInvalidValue;
  TG_TIMED(K_CN32_MATVEC, st,
           k_cn32_matvec_neu<<<dim3((unsigned)mgx, (unsigned)mgy, (unsigned)mgz),
                               dim3(MV_X, MV_Y), 0, st>>>(G, I, r0, r1, mzc));
  TG_TIMED(K_CN32_UPDATE, st, k_cn32_update<true><<<flat_blocks(G), NT, 0, st>>>(G.nvox, I));
  return cudaGetLastError();
}

cudaError_t launch_cn_ir_correct(const Geo& G, const Cn3& C, const Cn32& I, int mask,
                                 cudaStream_t st) {
  TG_TIMED(K_CN_IR_CORRECT, st, k_cn_ir_correct<<<flat_blocks(G), NT, 0, st>>>(G.nvox, C, I, mask));
  return cudaGetLastError();
}

}  // namespace tg
