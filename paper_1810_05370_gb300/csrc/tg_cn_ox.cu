// tg_cn_ox.cu -- the oxygen Crank-Nicolson solve of S2 in the mixed precision, in
// double-FP32 arithmetic.
//
// Section 3: (1 - dt/2 D) o+ = (1 + dt/2 D) o by Jacobi-preconditioned CG from o.  The
// necrosis rate of Eq. e:death switches with a smoothed Heaviside of slope 2/eps_H = 200 in
// o, so two solvers that stop at different points of the same tolerance leave necrotic fields
// measurably apart; the oxygen solve of the mixed precision therefore takes the FP64 path's
// CG iterates themselves (same start, same alpha and beta, same stopping test), not a refined
// FP32 solve.  The iterates x, r, p, q live as (hi, lo) FP32 pairs and every vector operation is
// an error-free double-FP32 operation (about 48 significant bits) on the FP32 units, which
// this GPU runs 64 times faster than its FP64 units; a thread sums its voxels' dot products in
// double-FP32, threads and blocks in FP64, in a fixed order.  CG scalars stay FP64.
//
// Kernels, one solve:  prep (diagonal and inverse pairs from the face pairs, x = o as pairs),
// init (rhs = x + s, r = 2 s with s = dt/2 D_h x, p = D^{-1} r and the three norms), then per
// iteration matvec (q = A p, <p, q>, alpha), update (x, r, <r, D^{-1} r>, <r, r>, beta and the
// test) and pupdate (p = D^{-1} r + beta p), and finish (o = x).
#include "tg_tiles.cuh"

namespace tg {
namespace {

__device__ __forceinline__ Df ld_df(const float2* a, long long i) { return df_of(a[i]); }
__device__ __forceinline__ void st_df(float2* a, long long i, Df v) {
  a[i] = make_float2(v.hi, v.lo);
}
__device__ __forceinline__ Df df_scale2(Df x) { return {2.0f * x.hi, 2.0f * x.lo}; }   // exact

// 1 / d to double-FP32 accuracy: FP32 reciprocal of the leading part, then one Newton step
// y + y (1 - d y) with the residual formed in double-FP32 (the Newton-Raphson iteration for
// the reciprocal roughly doubles the correct bits per step)
__device__ __forceinline__ Df df_recip(Df d) {
  const Df y = {1.0f / d.hi, 0.0f};
  const Df e = df_sub(Df{1.0f, 0.0f}, df_mul(d, y));
  return df_add(y, df_mul(y, e));
}

template <int NV>
__device__ __forceinline__ void df_acc(Df (&acc)[NV], int q, Df v) { acc[q] = df_add(acc[q], v); }

// the six faces of node c (pairs): +x, -x, +y, -y, +z, -z
struct FacesDf {
  Df xp, xm, yp, ym, zp, zm;
};
__device__ __forceinline__ FacesDf faces_df(const OxDf& O, const Nbr& nb, long long c) {
  FacesDf F;
  F.xp = ld_df(O.Kf[0], c);
  F.xm = ld_df(O.Kf[0], nb.at(-1, 0, 0));
  F.yp = ld_df(O.Kf[1], c);
  F.ym = ld_df(O.Kf[1], nb.at(0, -1, 0));
  F.zp = ld_df(O.Kf[2], c);
  F.zm = ld_df(O.Kf[2], nb.at(0, 0, -1));
  return F;
}

// the sums of a launch: each thread's double-FP32 sums as FP64, reduced over the blocks in order
template <int NV>
__device__ bool ox_reduce(const OxDf& O, const Df (&acc)[NV], double (&out)[NV]) {
  double v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = df_value(acc[q]);
  return reduce_last_block<NV>(v, O.partial, O.counter, out);
}

__global__ void __launch_bounds__(NT) k_ox_prep(Geo G, OxDf O) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    const long long c = nb.at(0, 0, 0);
    const FacesDf F = faces_df(O, nb, c);
    // d = 1 + (xp + xm) + (yp + ym) + (zp + zm), the FP64 diagonal's order
    Df d = df_add(df_add(df_add(Df{1.0f, 0.0f}, df_add(F.xp, F.xm)), df_add(F.yp, F.ym)),
                  df_add(F.zp, F.zm));
    st_df(O.dd, c, d);
    st_df(O.di, c, df_recip(d));
    O.x[c] = df_pack(O.o[c]);
  }
}

// rhs = x + s, r = 2 s (s = sum over faces of a (x_n - x_c)), p = D^{-1} r; (|rhs|^2, |r|^2,
// <r, D^{-1} r>)
__global__ void __launch_bounds__(NT) k_ox_init(Geo G, OxDf O) {
  Df acc[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      const FacesDf F = faces_df(O, nb, c);
      const Df xc = ld_df(O.x, c);
      Df s = df_mul(F.xp, df_sub(ld_df(O.x, nb.at(1, 0, 0)), xc));
      s = df_sub(s, df_mul(F.xm, df_sub(xc, ld_df(O.x, nb.at(-1, 0, 0)))));
      s = df_add(s, df_mul(F.yp, df_sub(ld_df(O.x, nb.at(0, 1, 0)), xc)));
      s = df_sub(s, df_mul(F.ym, df_sub(xc, ld_df(O.x, nb.at(0, -1, 0)))));
      s = df_add(s, df_mul(F.zp, df_sub(ld_df(O.x, nb.at(0, 0, 1)), xc)));
      s = df_sub(s, df_mul(F.zm, df_sub(xc, ld_df(O.x, nb.at(0, 0, -1)))));
      const Df rhs = df_add(xc, s);
      const Df r = df_scale2(s);
      const Df z = df_mul(ld_df(O.di, c), r);
      st_df(O.r, c, r);
      st_df(O.p, c, z);
      df_acc(acc, 0, df_mul(rhs, rhs));
      df_acc(acc, 1, df_mul(r, r));
      df_acc(acc, 2, df_mul(r, z));
    }
  }
  double out[3];
  if (ox_reduce<3>(O, acc, out) && threadIdx.x == 0 && threadIdx.y == 0)
    cg_after_init(*O.S, out[0], out[1], out[2]);
}

// q = d p - sum over faces of a p_n, <p, q>, alpha = rz / <p, q>
__global__ void __launch_bounds__(NT) k_ox_matvec(Geo G, OxDf O) {
  if (O.S->status != CG_RUNNING) return;
  Df acc[1] = {{0.0f, 0.0f}};
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      const FacesDf F = faces_df(O, nb, c);
      const Df pc = ld_df(O.p, c);
      Df off = df_mul(F.xp, ld_df(O.p, nb.at(1, 0, 0)));
      off = df_add(off, df_mul(F.xm, ld_df(O.p, nb.at(-1, 0, 0))));
      off = df_add(off, df_mul(F.yp, ld_df(O.p, nb.at(0, 1, 0))));
      off = df_add(off, df_mul(F.ym, ld_df(O.p, nb.at(0, -1, 0))));
      off = df_add(off, df_mul(F.zp, ld_df(O.p, nb.at(0, 0, 1))));
      off = df_add(off, df_mul(F.zm, ld_df(O.p, nb.at(0, 0, -1))));
      const Df q = df_sub(df_mul(ld_df(O.dd, c), pc), off);
      st_df(O.q, c, q);
      df_acc(acc, 0, df_mul(pc, q));
    }
  }
  double out[1];
  if (ox_reduce<1>(O, acc, out) && threadIdx.x == 0 && threadIdx.y == 0) {
    O.S->pq = out[0];
    O.S->alpha = O.S->rz / out[0];
  }
}

// x += alpha p, r -= alpha q; <r, D^{-1} r>, <r, r>; beta and the convergence test
__global__ void __launch_bounds__(NT) k_ox_update(Geo G, OxDf O) {
  if (O.S->status != CG_RUNNING) return;
  const Df a = df_split(O.S->alpha);
  Df acc[2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const long long c = ((long long)k * G.ny + j) * G.nx + i;
      st_df(O.x, c, df_add(ld_df(O.x, c), df_mul(a, ld_df(O.p, c))));
      const Df r = df_sub(ld_df(O.r, c), df_mul(a, ld_df(O.q, c)));
      st_df(O.r, c, r);
      df_acc(acc, 0, df_mul(r, df_mul(ld_df(O.di, c), r)));
      df_acc(acc, 1, df_mul(r, r));
    }
  }
  double out[2];
  if (ox_reduce<2>(O, acc, out) && threadIdx.x == 0 && threadIdx.y == 0)
    cg_after_update(*O.S, out[0], out[1]);
}

// p = D^{-1} r + beta p
__global__ void __launch_bounds__(NT) k_ox_pupdate(Geo G, OxDf O) {
  if (O.S->status != CG_RUNNING) return;
  const Df b = df_split(O.S->beta);
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    st_df(O.p, c, df_add(df_mul(ld_df(O.di, c), ld_df(O.r, c)), df_mul(b, ld_df(O.p, c))));
  }
}

// o = x (a vanishing right-hand side: o = 0)
__global__ void __launch_bounds__(NT) k_ox_finish(Geo G, OxDf O) {
  const bool zero = O.S->status == CG_ZERO_RHS;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    O.o[c] = zero ? 0.0 : df_value(ld_df(O.x, c));
  }
}

}  // namespace

cudaError_t launch_ox_start(const Geo& G, const OxDf& O, cudaStream_t st) {
  TG_TIMED(K_OX_PREP, st, k_ox_prep<<<G.grid, dim3(BX, BY), 0, st>>>(G, O));
  TG_TIMED(K_OX_INIT, st, k_ox_init<<<G.grid, dim3(BX, BY), 0, st>>>(G, O));
  return cudaGetLastError();
}

cudaError_t launch_ox_iter(const Geo& G, const OxDf& O, cudaStream_t st) {
  TG_TIMED(K_OX_MATVEC, st, k_ox_matvec<<<G.grid, dim3(BX, BY), 0, st>>>(G, O));
  TG_TIMED(K_OX_UPDATE, st, k_ox_update<<<G.grid, dim3(BX, BY), 0, st>>>(G, O));
  TG_TIMED(K_OX_PUPDATE, st, k_ox_pupdate<<<G.grid, dim3(BX, BY), 0, st>>>(G, O));
  return cudaGetLastError();
}

cudaError_t launch_ox_finish(const Geo& G, const OxDf& O, cudaStream_t st) {
  TG_TIMED(K_OX_FINISH, st, k_ox_finish<<<G.grid, dim3(BX, BY), 0, st>>>(G, O));
  return cudaGetLastError();
}

}  // namespace tg
