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

// The operator kernel is tiled: a block owns a 32 x 8 column of nodes and marches it through
// its z range, keeping three planes (k-1, k, k+1) of the search direction and of the node
// mu, lambda in shared memory with a one-node halo (34 x 10 per plane).  The search direction
// is formed while the plane is staged, p_new = D^{-1} r + beta p_old (the CG p-update of the
// previous iteration), written once per node and double-buffered so that neighbouring blocks
// still read p_old.  Each node is then read from global memory about 1.4 times (halo and
// z-overlap) instead of about 60 times.
constexpr int HX = BX + 2;
constexpr int HY = BY + 2;
constexpr int HXY = HX * HY;

struct Tile32 {
  float p[3][3][HXY];  // [plane slot][component][node]
  float mu[3][HXY];
  float la[3][HXY];
};

struct Consts32 {
  float ih2[3];
  float sc[3][3];
};

__device__ __forceinline__ bool running(const CgScal* S) { return S->status == CG_RUNNING; }

// Pointers to the centre node of one thread in each staged plane: p (3 components), mu and
// lambda of planes k-1, k, k+1; neighbours are then constant offsets (+-1, +-HX).
struct Cell {
  const float* p[3][3];   // [plane -1, 0, +1][component]
  const float* mu[3];
  const float* la[3];
};

__device__ __forceinline__ float tp(const Tile32&, const Cell& t, int a, int ox, int oy, int oz) {
  return t.p[oz + 1][a][ox + oy * HX];
}
__device__ __forceinline__ float tmu(const Tile32&, const Cell& t, int ox, int oy, int oz) {
  return t.mu[oz + 1][ox + oy * HX];
}
__device__ __forceinline__ float tla(const Tile32&, const Cell& t, int ox, int oy, int oz) {
  return t.la[oz + 1][ox + oy * HX];
}

struct Fac32 {
  float Fp[3], Fm[3];   // (lambda + 2 mu) faces / h_d^2 at +e_d and -e_d
  float Gp[3], Gm[3];   // mu faces / h_d^2
  float mup[3], mum[3]; // node mu at c +/- e_d
  float lap[3], lam[3]; // node lambda at c +/- e_d
  float eta;
};

__device__ __forceinline__ void tile_fac(const Tile32& T, const Cell& t, const float ih2[3],
                                         float eta, Fac32& f) {
  const float muc = tmu(T, t, 0, 0, 0), lac = tla(T, t, 0, 0, 0);
  f.eta = eta;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int ox = d == 0, oy = d == 1, oz = d == 2;
    f.mup[d] = tmu(T, t, ox, oy, oz);
    f.mum[d] = tmu(T, t, -ox, -oy, -oz);
    f.lap[d] = tla(T, t, ox, oy, oz);
    f.lam[d] = tla(T, t, -ox, -oy, -oz);
    const float gp = 0.5f * (muc + f.mup[d]), gm = 0.5f * (f.mum[d] + muc);
    const float lp = 0.5f * (lac + f.lap[d]), lm = 0.5f * (f.lam[d] + lac);
    f.Gp[d] = gp * ih2[d];
    f.Gm[d] = gm * ih2[d];
    f.Fp[d] = (lp + 2.0f * gp) * ih2[d];
    f.Fm[d] = (lm + 2.0f * gm) * ih2[d];
  }
}

// component A of (eta I - L_h) p at the centre node, all operands from the tile
template <int A>
__device__ __forceinline__ float row_tile(const Tile32& T, const Cell& t, const Fac32& f,
                                          const float sc[3][3]) {
  constexpr int D1 = (A + 1) % 3, D2 = (A + 2) % 3;
  float diag = f.eta, off = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int ox = d == 0, oy = d == 1, oz = d == 2;
    const float cp = (d == A) ? f.Fp[d] : f.Gp[d];
    const float cm = (d == A) ? f.Fm[d] : f.Gm[d];
    diag += cp + cm;
    off += cp * tp(T, t, A, ox, oy, oz) + cm * tp(T, t, A, -ox, -oy, -oz);
  }
  float v = diag * tp(T, t, A, 0, 0, 0) - off;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int D = k == 0 ? D1 : D2;
    // offsets of c + sa e_A + sd e_D
    const int ax = A == 0, ay = A == 1, az = A == 2;
    const int dx = D == 0, dy = D == 1, dz = D == 2;
    const float epp = tp(T, t, D, ax + dx, ay + dy, az + dz);
    const float epm = tp(T, t, D, -ax + dx, -ay + dy, -az + dz);
    const float emp = tp(T, t, D, ax - dx, ay - dy, az - dz);
    const float emm = tp(T, t, D, -ax - dx, -ay - dy, -az - dz);
    const float mixed = f.mup[D] * (epp - epm) - f.mum[D] * (emp - emm) +
                        f.lap[A] * (epp - emp) - f.lam[A] * (epm - emm);
    v -= sc[A][D] * mixed;
  }
  return v;
}

__global__ void __launch_bounds__(NT) k_elas32_matvec(Geo G, Consts32 K, Elas32 I) {
  if (!running(I.S)) return;
  const int it = I.S->it;
  const bool first = it == 0;                 // p = D^{-1} r (the old p is undefined)
  const float beta = first ? 0.0f : (float)I.S->beta;
  const float* __restrict__ po[3] = {I.p[it & 1][0], I.p[it & 1][1], I.p[it & 1][2]};
  float* pn[3] = {I.p[(it & 1) ^ 1][0], I.p[(it & 1) ^ 1][1], I.p[(it & 1) ^ 1][2]};

  __shared__ Tile32 T;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
  const int i = i0 + tx, j = j0 + ty;
  const bool on = (i < G.nx) && (j < G.ny);
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);

  // the (at most two) halo-tile nodes this thread stages: tile slot tid and tid + NT; their
  // wrapped (x, y) offsets (full modulo: a tile may be wider than the grid)
  auto wrapped = [&](int s) {
    int gi = (i0 - 1 + s % HX) % G.nx, gj = (j0 - 1 + s / HX) % G.ny;
    gi = gi < 0 ? gi + G.nx : gi;
    gj = gj < 0 ? gj + G.ny : gj;
    return (long long)gj * G.nx + gi;
  };
  const int hs1 = tid + NT;
  const bool two = hs1 < HXY;
  const long long ho0 = wrapped(tid);
  const long long ho1 = two ? wrapped(hs1) : 0;

  // a staged node: the three components of p_new and the node mu, lambda
  struct Staged {
    float p[3], mu, la;
  };
  auto fetch = [&](long long g, Staged& v) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float z = __ldg(I.dinv[a] + g) * __ldg(I.r[a] + g);
      v.p[a] = first ? z : z + beta * __ldg(po[a] + g);
    }
    v.mu = __ldg(I.mu + g);
    v.la = __ldg(I.lam + g);
  };
  auto put = [&](const Staged& v, int slot, int s) {
#pragma unroll
    for (int a = 0; a < 3; ++a) T.p[slot][a][s] = v.p[a];
    T.mu[slot][s] = v.mu;
    T.la[slot][s] = v.la;
  };
  auto plane_offset = [&](int kk) {
    const int kw = kk < 0 ? kk + G.nz : (kk >= G.nz ? kk - G.nz : kk);
    return (long long)kw * G.nxy;
  };
  // registers carry plane k+2 while plane k is computed (loads overlap the arithmetic)
  Staged r0, r1;
  {
    long long zo = plane_offset(k0 - 1);
    fetch(zo + ho0, r0);
    if (two) fetch(zo + ho1, r1);
    put(r0, 0, tid);
    if (two) put(r1, 0, hs1);
    zo = plane_offset(k0);
    fetch(zo + ho0, r0);
    if (two) fetch(zo + ho1, r1);
    put(r0, 1, tid);
    if (two) put(r1, 1, hs1);
    zo = plane_offset(k0 + 1);
    fetch(zo + ho0, r0);
    if (two) fetch(zo + ho1, r1);
    put(r0, 2, tid);
    if (two) put(r1, 2, hs1);
  }

  float part = 0.0f;
  const int ci = (ty + 1) * HX + (tx + 1);
  int s0 = 0, s1 = 1, s2 = 2;            // slots of planes k-1, k, k+1
  for (int k = k0; k < k1; ++k) {
    Cell t;
    const int sl[3] = {s0, s1, s2};
#pragma unroll
    for (int o = 0; o < 3; ++o) {
#pragma unroll
      for (int a = 0; a < 3; ++a) t.p[o][a] = &T.p[sl[o]][a][ci];
      t.mu[o] = &T.mu[sl[o]][ci];
      t.la[o] = &T.la[sl[o]][ci];
    }
    const bool more = k + 1 < k1;
    if (more) {                         // issue the loads of plane k+2
      const long long zo = plane_offset(k + 2);
      fetch(zo + ho0, r0);
      if (two) fetch(zo + ho1, r1);
    }
    __syncthreads();
    if (on) {
      const long long c = (long long)k * G.nxy + (long long)j * G.nx + i;
      Fac32 f;
      tile_fac(T, t, K.ih2, __ldg(I.eta + c), f);
      const float q0 = row_tile<0>(T, t, f, K.sc);
      const float q1 = row_tile<1>(T, t, f, K.sc);
      const float q2 = row_tile<2>(T, t, f, K.sc);
      const float p0 = tp(T, t, 0, 0, 0, 0), p1 = tp(T, t, 1, 0, 0, 0), p2 = tp(T, t, 2, 0, 0, 0);
      pn[0][c] = p0;
      pn[1][c] = p1;
      pn[2][c] = p2;
      I.q[0][c] = q0;
      I.q[1][c] = q1;
      I.q[2][c] = q2;
      part += p0 * q0 + p1 * q1 + p2 * q2;
    }
    __syncthreads();
    if (more) {                         // plane k-1 is free: it becomes plane k+2
      put(r0, s0, tid);
      if (two) put(r1, s0, hs1);
    }
    const int sf = s0;                  // rotate: (k-1, k, k+1) <- (k, k+1, k+2)
    s0 = s1;
    s1 = s2;
    s2 = sf;
  }
  double acc[1] = {(double)part};
  double out[1];
  if (reduce_last_block<1>(acc, I.partial, I.counter, out) && threadIdx.x == 0 && threadIdx.y == 0) {
    I.S->pq = out[0];
    I.S->alpha = I.S->rz / out[0];
  }
}

// e += alpha p, r -= alpha q with the p this iteration's operator kernel wrote; then
// <r, D^{-1} r> and <r, r>.  Flat over voxels, four at a time (128-bit accesses); the twelve
// products of one group are summed in FP32 and accumulated in FP64.
__global__ void __launch_bounds__(NT) k_elas32_update(long long n, Elas32 I) {
  if (!running(I.S)) return;
  const float alpha = (float)I.S->alpha;
  const int pb = (I.S->it & 1) ^ 1;
  const long long n4 = n / 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double drz = 0.0, drr = 0.0;
  for (long long v = t0; v < n4; v += stride) {
    float prz = 0.0f, prr = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float4* e4 = reinterpret_cast<float4*>(I.e[a]) + v;
      float4* r4 = reinterpret_cast<float4*>(I.r[a]) + v;
      const float4 p = __ldg(reinterpret_cast<const float4*>(I.p[pb][a]) + v);
      const float4 q = __ldg(reinterpret_cast<const float4*>(I.q[a]) + v);
      const float4 d = __ldg(reinterpret_cast<const float4*>(I.dinv[a]) + v);
      float4 e = *e4, r = *r4;
      e.x += alpha * p.x; e.y += alpha * p.y; e.z += alpha * p.z; e.w += alpha * p.w;
      r.x -= alpha * q.x; r.y -= alpha * q.y; r.z -= alpha * q.z; r.w -= alpha * q.w;
      *e4 = e;
      *r4 = r;
      prz += r.x * (d.x * r.x) + r.y * (d.y * r.y) + r.z * (d.z * r.z) + r.w * (d.w * r.w);
      prr += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
    }
    drz += (double)prz;
    drr += (double)prr;
  }
  for (long long c = 4 * n4 + t0; c < n; c += stride) {   // tail when n is not a multiple of 4
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      I.e[a][c] += alpha * I.p[pb][a][c];
      const float res = I.r[a][c] - alpha * I.q[a][c];
      I.r[a][c] = res;
      drz += (double)(res * (I.dinv[a][c] * res));
      drr += (double)(res * res);
    }
  }
  double acc[2] = {drz, drr};
  double out[2];
  if (reduce_last_block<2>(acc, I.partial, I.counter, out) && threadIdx.x == 0 && threadIdx.y == 0)
    cg_after_update(*I.S, out[0], out[1]);
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

// flat launches that reduce: never more blocks than the partial-sum buffer holds
static int reduce_blocks(const Geo& G, long long items) {
  long long b = (items + NT - 1) / NT;
  b = b < 8LL * 152 ? b : 8LL * 152;
  b = b < G.nblocks ? b : G.nblocks;
  return (int)(b > 0 ? b : 1);
}

cudaError_t launch_elas32_update(const Geo& G, const Elas32& I, cudaStream_t st) {
  k_elas32_update<<<reduce_blocks(G, (G.nvox + 3) / 4), NT, 0, st>>>(G.nvox, I);
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
