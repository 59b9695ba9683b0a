// tg_tiles.cuh -- per-tile building blocks of the iterative solvers (Crank-Nicolson diffusion
// CG, FP32 elasticity CG, FP64 refinement) shared by the per-simulation kernels
// (tg_diffusion.cu, tg_mixed.cu) and the batched persistent solvers (tg_batch.cu).
#pragma once

#include <type_traits>

#include "tg_internal.cuh"

namespace tg {

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

// Four plane slots: while planes k-1, k, k+1 are read, plane k+2 is written into the fourth,
// so one barrier per plane suffices.
constexpr int NSLOT = 4;
struct Tile32 {
  float p[NSLOT][3][HXY];  // [plane slot][component][node]
  float mu[NSLOT][HXY];
  float la[NSLOT][HXY];
};


__device__ __forceinline__ bool running(const CgScal* S) { return S->status == CG_RUNNING; }

// Loads of data that other blocks of the same (persistent) kernel may have written go to L2
// (COH = true); otherwise they may use the read-only path.
template <bool COH>
__device__ __forceinline__ float ldf(const float* p) {
  return COH ? __ldcg(p) : __ldg(p);
}
template <bool COH>
__device__ __forceinline__ float4 ldf4(const float4* p) {
  return COH ? __ldcg(p) : __ldg(p);
}
template <bool COH>
__device__ __forceinline__ double ldd(const double* p) {
  return COH ? __ldcg(p) : *p;
}

// CG scalars shared between blocks of a persistent kernel: copy in and out through volatile
// accesses (never from a possibly stale L1 line)
__device__ __forceinline__ CgScal ld_cg(const CgScal* p) {
  const volatile CgScal* v = p;
  CgScal s;
  s.rz = v->rz;
  s.rr = v->rr;
  s.bb = v->bb;
  s.pq = v->pq;
  s.alpha = v->alpha;
  s.beta = v->beta;
  s.rtol = v->rtol;
  s.scale = v->scale;
  s.it = v->it;
  s.maxit = v->maxit;
  s.status = v->status;
  s.pad = v->pad;
  return s;
}
__device__ __forceinline__ void st_cg(CgScal* p, const CgScal& s) {
  volatile CgScal* v = p;
  v->rz = s.rz;
  v->rr = s.rr;
  v->bb = s.bb;
  v->pq = s.pq;
  v->alpha = s.alpha;
  v->beta = s.beta;
  v->rtol = s.rtol;
  v->scale = s.scale;
  v->it = s.it;
  v->maxit = s.maxit;
  v->status = s.status;
  v->pad = s.pad;
}


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

// One tile (bx, by, bz) of the FP32 operator with the fused p-update, for CG iteration `it`
// with coefficient beta; returns this thread's FP32 part of <p_new, A p_new>.  T is the
// block's shared staging area.  With Jacobi the tile forms p_new = D^{-1} r + beta p_old
// while staging and writes it; with SPEC the spectral preconditioner's last pass already
// wrote p_new (into the buffer p[(it & 1) ^ 1]), which the tile only reads.
template <bool COH, bool SPEC = false>
__device__ __forceinline__ float elas32_matvec_tile(const Geo& G, const Consts32& K,
                                                    const Elas32& I, int it, double beta_d,
                                                    int bx, int by, int bz, Tile32& T) {
  const bool first = it == 0;                 // p = D^{-1} r (the old p is undefined)
  const float beta = first ? 0.0f : (float)beta_d;
  const float* __restrict__ po[3] = {I.p[it & 1][0], I.p[it & 1][1], I.p[it & 1][2]};
  float* pn[3] = {I.p[(it & 1) ^ 1][0], I.p[(it & 1) ^ 1][1], I.p[(it & 1) ^ 1][2]};

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int i0 = bx * BX, j0 = by * BY;
  const int i = i0 + tx, j = j0 + ty;
  const bool on = (i < G.nx) && (j < G.ny);
  const int k0 = bz * G.zc, k1 = min(G.nz, k0 + G.zc);

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
      if (SPEC) {   // the preconditioner's last pass wrote p_new = z + beta p_old
        v.p[a] = ldf<COH>(pn[a] + g);
      } else {
        const float z = __ldg(I.dinv[a] + g) * ldf<COH>(I.r[a] + g);
        v.p[a] = first ? z : z + beta * ldf<COH>(po[a] + g);
      }
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
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    const long long zo = plane_offset(k0 - 1 + o);
    fetch(zo + ho0, r0);
    if (two) fetch(zo + ho1, r1);
    put(r0, o, tid);
    if (two) put(r1, o, hs1);
  }

  float part = 0.0f;
  const int ci = (ty + 1) * HX + (tx + 1);
  int s0 = 0, s1 = 1, s2 = 2, s3 = 3;    // slots of planes k-1, k, k+1 and the free one
  // eta of the thread's own node, loaded one plane ahead
  const long long col = (long long)j * G.nx + i;
  float eta_next = (on && k0 < k1) ? __ldg(I.eta + (long long)k0 * G.nxy + col) : 0.0f;
  for (int k = k0; k < k1; ++k) {
    const float eta_k = eta_next;
    if (on && k + 1 < k1) eta_next = __ldg(I.eta + (long long)(k + 1) * G.nxy + col);
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
    __syncthreads();                    // plane k+1 (written last iteration) is visible
    if (on) {
      const long long c = (long long)k * G.nxy + col;
      Fac32 f;
      tile_fac(T, t, K.ih2, eta_k, f);
      const float q0 = row_tile<0>(T, t, f, K.sc);
      const float q1 = row_tile<1>(T, t, f, K.sc);
      const float q2 = row_tile<2>(T, t, f, K.sc);
      const float p0 = tp(T, t, 0, 0, 0, 0), p1 = tp(T, t, 1, 0, 0, 0), p2 = tp(T, t, 2, 0, 0, 0);
      if (!SPEC) {
        pn[0][c] = p0;
        pn[1][c] = p1;
        pn[2][c] = p2;
      }
      I.q[0][c] = q0;
      I.q[1][c] = q1;
      I.q[2][c] = q2;
      part += p0 * q0 + p1 * q1 + p2 * q2;
    }
    if (more) {                         // plane k+2 goes to the free slot
      put(r0, s3, tid);
      if (two) put(r1, s3, hs1);
    }
    const int sf = s0;                  // rotate: (k-1, k, k+1, free) <- (k, k+1, k+2, k-1)
    s0 = s1;
    s1 = s2;
    s2 = s3;
    s3 = sf;
  }
  __syncthreads();                      // the tile may be restaged by the caller's next item
  return part;
}

// The FP32 operator on the spectral path (p_new already written by the preconditioner), with
// the tile layout of elas32_matvec_tile and its arithmetic.  The z loop is unrolled by the
// four plane slots, so the slots of planes k-1, k, k+1 and of the plane being staged are
// compile-time constants and every shared address is the thread's base plus a constant (the
// rotating slots of elas32_matvec_tile cost ~40 integer instructions per node).
template <int S0, int S1, int S2>
__device__ __forceinline__ Cell cell_of(Tile32& T, int ci) {
  Cell t;
  constexpr int sl[3] = {S0, S1, S2};
#pragma unroll
  for (int o = 0; o < 3; ++o) {
#pragma unroll
    for (int a = 0; a < 3; ++a) t.p[o][a] = &T.p[sl[o]][a][ci];
    t.mu[o] = &T.mu[sl[o]][ci];
    t.la[o] = &T.la[sl[o]][ci];
  }
  return t;
}

struct SpecTileCtx {
  const float* __restrict__ pn[3];
  long long ho0, ho1, col;
  int tid, hs1, ci, k1;
  bool two, on;
};

struct StagedNode {
  float p[3], mu, la;
};

__device__ __forceinline__ long long spec_plane_offset(const Geo& G, int kk) {
  const int kw = kk < 0 ? kk + G.nz : (kk >= G.nz ? kk - G.nz : kk);
  return (long long)kw * G.nxy;
}

__device__ __forceinline__ void spec_fetch(const SpecTileCtx& X, const Elas32& I, long long g,
                                           StagedNode& v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) v.p[a] = __ldg(X.pn[a] + g);
  v.mu = __ldg(I.mu + g);
  v.la = __ldg(I.lam + g);
}

template <int S>
__device__ __forceinline__ void spec_put(Tile32& T, const StagedNode& v, int s) {
#pragma unroll
  for (int a = 0; a < 3; ++a) T.p[S][a][s] = v.p[a];
  T.mu[S][s] = v.mu;
  T.la[S][s] = v.la;
}

// plane k from slots (S0, S1, S2); plane k + 2 is staged into slot S3
template <int S0, int S1, int S2, int S3>
__device__ __forceinline__ void spec_step(const Geo& G, const Consts32& K, const Elas32& I,
                                          const SpecTileCtx& X, Tile32& T, int k, float& eta_next,
                                          StagedNode& r0, StagedNode& r1, float& part) {
  const float eta_k = eta_next;
  const bool more = k + 1 < X.k1;
  if (X.on && more) eta_next = __ldg(I.eta + (long long)(k + 1) * G.nxy + X.col);
  if (more) {
    const long long zo = spec_plane_offset(G, k + 2);
    spec_fetch(X, I, zo + X.ho0, r0);
    if (X.two) spec_fetch(X, I, zo + X.ho1, r1);
  }
  __syncthreads();   // plane k + 1 (staged by the previous step) is visible
  if (X.on) {
    const Cell t = cell_of<S0, S1, S2>(T, X.ci);
    const long long c = (long long)k * G.nxy + X.col;
    Fac32 f;
    tile_fac(T, t, K.ih2, eta_k, f);
    const float q0 = row_tile<0>(T, t, f, K.sc);
    const float q1 = row_tile<1>(T, t, f, K.sc);
    const float q2 = row_tile<2>(T, t, f, K.sc);
    I.q[0][c] = q0;
    I.q[1][c] = q1;
    I.q[2][c] = q2;
    part += tp(T, t, 0, 0, 0, 0) * q0 + tp(T, t, 1, 0, 0, 0) * q1 + tp(T, t, 2, 0, 0, 0) * q2;
  }
  if (more) {
    spec_put<S3>(T, r0, X.tid);
    if (X.two) spec_put<S3>(T, r1, X.hs1);
  }
}

__device__ __forceinline__ float elas32_matvec_tile_spec(const Geo& G, const Consts32& K,
                                                         const Elas32& I, int it, int bx, int by,
                                                         int bz, Tile32& T) {
  SpecTileCtx X;
#pragma unroll
  for (int a = 0; a < 3; ++a) X.pn[a] = I.p[(it & 1) ^ 1][a];
  const int tx = threadIdx.x, ty = threadIdx.y;
  X.tid = ty * BX + tx;
  const int i0 = bx * BX, j0 = by * BY;
  const int i = i0 + tx, j = j0 + ty;
  X.on = (i < G.nx) && (j < G.ny);
  const int k0 = bz * G.zc;
  X.k1 = min(G.nz, k0 + G.zc);
  auto wrapped = [&](int s) {   // full modulo: a tile may be wider than the grid
    int gi = (i0 - 1 + s % HX) % G.nx, gj = (j0 - 1 + s / HX) % G.ny;
    gi = gi < 0 ? gi + G.nx : gi;
    gj = gj < 0 ? gj + G.ny : gj;
    return (long long)gj * G.nx + gi;
  };
  X.hs1 = X.tid + NT;
  X.two = X.hs1 < HXY;
  X.ho0 = wrapped(X.tid);
  X.ho1 = X.two ? wrapped(X.hs1) : 0;
  X.ci = (ty + 1) * HX + (tx + 1);
  X.col = (long long)j * G.nx + i;
  StagedNode r0, r1;
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    const long long zo = spec_plane_offset(G, k0 - 1 + o);
    spec_fetch(X, I, zo + X.ho0, r0);
    if (X.two) spec_fetch(X, I, zo + X.ho1, r1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T.p[o][a][X.tid] = r0.p[a];
      if (X.two) T.p[o][a][X.hs1] = r1.p[a];
    }
    T.mu[o][X.tid] = r0.mu;
    T.la[o][X.tid] = r0.la;
    if (X.two) {
      T.mu[o][X.hs1] = r1.mu;
      T.la[o][X.hs1] = r1.la;
    }
  }
  float part = 0.0f;
  float eta_next = (X.on && k0 < X.k1) ? __ldg(I.eta + (long long)k0 * G.nxy + X.col) : 0.0f;
  for (int k = k0; k < X.k1; k += 4) {
    spec_step<0, 1, 2, 3>(G, K, I, X, T, k, eta_next, r0, r1, part);
    if (k + 1 < X.k1) spec_step<1, 2, 3, 0>(G, K, I, X, T, k + 1, eta_next, r0, r1, part);
    if (k + 2 < X.k1) spec_step<2, 3, 0, 1>(G, K, I, X, T, k + 2, eta_next, r0, r1, part);
    if (k + 3 < X.k1) spec_step<3, 0, 1, 2>(G, K, I, X, T, k + 3, eta_next, r0, r1, part);
  }
  __syncthreads();
  return part;
}

// e += alpha p, r -= alpha q (p as written by this iteration's operator kernel, buffer pb),
// over float4 groups g = g0, g0 + gs, ... < g1 of an n-voxel system, plus the scalar tail
// n - n % 4 .. n when `tail` is set; accumulates <r, D^{-1} r> and <r, r>: the twelve products
// of one group summed in FP32, the groups in FP64.
template <bool COH, bool SPEC = false>
__device__ __forceinline__ void elas32_update_range(const Elas32& I, long long n, long long g0,
                                                    long long g1, long long gs, float alpha,
                                                    int pb, bool tail, double& drz,
                                                    double& drr) {
  for (long long v = g0; v < g1; v += gs) {
    float prz = 0.0f, prr = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float4* e4 = reinterpret_cast<float4*>(I.e[a]) + v;
      float4* r4 = reinterpret_cast<float4*>(I.r[a]) + v;
      const float4 p = ldf4<COH>(reinterpret_cast<const float4*>(I.p[pb][a]) + v);
      const float4 q = ldf4<COH>(reinterpret_cast<const float4*>(I.q[a]) + v);
      float4 e = *e4, r = *r4;
      e.x += alpha * p.x; e.y += alpha * p.y; e.z += alpha * p.z; e.w += alpha * p.w;
      r.x -= alpha * q.x; r.y -= alpha * q.y; r.z -= alpha * q.z; r.w -= alpha * q.w;
      *e4 = e;
      *r4 = r;
      if (!SPEC) {
        const float4 d = __ldg(reinterpret_cast<const float4*>(I.dinv[a]) + v);
        prz += r.x * (d.x * r.x) + r.y * (d.y * r.y) + r.z * (d.z * r.z) + r.w * (d.w * r.w);
      }
      prr += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
    }
    drz += (double)prz;
    drr += (double)prr;
  }
  if (tail) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    for (long long c = 4 * (n / 4) + tid; c < n; c += nth) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        I.e[a][c] += alpha * ldf<COH>(I.p[pb][a] + c);
        const float res = I.r[a][c] - alpha * ldf<COH>(I.q[a] + c);
        I.r[a][c] = res;
        if (!SPEC) drz += (double)(res * (I.dinv[a][c] * res));
        drr += (double)(res * res);
      }
    }
  }
}


// FP64 residual r = rhs - A u over one tile; writes the FP32 inner right-hand side r and
// zeroes the FP32 correction e; accumulates (|rhs|^2, |r|^2, <r, D^{-1} r>).
__device__ __forceinline__ void elas_ir_residual_tile(const Geo& G, const Elas& E, const Elas32& I,
                                                      int minus_b, int bx, int by, int bz,
                                                      double (&acc)[3]) {
  const double* const u[3] = {E.u[0], E.u[1], E.u[2]};
  const int i = bx * BX + threadIdx.x;
  const int j = by * BY + threadIdx.y;
  if (i < G.nx && j < G.ny) {
    const int k0 = bz * G.zc, k1 = min(G.nz, k0 + G.zc);
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
        const float z32 = E.jacobi ? I.dinv[a][c] * r32 : 0.0f;
        I.r[a][c] = r32;
        I.e[a][c] = 0.0f;
        acc[0] += rhs * rhs;
        acc[1] += res * res;
        acc[2] += (double)r32 * (double)z32;
      }
    }
  }
}

// The same residual in double-FP32 arithmetic (Elas::df): the operator's faces, diagonal, u,
// mu, lambda and b are (hi, lo) FP32 pairs, and each component's residual b - A u is one
// compensated sum (CSum) started at b, into which every product of the operator enters with
// its rounding error, so the FP64 units only convert the per-thread sums.  The differences of
// neighbouring u in the mixed derivatives are double-FP32 differences.  Sums of squares are
// formed in FP32 per thread (a few dozen terms of one sign) and in FP64 across threads.
__device__ __forceinline__ Df ndf(float2 v) { return Df{-v.x, -v.y}; }

template <int A, int D>
__device__ __forceinline__ Df elas_mixed_cs(const Nbr& nb, const float2* __restrict__ xd,
                                            const float2* __restrict__ mu,
                                            const float2* __restrict__ lam) {
  const Df epp = df_of(xd[at2<A, D>(nb, +1, +1)]);
  const Df epm = df_of(xd[at2<A, D>(nb, -1, +1)]);
  const Df emp = df_of(xd[at2<A, D>(nb, +1, -1)]);
  const Df emm = df_of(xd[at2<A, D>(nb, -1, -1)]);
  CSum m = {0.0f, 0.0f};
  cs_fma(m, df_of(mu[at1<D>(nb, +1)]), df_sub_near(epp, epm));
  cs_fma(m, ndf(mu[at1<D>(nb, -1)]), df_sub_near(emp, emm));
  cs_fma(m, df_of(lam[at1<A>(nb, +1)]), df_sub_near(epp, emp));
  cs_fma(m, ndf(lam[at1<A>(nb, -1)]), df_sub_near(epm, emm));
  return cs_value(m);
}

// component A of rhs - (eta I - L_h) u at node c
template <int A>
__device__ __forceinline__ Df elas_res_row_cs(const Nbr& nb, long long c, const Elas& E,
                                              const Df (&sc)[3][3], Df rhs) {
  constexpr int D1 = (A + 1) % 3, D2 = (A + 2) % 3;
  const float2* __restrict__ xa = E.udf[A];
  const float2* __restrict__ CA = reinterpret_cast<const float2*>(E.F[A]);
  const float2* __restrict__ C1 = reinterpret_cast<const float2*>(E.G[D1]);
  const float2* __restrict__ C2 = reinterpret_cast<const float2*>(E.G[D2]);
  const float2* __restrict__ DS = reinterpret_cast<const float2*>(E.dsum[A]);
  CSum v = {rhs.hi, rhs.lo};
  cs_fma(v, ndf(DS[c]), df_of(xa[c]));
  cs_fma(v, df_of(CA[c]), df_of(xa[at1<A>(nb, 1)]));
  cs_fma(v, df_of(CA[at1<A>(nb, -1)]), df_of(xa[at1<A>(nb, -1)]));
  cs_fma(v, df_of(C1[c]), df_of(xa[at1<D1>(nb, 1)]));
  cs_fma(v, df_of(C1[at1<D1>(nb, -1)]), df_of(xa[at1<D1>(nb, -1)]));
  cs_fma(v, df_of(C2[c]), df_of(xa[at1<D2>(nb, 1)]));
  cs_fma(v, df_of(C2[at1<D2>(nb, -1)]), df_of(xa[at1<D2>(nb, -1)]));
  cs_fma(v, sc[A][D1], elas_mixed_cs<A, D1>(nb, E.udf[D1], E.mudf, E.lamdf));
  cs_fma(v, sc[A][D2], elas_mixed_cs<A, D2>(nb, E.udf[D2], E.mudf, E.lamdf));
  return cs_value(v);
}

// The mixed-derivative weights 1 / (4 h_a h_d) as (hi, lo) pairs, passed as a kernel argument
// (read from the constant bank where used, so they take no registers).
struct ScDf {
  Df v[3][3];
};
inline ScDf sc_df_host(const Geo& G) {
  ScDf s;
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) s.v[a][d] = df_split_host(G.s_cross[a][d]);
  return s;
}

// b holds (hi, lo) pairs as well: E.b[a] reinterpreted
__device__ __forceinline__ void elas_ir_residual_tile_df(const Geo& G, const Elas& E,
                                                         const Elas32& I, int minus_b, int bx,
                                                         int by, int bz, const ScDf& scd,
                                                         double (&acc)[3]) {
  const Df(&sc)[3][3] = scd.v;
  float sbb = 0.0f, srr = 0.0f, srz = 0.0f;
  const int i = bx * BX + threadIdx.x;
  const int j = by * BY + threadIdx.y;
  if (i < G.nx && j < G.ny) {
    const int k0 = bz * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      Df rhs[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float2 bv = reinterpret_cast<const float2*>(E.b[a])[c];
        rhs[a] = minus_b ? Df{-bv.x, -bv.y} : Df{bv.x, bv.y};
      }
      const Df res[3] = {elas_res_row_cs<0>(nb, c, E, sc, rhs[0]),
                         elas_res_row_cs<1>(nb, c, E, sc, rhs[1]),
                         elas_res_row_cs<2>(nb, c, E, sc, rhs[2])};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float r32 = __fadd_rn(res[a].hi, res[a].lo);
        const float z32 = E.jacobi ? I.dinv[a][c] * r32 : 0.0f;
        I.r[a][c] = r32;
        I.e[a][c] = 0.0f;
        sbb += rhs[a].hi * rhs[a].hi;
        srr += r32 * r32;
        srz += r32 * z32;
      }
    }
  }
  acc[0] += (double)sbb;
  acc[1] += (double)srr;
  acc[2] += (double)srz;
}

// Outer decision after a residual (the same test as the FP64 solve: |r| <= rtol |rhs|) and the
// start of the inner FP32 solve A e = r with relative target max(tau_min, half of what the
// outer still needs).  O.pad counts the inner iterations spent so far; a solve that exceeds
// max_sweeps residuals or maxit inner iterations stops with CG_MAXIT.  With normalize the
// inner right-hand side is to be multiplied by S.scale, the power of two nearest 1 / |r|, so
// that the FP32 iteration sees values of order one whatever the residual's size (deep
// tolerances or small adjoint sources would otherwise underflow FP32 products); the inner
// scalars are set for the scaled system and the correction divides by S.scale.
__device__ __forceinline__ void elas_ir_residual_finalize(CgScal& O, CgScal& S, double bb,
                                                          double rr, double rz, double tau_min,
                                                          int max_sweeps,
                                                          bool normalize = false) {
  if (O.it > 0) O.pad += S.it;
  O.bb = bb;
  O.rr = rr;
  O.it += 1;
  if (bb == 0.0) {
    O.status = CG_ZERO_RHS;
  } else if (!isfinite(rr)) {
    O.status = CG_NONFINITE;
  } else if (sqrt(rr) <= O.rtol * sqrt(bb)) {
    O.status = CG_CONVERGED;
  } else if (O.it > max_sweeps || O.pad >= O.maxit) {
    O.status = CG_MAXIT;
  } else {
    O.status = CG_RUNNING;
  }
  const double s =
      (normalize && rr > 0.0 && isfinite(rr)) ? exp2(-rint(0.5 * log2(rr))) : 1.0;
  S.scale = s;
  S.bb = rr * s * s;
  S.rr = rr * s * s;
  S.rz = rz * s * s;
  S.it = 0;
  S.maxit = O.maxit;
  S.alpha = 0.0;
  S.beta = 0.0;
  S.rtol = (rr > 0.0) ? fmax(tau_min, 0.5 * O.rtol * sqrt(bb / rr)) : 1.0;
  S.status = (O.status == CG_RUNNING) ? CG_RUNNING : CG_CONVERGED;
}

// u += e / scale, du += e / scale over voxels c = c0, c0 + cs, ... < c1 (scale: the inner
// right-hand side's factor, a power of two)
__device__ __forceinline__ void elas_ir_correct_range(const Elas& E, const Elas32& I, long long c0,
                                                      long long c1, long long cs,
                                                      double inv_scale = 1.0) {
  for (long long c = c0; c < c1; c += cs) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double e = f64_of_scaled(I.e[a][c], inv_scale);   // exact; no FP64 operation
      const double un = E.u[a][c] + e;
      E.u[a][c] = un;
      E.du[a][c] += e;
      if (E.df) E.udf[a][c] = df_pack(un);
    }
  }
}


// ------------------------------------------------------------------------------ CN tiles

struct Faces {
  double xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ Faces load_faces(const Cn3& C, const Nbr& nb, long long c) {
  Faces F;
  F.xp = C.Kf[0][c];
  F.xm = C.Kf[0][nb.at(-1, 0, 0)];
  F.yp = C.Kf[1][c];
  F.ym = C.Kf[1][nb.at(0, -1, 0)];
  F.zp = C.Kf[2][c];
  F.zm = C.Kf[2][nb.at(0, 0, -1)];
  return F;
}

// CN start on one tile: x0 = c, rhs = c + s, r0 = 2 s with s = dt/2 D_h c; accumulates
// (|rhs|^2, |r|^2, <r, D^{-1} r>) per right-hand side in the bit mask (bit r: solve r).
__device__ __forceinline__ void cn_init_tile(const Geo& G, const Cn3& C, int bx, int by, int bz,
                                             double (&acc)[9], int mask = 7) {
  const int i = bx * BX + threadIdx.x;
  const int j = by * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = bz * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    const long long c = nb.at(0, 0, 0);
    const Faces F = load_faces(C, nb, c);
    const double di = C.dinv[c];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!((mask >> r) & 1)) continue;
      const double* x = C.x[r];
      const double xc = x[c];
      const double s = F.xp * (x[nb.at(1, 0, 0)] - xc) - F.xm * (xc - x[nb.at(-1, 0, 0)]) +
                       F.yp * (x[nb.at(0, 1, 0)] - xc) - F.ym * (xc - x[nb.at(0, -1, 0)]) +
                       F.zp * (x[nb.at(0, 0, 1)] - xc) - F.zm * (xc - x[nb.at(0, 0, -1)]);
      const double rhs = xc + s;
      const double res = 2.0 * s;
      const double z = di * res;
      C.r[r][c] = res;
      C.p[r][c] = z;
      acc[3 * r + 0] += rhs * rhs;
      acc[3 * r + 1] += res * res;
      acc[3 * r + 2] += res * z;
    }
  }
}

// q = A p and <p, q> for the running solves act[] on one tile
template <bool COH>
__device__ __forceinline__ void cn_matvec_tile(const Geo& G, const Cn3& C, const bool (&act)[3],
                                               int bx, int by, int bz, double (&acc)[3]) {
  const int i = bx * BX + threadIdx.x;
  const int j = by * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = bz * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    const long long c = nb.at(0, 0, 0);
    const Faces F = load_faces(C, nb, c);
    const double d = C.dsum[c];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!act[r]) continue;
      const double* p = C.p[r];
      const double pc = ldd<COH>(p + c);
      const double q = d * pc - (F.xp * ldd<COH>(p + nb.at(1, 0, 0)) + F.xm * ldd<COH>(p + nb.at(-1, 0, 0)) +
                                 F.yp * ldd<COH>(p + nb.at(0, 1, 0)) + F.ym * ldd<COH>(p + nb.at(0, -1, 0)) +
                                 F.zp * ldd<COH>(p + nb.at(0, 0, 1)) + F.zm * ldd<COH>(p + nb.at(0, 0, -1)));
      C.q[r][c] = q;
      acc[r] += pc * q;
    }
  }
}

// x += alpha p, r -= alpha q; accumulates <r, D^{-1} r>, <r, r> per running solve
__device__ __forceinline__ void cn_update_tile(const Geo& G, const Cn3& C, const bool (&act)[3],
                                               const double (&alpha)[3], int bx, int by, int bz,
                                               double (&acc)[6]) {
  const int i = bx * BX + threadIdx.x;
  const int j = by * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = bz * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    const double di = C.dinv[c];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (!act[r]) continue;
      C.x[r][c] += alpha[r] * C.p[r][c];
      const double res = C.r[r][c] - alpha[r] * C.q[r][c];
      C.r[r][c] = res;
      acc[2 * r + 0] += res * (di * res);
      acc[2 * r + 1] += res * res;
    }
  }
}

// p = D^{-1} r + beta p for the running solves
__device__ __forceinline__ void cn_pupdate_tile(const Geo& G, const Cn3& C, const bool (&act)[3],
                                                const double (&beta)[3], int bx, int by, int bz) {
  const int i = bx * BX + threadIdx.x;
  const int j = by * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = bz * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    const double di = C.dinv[c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      if (act[r]) C.p[r][c] = di * C.r[r][c] + beta[r] * C.p[r][c];
  }
}

}  // namespace tg
