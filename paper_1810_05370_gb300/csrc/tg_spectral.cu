// tg_spectral.cu -- the constant-coefficient spectral preconditioner of the elasticity solve.
//
// Section 3 preconditions the variable-coefficient elasticity solve by solving the same
// equation with constant Lame coefficients (their averages over the domain), which the
// Fourier transform diagonalises.  Here the operator is the finite-difference one, so the
// exact inverse uses its discrete symbol: on the grid mode exp(i theta . j), theta_d =
// 2 pi k_d / n_d, the compact second difference gives -S_d = -4 sin^2(theta_d / 2) / h_d^2
// and the centred first difference i T_d = i sin(theta_d) / h_d, so eta0 I - L_h[mu0, lam0]
// acts on the mode's amplitude vector as
//   M = diag(D) + c T T^T,   D_a = eta0 + mu0 (S_0 + S_1 + S_2) + c (S_a - T_a^2),
//   c = lam0 + mu0,
// whose inverse is Sherman-Morrison's:  M^{-1} r = D^{-1} r - c D^{-1} T (T^T D^{-1} r) /
// (1 + c T^T D^{-1} T).
//
// z = F^{-1} M^{-1} F r takes five passes over the three components, each a batch of 1-D
// FFTs staged in shared memory:
//   x forward  two real rows form one complex line; the half spectrum (kx <= nx/2) of both
//              is split off the line's transform and written to W;
//   y forward  columns of W, in place;
//   z          columns of all three components together: forward transform, the 3x3
//              inverse per mode (with the 1/V normalisation) and <r, z> by Parseval's
//              identity (a sum of non-negative terms r^* M^{-1} r^), inverse transform, in place;
//   y inverse  in place;
//   x inverse  the Hermitian half spectra of two rows form one complex line whose inverse
//              transform carries both real rows; writes z.
// The 1-D transforms are Stockham autosort FFTs whose butterflies are radix-16 DFTs held in
// registers (one radix-2, 4 or 8 stage takes the remainder of log2 n), ping-ponging between
// two shared-memory buffers with one barrier per stage; each block keeps its line length's
// twiddles in shared memory and issues its global loads in batches of eight per thread.
#include <cuda.h>           // CUtensorMap (types only; the encoder comes from the driver)
#include <cudaTypedefs.h>

#include "tg_tiles.cuh"

namespace tg {
namespace {

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiplication by -i (forward, SGN = -1) or +i (inverse, SGN = +1)
template <int SGN, typename C> __device__ __forceinline__ C rot(C a) {
  return SGN < 0 ? C{a.y, -a.x} : C{-a.y, a.x};
}
// the table holds exp(-2 pi i k / n); the inverse transform uses its conjugate
template <int SGN, typename C> __device__ __forceinline__ C root(const C* tw, int k) {
  const C w = tw[k];
  return SGN < 0 ? w : C{w.x, -w.y};
}

// --------------------------------------------------------------- small DFTs in registers
// v[0..R) in, X[0..R) out in natural order, X[k] = sum_m v[m] exp(SGN 2 pi i m k / R).
template <int SGN, typename C> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  const C a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = rot<SGN>(csub(v1, v3));
  v0 = cadd(a0, a2);
  v1 = cadd(a1, a3);
  v2 = csub(a0, a2);
  v3 = csub(a1, a3);
}

// v * exp(SGN 2 pi i m / 16) for the constant m; cos and sin of m pi / 8 written out
template <int SGN, int M, typename C> __device__ __forceinline__ C w16(C v) {
  using R = decltype(v.x);
  constexpr double c1 = 0.92387953251128674, s1 = 0.38268343236508977, h = 0.70710678118654752;
  constexpr double cs = M == 1 ? c1 : M == 2 ? h : M == 3 ? s1 : M == 6 ? -h : M == 9 ? -c1 : 1.0;
  constexpr double sn = M == 1 ? s1 : M == 2 ? h : M == 3 ? c1 : M == 6 ? h : M == 9 ? -s1 : 0.0;
  if constexpr (M == 0) {
    return v;
  } else if constexpr (M == 4) {
    return rot<SGN>(v);                 // exp(SGN i pi / 2) = SGN i
  } else {
    const R c = (R)cs, w = (R)(SGN < 0 ? -sn : sn);
    return C{v.x * c - v.y * w, v.x * w + v.y * c};
  }
}

template <int LR, int SGN, typename C> __device__ __forceinline__ void dft(C (&v)[1 << LR]) {
  if constexpr (LR == 1) {
    const C t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  } else if constexpr (LR == 2) {
    dft4<SGN>(v[0], v[1], v[2], v[3]);
  } else if constexpr (LR == 3) {
    // even and odd halves, then X[k] = E[k] + W8^k O[k], X[k + 4] = E[k] - W8^k O[k]
    dft4<SGN>(v[0], v[2], v[4], v[6]);
    dft4<SGN>(v[1], v[3], v[5], v[7]);
    const C o1 = w16<SGN, 2>(v[3]), o2 = w16<SGN, 4>(v[5]), o3 = w16<SGN, 6>(v[7]);
    const C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
  } else {
    // 16 = 4 x 4: Y_q = DFT4 of v[q + 4m] (lands at v[q + 4k]), Z_q[k] = W16^{qk} Y_q[k],
    // X[k + 4t] = DFT4 over q of Z_q[k]
    dft4<SGN>(v[0], v[4], v[8], v[12]);
    dft4<SGN>(v[1], v[5], v[9], v[13]);
    dft4<SGN>(v[2], v[6], v[10], v[14]);
    dft4<SGN>(v[3], v[7], v[11], v[15]);
    v[5] = w16<SGN, 1>(v[5]);
    v[6] = w16<SGN, 2>(v[6]);
    v[7] = w16<SGN, 3>(v[7]);
    v[9] = w16<SGN, 2>(v[9]);
    v[10] = w16<SGN, 4>(v[10]);
    v[11] = w16<SGN, 6>(v[11]);
    v[13] = w16<SGN, 3>(v[13]);
    v[14] = w16<SGN, 6>(v[14]);
    v[15] = w16<SGN, 9>(v[15]);
    dft4<SGN>(v[0], v[1], v[2], v[3]);
    dft4<SGN>(v[4], v[5], v[6], v[7]);
    dft4<SGN>(v[8], v[9], v[10], v[11]);
    dft4<SGN>(v[12], v[13], v[14], v[15]);
    // X[k + 4t] sits at v[4k + t]: transpose the 4 x 4 block
    C t[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) t[q] = v[q];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = t[4 * (q & 3) + (q >> 2)];
  }
}

// One Stockham stage of radix 2^LR over lo * hi lines of length n = 2^ln: sub-transforms of
// length Ns = 2^lNs are merged into ones of length Ns * R.  Line l = lh * lo + ll (ll < lo,
// lh < hi, lo a power of two) has element e at a[l * ls + e * es].  Work item `it` is
// (ll, j, lh) with ll fastest, so consecutive threads take consecutive interleaved lines
// (es > 1) or consecutive butterflies of one line (lo = 1, es = 1).  tw[k] =
// exp(-2 pi i k / n) (the inverse transform conjugates it).
template <int LR, int SGN, typename C>
__device__ __forceinline__ void fft_stage(const C* a, C* b, int ln, int lNs, int llo, int hi,
                                          int ls, int es, const C* tw) {
  constexpr int R = 1 << LR;
  const int lnb = ln - LR, nb = 1 << lnb, Ns = 1 << lNs, lts = ln - lNs - LR;
  const int lo_mask = (1 << llo) - 1;
  const int total = hi << (llo + lnb);
  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    const int ll = it & lo_mask;
    const int rest = it >> llo;
    const int j = rest & (nb - 1);
    const int l = ((rest >> lnb) << llo) + ll;
    const int k = j & (Ns - 1);           // position inside the current sub-transform
    const int d = ((j >> lNs) << (lNs + LR)) + k;
    const C* src = a + l * ls;
    C* dst = b + l * ls;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * es];
    if (k > 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], root<SGN>(tw, (r * k) << lts));
    }
    dft<LR, SGN>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(d + r * Ns) * es] = v[r];
  }
}

// Transforms the lines (layout as in fft_stage) of length n = 2^ln, n >= 2: one stage of
// radix 2, 4 or 8 for the remainder of ln mod 4, then radix-16 stages, one barrier after
// each.  Entry: a and tw loaded and visible to the block.  Returns the buffer holding the
// result (visible to the block).
template <int SGN, typename C>
__device__ C* fft_lines(C* a, C* b, int ln, int llo, int hi, int ls, int es, const C* tw) {
  int lNs = ln & 3;
  if (lNs == 1) fft_stage<1, SGN>(a, b, ln, 0, llo, hi, ls, es, tw);
  if (lNs == 2) fft_stage<2, SGN>(a, b, ln, 0, llo, hi, ls, es, tw);
  if (lNs == 3) fft_stage<3, SGN>(a, b, ln, 0, llo, hi, ls, es, tw);
  if (lNs != 0) {
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
  }
  for (; lNs < ln; lNs += 4) {
    fft_stage<4, SGN>(a, b, ln, lNs, llo, hi, ls, es, tw);
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
  }
  return a;
}

// The same transforms in place in one buffer, for plans whose every stage has at most one
// butterfly per thread (the launch's shape guarantees it): a thread reads its butterfly's
// inputs, the block synchronises, the thread writes the outputs where the ping-pong stage
// would have written them in the other buffer, so the values are those of fft_lines bit for
// bit.  Two barriers per stage, half the shared memory.
template <int LR, int SGN, typename C>
__device__ __forceinline__ void fft_stage_inplace(C* a, int ln, int lNs, int llo, int hi, int ls,
                                                  int es, const C* tw) {
  constexpr int R = 1 << LR;
  const int lnb = ln - LR, nb = 1 << lnb, Ns = 1 << lNs, lts = ln - lNs - LR;
  const int lo_mask = (1 << llo) - 1;
  const int total = hi << (llo + lnb);
  const int it = threadIdx.x;
  const bool act = it < total;
  C v[R];
  int base = 0, d = 0;
  if (act) {
    const int ll = it & lo_mask;
    const int rest = it >> llo;
    const int j = rest & (nb - 1);
    const int l = ((rest >> lnb) << llo) + ll;
    const int k = j & (Ns - 1);
    d = ((j >> lNs) << (lNs + LR)) + k;
    base = l * ls;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = a[base + (j + r * nb) * es];
    if (k > 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], root<SGN>(tw, (r * k) << lts));
    }
    dft<LR, SGN>(v);
  }
  __syncthreads();   // every input of the stage is read
  if (act) {
#pragma unroll
    for (int r = 0; r < R; ++r) a[base + (d + r * Ns) * es] = v[r];
  }
}

template <int SGN, typename C>
__device__ C* fft_lines_inplace(C* a, int ln, int llo, int hi, int ls, int es, const C* tw) {
  int lNs = ln & 3;
  if (lNs == 1) fft_stage_inplace<1, SGN>(a, ln, 0, llo, hi, ls, es, tw);
  if (lNs == 2) fft_stage_inplace<2, SGN>(a, ln, 0, llo, hi, ls, es, tw);
  if (lNs == 3) fft_stage_inplace<3, SGN>(a, ln, 0, llo, hi, ls, es, tw);
  if (lNs != 0) __syncthreads();
  for (; lNs < ln; lNs += 4) {
    fft_stage_inplace<4, SGN>(a, ln, lNs, llo, hi, ls, es, tw);
    __syncthreads();
  }
  return a;
}

__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

// The x passes' transform of pb interleaved lines: FORM 0 in two buffers, 1 in place, 2 as the
// shape's x_inpl says (the hot kernels are instantiated per form, so each holds one path)
template <int SGN, int FORM, typename C>
__device__ __forceinline__ const C* fft_x(bool inpl, C* a, C* b, int ln, int llo, int es,
                                          const C* tw) {
  if (FORM == 1 || (FORM == 2 && inpl)) return fft_lines_inplace<SGN>(a, ln, llo, 1, 1, es, tw);
  return fft_lines<SGN>(a, b, ln, llo, 1, 1, es, tw);
}

// --------------------------------------------------- stages that read or write global memory
// The y and z passes keep their lines interleaved both in global memory (consecutive mode
// columns are contiguous) and in shared memory, so the first stage of a transform can gather
// its radix-16 inputs straight from global memory into registers (16 loads in flight per
// thread) and the last stage can scatter its outputs straight back: two shared-memory round
// trips and a barrier fewer per transform.  Accessors: element e of line l.
template <typename C> struct SmemIO {
  C* p;
  int ls, es;
  __device__ __forceinline__ C ld(int l, int e) const { return p[l * ls + e * es]; }
  __device__ __forceinline__ void st(int l, int e, C v) const { p[l * ls + e * es] = v; }
};

// y pass: line l = mode column kx0 + l of one (component, z) plane; element e = row y
template <typename C> struct ColIO {
  C* W;     // &W[comp][z][0][kx0]
  int nxp, ncol;
  __device__ __forceinline__ C ld(int l, int e) const {
    return l < ncol ? W[(size_t)e * nxp + l] : C{0, 0};
  }
  __device__ __forceinline__ void st(int l, int e, C v) const {
    if (l < ncol) W[(size_t)e * nxp + l] = v;
  }
};

// z pass: line l = (component l >> ltz, column l & (tz - 1)); element e = plane kz
template <typename C> struct ZIO {
  C* W;     // &W[0][0][ky][kx0]
  size_t plane, comp_stride;
  int tz, ltz, ncol;
  __device__ __forceinline__ size_t at(int l, int e) const {
    return (size_t)(l >> ltz) * comp_stride + (size_t)e * plane + (l & (tz - 1));
  }
  __device__ __forceinline__ C ld(int l, int e) const {
    return (l & (tz - 1)) < ncol ? W[at(l, e)] : C{0, 0};
  }
  __device__ __forceinline__ void st(int l, int e, C v) const {
    if ((l & (tz - 1)) < ncol) W[at(l, e)] = v;
  }
};

// fft_stage with accessors for its source and destination (same work mapping)
template <int LR, int SGN, typename C, class SRC, class DST>
__device__ __forceinline__ void fft_stage_io(const SRC& src, const DST& dst, int ln, int lNs,
                                             int llo, int hi, const C* tw) {
  constexpr int R = 1 << LR;
  const int lnb = ln - LR, nb = 1 << lnb, Ns = 1 << lNs, lts = ln - lNs - LR;
  const int lo_mask = (1 << llo) - 1;
  const int total = hi << (llo + lnb);
  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    const int ll = it & lo_mask;
    const int rest = it >> llo;
    const int j = rest & (nb - 1);
    const int l = ((rest >> lnb) << llo) + ll;
    const int k = j & (Ns - 1);
    const int d = ((j >> lNs) << (lNs + LR)) + k;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src.ld(l, j + r * nb);
    if (k > 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], root<SGN>(tw, (r * k) << lts));
    }
    dft<LR, SGN>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) dst.st(l, d + r * Ns, v[r]);
  }
}

template <int SGN, typename C, class SRC, class DST>
__device__ __forceinline__ void stage_any(int LR, const SRC& src, const DST& dst, int ln, int lNs,
                                          int llo, int hi, const C* tw) {
  if (LR == 1) fft_stage_io<1, SGN>(src, dst, ln, lNs, llo, hi, tw);
  else if (LR == 2) fft_stage_io<2, SGN>(src, dst, ln, lNs, llo, hi, tw);
  else if (LR == 3) fft_stage_io<3, SGN>(src, dst, ln, lNs, llo, hi, tw);
  else fft_stage_io<4, SGN>(src, dst, ln, lNs, llo, hi, tw);
}

// Transforms of length 2^ln (plan as in fft_lines) whose first stage reads global memory
// through an accessor and/or whose last stage writes it; a and b are the shared ping-pong
// buffers (layout ls, es).  The first stage never uses twiddles (Ns = 1), so tw only has to be
// visible by the second stage: a barrier follows every stage but the last.
template <int SGN, typename C, class SRC>
__device__ C* fft_from_global(const SRC& first, C* a, C* b, int ls, int es, int ln, int llo,
                              int hi, const C* tw) {
  const int rem = ln & 3, nst = (rem ? 1 : 0) + (ln >> 2);
  int lNs = 0;
  C* cur = b;
  C* oth = a;
  for (int s = 0; s < nst; ++s) {
    const int LR = (s == 0 && rem) ? rem : 4;
    if (s == 0)
      stage_any<SGN>(LR, first, SmemIO<C>{cur, ls, es}, ln, lNs, llo, hi, tw);
    else
      stage_any<SGN>(LR, SmemIO<C>{oth, ls, es}, SmemIO<C>{cur, ls, es}, ln, lNs, llo, hi, tw);
    __syncthreads();
    lNs += LR;
    C* t = cur;   // the result of this stage becomes the next input
    cur = oth;
    oth = t;
  }
  return oth;     // holds the last stage's output
}

// input in `in` (visible to the block), scratch `oth`; the last stage writes through `last`
template <int SGN, typename C, class DST>
__device__ void fft_to_global(C* in, C* oth, const DST& last, int ls, int es, int ln, int llo,
                              int hi, const C* tw) {
  const int rem = ln & 3, nst = (rem ? 1 : 0) + (ln >> 2);
  int lNs = 0;
  for (int s = 0; s < nst; ++s) {
    const int LR = (s == 0 && rem) ? rem : 4;
    if (s == nst - 1) {
      stage_any<SGN>(LR, SmemIO<C>{in, ls, es}, last, ln, lNs, llo, hi, tw);
    } else {
      stage_any<SGN>(LR, SmemIO<C>{in, ls, es}, SmemIO<C>{oth, ls, es}, ln, lNs, llo, hi, tw);
      __syncthreads();
      C* t = in;
      in = oth;
      oth = t;
    }
    lNs += LR;
  }
}

// global lines in place: through shared memory, both ends direct
template <int SGN, typename C, class IO>
__device__ void fft_global_inplace(const IO& io, C* a, C* b, int ls, int es, int ln, int llo,
                                   int hi, const C* tw) {
  const int rem = ln & 3, nst = (rem ? 1 : 0) + (ln >> 2);
  if (nst == 1) {   // one stage: stage into shared memory first (its reads and writes overlap)
    C* r = fft_from_global<SGN>(io, a, b, ls, es, ln, llo, hi, tw);
    const int nl = hi << llo, n = 1 << ln;
    for (int q = threadIdx.x; q < nl * n; q += blockDim.x) {
      const int l = q % nl, e = q / nl;
      io.st(l, e, r[l * ls + e * es]);
    }
    return;
  }
  // first stage: global -> b; middle stages ping-pong; last stage -> global
  const int LR0 = rem ? rem : 4;
  stage_any<SGN>(LR0, io, SmemIO<C>{b, ls, es}, ln, 0, llo, hi, tw);
  __syncthreads();
  const int rest_ln = ln;   // the remaining stages continue from Ns = 2^LR0
  int lNs = LR0;
  C* in = b;
  C* oth = a;
  for (int s = 1; s < nst; ++s) {
    if (s == nst - 1) {
      stage_any<SGN>(4, SmemIO<C>{in, ls, es}, io, rest_ln, lNs, llo, hi, tw);
    } else {
      stage_any<SGN>(4, SmemIO<C>{in, ls, es}, SmemIO<C>{oth, ls, es}, rest_ln, lNs, llo, hi, tw);
      __syncthreads();
      C* t = in;
      in = oth;
      oth = t;
    }
    lNs += 4;
  }
}

// Global -> shared staging in batches of LB elements per thread: all loads of a batch are
// issued before any result is stored, so each thread keeps LB loads in flight.
constexpr int LB = 8;

// the n twiddles of one line length into shared memory
template <typename C>
__device__ __forceinline__ void load_roots(C* dst, const C* __restrict__ src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

template <typename C> __device__ __forceinline__ C* smem_cx() {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return reinterpret_cast<C*>(smem_raw);
}

template <typename R>
__device__ __forceinline__ bool spec_skip(const CgScal* S) {
  return S != nullptr && S->status != CG_RUNNING;
}

// Sum of one value per thread over a launch of any block size (a multiple of 32): warps,
// then the block's warps in order into partial[b]; the last block to finish sums the
// partials (each thread a fixed stride, then its warps in order: deterministic) and returns
// true in thread 0 with the total.
__device__ bool block_sum_last(double v, double* partial, unsigned int* counter, int b, int nb,
                               double& total) {
  __shared__ double sh[32];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[w];
    partial[b] = s;
    __threadfence();
    am_last = atomicAdd(counter, 1u) == (unsigned int)(nb - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double s = 0.0;   // every thread a fixed stride of the partials, then warps in order
  for (int k = threadIdx.x; k < nb; k += blockDim.x) s += __ldcg(partial + k);
  s = warp_sum(s);
  __syncthreads();
  if (lane == 0) sh[warp] = s;
  __syncthreads();
  if (threadIdx.x != 0) return false;
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += sh[w];
  total = t;
  *counter = 0u;
  return true;
}

// ---------------------------------------------------------------------------- x forward
// block (pair tile, z, component): rows y0 .. y0 + 2 pb - 1 of plane z.  The staged lines
// are interleaved, element e of line l at e * es + l; es = pb + 1 keeps the row-wise staging
// accesses (consecutive e) free of bank conflicts.
template <typename R>
struct XTile {
  using C = typename CxOf<R>::T;
  int n, ln, pb, es, comp, z, y0;
  size_t row0;   // first voxel of the block's rows in a component array
};

template <typename R>
__device__ __forceinline__ XTile<R> x_tile(const Spec<R>& V) {
  XTile<R> t;
  t.n = V.nx;
  t.ln = ilog2(V.nx);
  t.pb = V.pb;
  t.es = V.pb + 1;
  t.comp = blockIdx.z;
  t.z = blockIdx.y;
  t.y0 = 2 * V.pb * blockIdx.x;
  t.row0 = ((size_t)t.z * V.ny + t.y0) * V.nx;
  return t;
}

// transform the staged rows (in a) and write both half spectra to W
template <typename R, int FORM>
__device__ __forceinline__ void x_fwd_finish(const Spec<R>& V, const XTile<R>& t,
                                             typename CxOf<R>::T* a, typename CxOf<R>::T* b,
                                             const typename CxOf<R>::T* tw) {
  using C = typename CxOf<R>::T;
  const int n = t.n, es = t.es;
  const C* F = fft_x<-1, FORM>(V.x_inpl != 0, a, b, t.ln, ilog2(t.pb), es, tw);
  C* W = V.W + (((size_t)t.comp * V.nz + t.z) * V.ny + t.y0) * V.nxp;
  for (int idx = threadIdx.x; idx < t.pb * V.nxh; idx += blockDim.x) {
    const int l = idx / V.nxh, k = idx - l * V.nxh;
    const C f = F[k * es + l], g = F[((n - k) & (n - 1)) * es + l];
    // row 2l: (f + conj g) / 2;  row 2l+1: (f - conj g) / (2i)
    W[(size_t)(2 * l) * V.nxp + k] = C{(R)0.5 * (f.x + g.x), (R)0.5 * (f.y - g.y)};
    W[(size_t)(2 * l + 1) * V.nxp + k] = C{(R)0.5 * (f.y + g.y), (R)-0.5 * (f.x - g.x)};
  }
}

template <typename R>
__global__ void __launch_bounds__(NT) k_spec_x_fwd(Spec<R> V, const R* __restrict__ r0,
                                                   const R* __restrict__ r1,
                                                   const R* __restrict__ r2, const CgScal* S) {
  using C = typename CxOf<R>::T;
  if (spec_skip<R>(S)) return;
  const XTile<R> t = x_tile(V);
  const int n = t.n, ln = t.ln, es = t.es;
  C* tw = smem_cx<C>();
  C* a = tw + n;
  C* b = a + (size_t)es * n;
  load_roots(tw, V.tw[0], n);
  const R* src = t.comp == 0 ? r0 : (t.comp == 1 ? r1 : r2);
  const R* sc = V.s[t.comp];   // the transform takes s r with the scaled preconditioner
  const int total = t.pb * n;
  for (int i0 = threadIdx.x; i0 < total; i0 += LB * blockDim.x) {
    R va[LB], vb[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) {
        const size_t o = t.row0 + (size_t)(2 * (idx >> ln)) * n + (idx & (n - 1));
        va[u] = __ldg(src + o);
        vb[u] = __ldg(src + o + n);
        if (sc) {
          va[u] *= __ldg(sc + o);
          vb[u] *= __ldg(sc + o + n);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) a[(idx & (n - 1)) * es + (idx >> ln)] = C{va[u], vb[u]};
    }
  }
  __syncthreads();
  x_fwd_finish<R, 2>(V, t, a, b, tw);
}

// The mixed precision's CG update fused into the x forward pass: for the block's rows
// e += alpha p, r -= alpha q (p as written by this iteration's operator kernel), the new r
// staged straight into the transform, and <r, r> reduced over the launch; the last block
// takes the convergence decision.  Saves the pass that re-read r.
__global__ void __launch_bounds__(NT, 4) k_spec_update_xfwd(Spec<float> V, Elas32 I) {
  using C = float2;
  if (!running(I.S)) return;
  const float alpha = (float)I.S->alpha;
  const int pbuf = (I.S->it & 1) ^ 1;
  const XTile<float> t = x_tile(V);
  const int n = t.n, ln = t.ln, es = t.es;
  C* tw = smem_cx<C>();
  C* a = tw + n;
  C* b = a + (size_t)es * n;
  load_roots(tw, V.tw[0], n);
  float* e = I.e[t.comp];
  float* r = I.r[t.comp];
  const float* p = I.p[pbuf][t.comp];
  const float* q = I.q[t.comp];
  const float* sc = V.s[t.comp];   // the transform takes s r with the scaled preconditioner
  constexpr int UB = 4;
  float rr = 0.0f;
  const int total = t.pb * n;
  for (int i0 = threadIdx.x; i0 < total; i0 += UB * blockDim.x) {
    float ea[UB], eb[UB], ra[UB], rb[UB], pa[UB], pbv[UB], qa[UB], qb[UB], sa[UB], sb[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) {
        const size_t o = t.row0 + (size_t)(2 * (idx >> ln)) * n + (idx & (n - 1));
        ea[u] = e[o];
        eb[u] = e[o + n];
        ra[u] = r[o];
        rb[u] = r[o + n];
        pa[u] = p[o];
        pbv[u] = p[o + n];
        qa[u] = q[o];
        qb[u] = q[o + n];
        sa[u] = sc ? __ldg(sc + o) : 1.0f;
        sb[u] = sc ? __ldg(sc + o + n) : 1.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) {
        const size_t o = t.row0 + (size_t)(2 * (idx >> ln)) * n + (idx & (n - 1));
        const float xa = ra[u] - alpha * qa[u], xb = rb[u] - alpha * qb[u];
        e[o] = ea[u] + alpha * pa[u];
        e[o + n] = eb[u] + alpha * pbv[u];
        r[o] = xa;
        r[o + n] = xb;
        rr += xa * xa + xb * xb;
        a[(idx & (n - 1)) * es + (idx >> ln)] = C{xa * sa[u], xb * sb[u]};
      }
    }
  }
  double acc[1] = {(double)rr};
  double out[1];
  const int nb = gridDim.x * gridDim.y * gridDim.z;
  const int bl = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  if (reduce_indexed<1>(acc, V.partial, V.counter, bl, nb, out) && threadIdx.x == 0)
    cg_after_update_rr(*I.S, out[0]);   // reduce_indexed's barriers also publish the staging
  __syncthreads();
  x_fwd_finish<float, 0>(V, t, a, b, tw);   // two buffers (in place it ran slower)
}

// ---------------------------------------------------------------------------- y pass
// block (mode-column tile, z, component), in place; the FP32 pass at four blocks per SM
template <typename R, int SGN>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 4 : 0) k_spec_y(Spec<R> V, const CgScal* S) {
  using C = typename CxOf<R>::T;
  if (spec_skip<R>(S)) return;
  const int tx = V.tx, ltx = ilog2(tx);
  C* tw = smem_cx<C>();
  C* a = tw + V.ny;
  C* b = spec_y_buffers(V.ny) == 1 ? a : a + (size_t)tx * V.ny;   // one or two stages: b only
  load_roots(tw, V.tw[1], V.ny);
  const int kx0 = blockIdx.x * tx, z = blockIdx.y, comp = blockIdx.z;
  const ColIO<C> io{V.W + ((size_t)comp * V.nz + z) * V.ny * V.nxp + kx0, V.nxp,
                    min(tx, V.nxh - kx0)};
  fft_global_inplace<SGN>(io, a, b, 1, tx, ilog2(V.ny), ltx, 1, tw);
}

// ---------------------------------------------------------------------------- z pass
// block (mode-column tile, ky): the three components' z columns; forward transform, the
// constant-coefficient inverse per mode, inverse transform; in place
template <typename R>
__global__ void __launch_bounds__(NT) k_spec_z(Spec<R> V, CgScal* S) {
  using C = typename CxOf<R>::T;
  if (spec_skip<R>(S)) return;
  const int tz = V.tz, ltz = ilog2(tz), lw = 3 * tz;   // lines: (component, column)
  C* tw = smem_cx<C>();
  C* a = tw + V.nz;
  C* b = a + (size_t)lw * V.nz;
  load_roots(tw, V.tw[2], V.nz);
  const int kx0 = blockIdx.x * tz, ky = blockIdx.y;
  const int ncol = min(tz, V.nxh - kx0);
  const size_t plane = (size_t)V.ny * V.nxp, comp_stride = (size_t)V.nz * plane;
  const ZIO<C> io{V.W + (size_t)ky * V.nxp + kx0, plane, comp_stride, tz, ltz, ncol};
  C* F = fft_from_global<-1>(io, a, b, 1, lw, ilog2(V.nz), ltz, 3, tw);
  C* other = F == a ? b : a;
  const R mu0 = (R)V.mean[0], lam0 = (R)V.mean[1], eta0 = (R)V.mean[2];
  const R c = lam0 + mu0;
  const R inv_vol = (R)(1.0 / ((double)V.nx * V.ny * V.nz));
  const R Sy = V.S[1][ky], Ty = V.T[1][ky];
  // <r, z> by Parseval: sum over modes of conj(r^) z^ (z^ already carries 1/V), each stored
  // mode with 0 < kx < nx/2 standing for its conjugate as well; every term is >= 0
  R rz_part = (R)0;
  for (int idx = threadIdx.x; idx < tz * V.nz; idx += blockDim.x) {
    const int kz = idx >> ltz, col = idx & (tz - 1);
    if (col >= ncol) continue;
    const int kx = kx0 + col;
    const R Sv[3] = {V.S[0][kx], Sy, V.S[2][kz]};
    const R Tv[3] = {V.T[0][kx], Ty, V.T[2][kz]};
    const R base = eta0 + mu0 * (Sv[0] + Sv[1] + Sv[2]);
    C y[3];
    R tdt = (R)0;                             // T^T D^{-1} T
    C s = {(R)0, (R)0};                       // T^T D^{-1} r
    R dinv[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const R D = base + c * (Sv[q] - Tv[q] * Tv[q]);
      dinv[q] = D > (R)0 ? (R)1 / D : (R)0;   // D = 0 only for the mean mode when eta0 = 0
      const C rq = F[(size_t)kz * lw + q * tz + col];
      y[q] = C{rq.x * dinv[q], rq.y * dinv[q]};
      tdt += Tv[q] * Tv[q] * dinv[q];
      s.x += Tv[q] * y[q].x;
      s.y += Tv[q] * y[q].y;
    }
    const R f = c / ((R)1 + c * tdt);
    const R wgt = (kx == 0 || kx == V.nx / 2) ? (R)1 : (R)2;   // conjugate modes not stored
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const R g = f * Tv[q] * dinv[q];
      const C rq = F[(size_t)kz * lw + q * tz + col];
      const C zq = C{(y[q].x - g * s.x) * inv_vol, (y[q].y - g * s.y) * inv_vol};
      rz_part += wgt * (rq.x * zq.x + rq.y * zq.y);
      F[(size_t)kz * lw + q * tz + col] = zq;
    }
  }
  __syncthreads();
  fft_to_global<+1>(F, other, io, 1, lw, ilog2(V.nz), ltz, 3, tw);
  if (S == nullptr) return;
  double out;
  if (block_sum_last((double)rz_part, V.partial, V.counter, blockIdx.y * gridDim.x + blockIdx.x,
                     gridDim.x * gridDim.y, out))
    cg_after_precond(*S, out);
}

// ------------------------------------------------------------- z pass, in registers (FP32)
// For nz = 16 P (P = 8 or 16) each column's transforms run in registers.  A block takes
// ZR_COLS mode columns kx at one ky with P threads per column; thread t of a column loads the
// elements kz = t + P m (m < 16) of a component.  Forward transform, four-step with
// nz = 16 x P:
//   A[t][k2] = sum_m x[t + P m] exp(-2 pi i m k2 / 16)        DFT16 in registers
//   B[t][k2] = A[t][k2] exp(-2 pi i t k2 / nz)                 twiddle
//   X[k2 + 16 k1] = sum_t B[t][k2] exp(-2 pi i t k1 / P)       DFT_P after an exchange
// The exchange goes through shared memory: thread t then owns the J = 16 / P columns
// k2 = t + P j and holds the modes kz = k2 + 16 k1.  The inverse transform retraces the steps
// (inverse DFT_P, exchange back, conjugate twiddle, inverse DFT16), so every element crosses
// shared memory twice per component instead of four times.  A thread holds one component in
// registers at a time: the spectra of components 0 and 1 wait in thread-private shared-memory
// slots while component 2 is transformed, the 3x3 inverse reads them back mode by mode, and
// component 2 stays in registers from its forward to its inverse transform.  Consecutive
// threads take consecutive columns, so a warp's loads and stores of one plane are rows of W.
constexpr int ZR_COLS = 8;

// exchange buffer: 16 rows k2 of P x ZR_COLS elements, padded by ZR_COLS so that the column
// groups t and t + 1 of a half-warp fall in different banks
template <int P>
__host__ __device__ constexpr int zr_row() { return (P + 1) * ZR_COLS; }
template <int P>
constexpr size_t spec_smem_zr() {   // twiddles, the exchange buffer, two components' spectra
  return (size_t)(16 * P + 16 * zr_row<P>() + 2 * 16 * ZR_COLS * P) * sizeof(float2);
}

template <int P>
__global__ void __launch_bounds__(ZR_COLS * P, 512 / (ZR_COLS * P))
    k_spec_zr(Spec<float> V, CgScal* S) {
  using C = float2;
  constexpr int N = 16 * P, J = 16 / P, LP = P == 16 ? 4 : (P == 8 ? 3 : 2);
  constexpr int NTH = ZR_COLS * P;
  static_assert(P == 4 || P == 8 || P == 16, "nz = 64, 128 or 256");
  if (spec_skip<float>(S)) return;
  C* tw = smem_cx<C>();
  C* xb = tw + N;                       // exchange buffer
  C* held = xb + 16 * zr_row<P>();      // spectra of components 0 and 1: [q][i][thread]
  load_roots(tw, V.tw[2], N);
  const int c = threadIdx.x % ZR_COLS, t = threadIdx.x / ZR_COLS;
  const int kx = blockIdx.x * ZR_COLS + c, ky = blockIdx.y;
  const bool valid = kx < V.nxh;
  // element offsets stay below 3 nz ny nxp < 2^31 for nz <= 256
  const int plane = V.ny * V.nxp, comp_stride = N * plane;
  C* col = V.W + ky * V.nxp + (valid ? kx : 0) + t * plane;
  auto slot = [&](int k2, int tt) { return k2 * zr_row<P>() + tt * ZR_COLS + c; };
  auto hslot = [&](int q, int i) { return (q * 16 + i) * NTH + (int)threadIdx.x; };
  C v[16];

  // forward transform of component q: modes kz = t + P j + 16 k1 end at v[j P + k1]
  auto forward = [&](int q) {
    const C* src = col + q * comp_stride;
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = valid ? src[P * m * plane] : C{0.0f, 0.0f};
    if (q == 0) __syncthreads();   // twiddles visible
    dft<4, -1>(v);
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], tw[t * k2]);
    if (q > 0) __syncthreads();    // the previous exchange has been read
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) xb[slot(k2, t)] = v[k2];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int u = 0; u < P; ++u) v[j * P + u] = xb[slot(t + P * j, u)];
#pragma unroll
    for (int j = 0; j < J; ++j) dft<LP, -1>(*reinterpret_cast<C(*)[P]>(&v[j * P]));
  };
  // inverse transform of the modes in v (component q) and the store of its elements
  auto inverse = [&](int q) {
#pragma unroll
    for (int j = 0; j < J; ++j) dft<LP, +1>(*reinterpret_cast<C(*)[P]>(&v[j * P]));
    __syncthreads();               // the previous exchange has been read
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int u = 0; u < P; ++u) xb[slot(t + P * j, u)] = v[j * P + u];
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) v[k2] = xb[slot(k2, t)];
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], root<+1>(tw, t * k2));
    dft<4, +1>(v);
    if (valid) {
      C* dst = col + q * comp_stride;
#pragma unroll
      for (int m = 0; m < 16; ++m) dst[P * m * plane] = v[m];
    }
  };

#pragma unroll
  for (int q = 0; q < 2; ++q) {
    forward(q);
#pragma unroll
    for (int i = 0; i < 16; ++i) held[hslot(q, i)] = v[i];
  }
  forward(2);

  // the 3x3 inverse per mode (as in k_spec_z; reciprocals to FP32 accuracy suffice for a
  // preconditioner) and the Parseval term of <r, z>
  const float mu0 = (float)V.mean[0], lam0 = (float)V.mean[1], eta0 = (float)V.mean[2];
  const float cc = lam0 + mu0;
  const float inv_vol = (float)(1.0 / ((double)V.nx * V.ny * V.nz));
  const float Sx = V.S[0][valid ? kx : 0], Tx = V.T[0][valid ? kx : 0];
  const float Sy = V.S[1][ky], Ty = V.T[1][ky];
  const float wgt = !valid ? 0.0f : ((kx == 0 || kx == V.nx / 2) ? 1.0f : 2.0f);
  float rz_part = 0.0f;
#pragma unroll
  for (int j = 0; j < J; ++j) {
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      const int i = j * P + k1, kz = t + P * j + 16 * k1;
      const float Sv[3] = {Sx, Sy, __ldg(V.S[2] + kz)};
      const float Tv[3] = {Tx, Ty, __ldg(V.T[2] + kz)};
      const float base = eta0 + mu0 * (Sv[0] + Sv[1] + Sv[2]);
      const C rv[3] = {held[hslot(0, i)], held[hslot(1, i)], v[i]};
      float tdt = 0.0f, dinv[3];
      C y[3], s = {0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float D = base + cc * (Sv[q] - Tv[q] * Tv[q]);
        dinv[q] = D > 0.0f ? __fdividef(1.0f, D) : 0.0f;
        y[q] = C{rv[q].x * dinv[q], rv[q].y * dinv[q]};
        tdt += Tv[q] * Tv[q] * dinv[q];
        s.x += Tv[q] * y[q].x;
        s.y += Tv[q] * y[q].y;
      }
      const float f = __fdividef(cc, 1.0f + cc * tdt);
      C zv[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float g = f * Tv[q] * dinv[q];
        zv[q] = C{(y[q].x - g * s.x) * inv_vol, (y[q].y - g * s.y) * inv_vol};
        rz_part += wgt * (rv[q].x * zv[q].x + rv[q].y * zv[q].y);
      }
      held[hslot(0, i)] = zv[0];
      held[hslot(1, i)] = zv[1];
      v[i] = zv[2];
    }
  }

  inverse(2);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = held[hslot(q, i)];
    inverse(q);
  }
  if (S == nullptr) return;
  double out;
  if (block_sum_last((double)rz_part, V.partial, V.counter, blockIdx.y * gridDim.x + blockIdx.x,
                     gridDim.x * gridDim.y, out))
    cg_after_precond(*S, out);
}

// ------------------------------------------------- z pass, tiles staged by TMA (FP32)
// The register z pass above with its global traffic moved to the tensor-memory accelerator:
// one thread issues three bulk tensor copies (the block's ZR_COLS mode columns at one ky, all
// nz planes, one component each) that land in shared memory and complete on an mbarrier; the
// threads transform from and back into that tile, a thread's elements staying in its own slots
// of the tile between the forward transform, the 3x3 inverse and the inverse transform (the
// forward transform leaves the modes of a column thread on the planes it loaded); three bulk
// tensor stores write the tile back.  No global load or store is issued by the threads, and
// nothing of the tile is held in registers across the copies.  Waits on the mbarrier are
// bounded in time; a wait that gives up marks the solve CG_TIMEOUT and returns.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// true once the phase completed; false after limit_ns
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 63 && globaltimer_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, int c0, int c1, int c2,
                                             int c3, const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
      ::"l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit_and_wait() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr uint64_t ZR_WAIT_NS = 2000000000ull;   // 2 s for a tile that takes microseconds

template <int P>
constexpr size_t spec_smem_zr_tma() {   // tile (3 components), twiddles, S_z and T_z, barrier
  return (size_t)(3 * 16 * P * ZR_COLS + 16 * P) * sizeof(float2) + 2 * 16 * P * sizeof(float) +
         16;
}

template <int P>
__global__ void __launch_bounds__(ZR_COLS * P)
    k_spec_zr_tma(const __grid_constant__ CUtensorMap map, Spec<float> V, CgScal* S) {
  using C = float2;
  constexpr int N = 16 * P, J = 16 / P, LP = P == 16 ? 4 : (P == 8 ? 3 : 2);
  constexpr int TILE = N * ZR_COLS;            // elements of one component
  static_assert(P == 8 || P == 16, "nz = 128 or 256");
  if (spec_skip<float>(S)) return;
  extern __shared__ __align__(1024) unsigned char zr_smem[];
  C* tile = reinterpret_cast<C*>(zr_smem);     // [component][plane][column]
  C* tw = tile + 3 * TILE;
  float* Sz = reinterpret_cast<float*>(tw + N);   // the z symbols S_z, T_z of the N modes
  float* Tz = Sz + N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Tz + N);
  const int c = threadIdx.x % ZR_COLS, t = threadIdx.x / ZR_COLS;
  const int kx0 = blockIdx.x * ZR_COLS, ky = blockIdx.y;
  const bool valid = kx0 + c < V.nxh;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, 3u * TILE * (uint32_t)sizeof(C));
#pragma unroll
    for (int q = 0; q < 3; ++q) tma_load_4d(tile + q * TILE, &map, kx0, ky, 0, q, bar);
  }
  load_roots(tw, V.tw[2], N);
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    Sz[k] = V.S[2][k];
    Tz[k] = V.T[2][k];
  }
  __syncthreads();                             // barrier initialised, tables visible
  if (!mbar_wait_bounded(bar, 0, ZR_WAIT_NS)) {
    if (threadIdx.x == 0) S->status = CG_TIMEOUT;
    mbar_wait_bounded(bar, 0, ZR_WAIT_NS);     // the copies in flight target this tile
    return;
  }
  auto el = [&](int q, int z) -> C& { return tile[q * TILE + z * ZR_COLS + c]; };
  // The four-step transform's exchange runs in place, in the component's own tile region
  // (no separate buffer: 50 KB per block instead of 69 KB, four blocks per SM instead of
  // three): element (row, col) of the exchange, 16 rows of P x ZR_COLS, sits at
  // row * P * ZR_COLS + ((col * ZR_COLS + c) ^ 8 (row & 1)).  The swizzle moves odd rows by
  // half a 16-element bank group, so the two rows a half-warp reads at once fall in different
  // banks (without it the transposed reads conflict two ways).
  auto xpos = [&](int q, int row, int col) {
    return q * TILE + row * (P * ZR_COLS) + ((col * ZR_COLS + c) ^ ((row & 1) << 3));
  };
  C v[16];

  // forward transform of component q (four-step, nz = 16 x P, as in k_spec_zr): the modes
  // kz = t + P j + 16 k1 land in v[j P + k1] and are kept on the planes kz of the tile
  auto forward = [&](int q) {
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = el(q, t + P * m);
    dft<4, -1>(v);
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], tw[t * k2]);
    __syncthreads();                           // every thread has read component q
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) tile[xpos(q, k2, t)] = v[k2];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int u = 0; u < P; ++u) v[j * P + u] = tile[xpos(q, t + P * j, u)];
#pragma unroll
    for (int j = 0; j < J; ++j) dft<LP, -1>(*reinterpret_cast<C(*)[P]>(&v[j * P]));
    __syncthreads();                           // every thread has read the exchange
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) el(q, t + P * j + 16 * k1) = v[j * P + k1];
  };
  auto inverse = [&](int q) {
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) v[j * P + k1] = el(q, t + P * j + 16 * k1);
#pragma unroll
    for (int j = 0; j < J; ++j) dft<LP, +1>(*reinterpret_cast<C(*)[P]>(&v[j * P]));
    __syncthreads();                           // every thread has read component q
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int u = 0; u < P; ++u) tile[xpos(q, t + P * j, u)] = v[j * P + u];
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) v[k2] = tile[xpos(q, k2, t)];
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], root<+1>(tw, t * k2));
    dft<4, +1>(v);
    __syncthreads();                           // every thread has read the exchange
#pragma unroll
    for (int m = 0; m < 16; ++m) el(q, t + P * m) = v[m];
  };

#pragma unroll 1
  for (int q = 0; q < 3; ++q) forward(q);

  // the 3x3 inverse per mode (as in k_spec_zr) and the Parseval term of <r, z>; columns past
  // nx/2 (row padding, whatever they hold) take no part in the sum
  const int kx = valid ? kx0 + c : 0;
  const float mu0 = (float)V.mean[0], lam0 = (float)V.mean[1], eta0 = (float)V.mean[2];
  const float cc = lam0 + mu0;
  const float inv_vol = 1.0f / ((float)V.nx * (float)V.ny * (float)V.nz);
  const float Sx = V.S[0][kx], Tx = V.T[0][kx];
  const float Sy = V.S[1][ky], Ty = V.T[1][ky];
  const float wgt = (kx == 0 || kx == V.nx / 2) ? 1.0f : 2.0f;
  float rz_part = 0.0f;
#pragma unroll
  for (int j = 0; j < J; ++j) {
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      const int kz = t + P * j + 16 * k1;
      const float Sv[3] = {Sx, Sy, Sz[kz]};
      const float Tv[3] = {Tx, Ty, Tz[kz]};
      const float base = eta0 + mu0 * (Sv[0] + Sv[1] + Sv[2]);
      const C rv[3] = {el(0, kz), el(1, kz), el(2, kz)};
      float tdt = 0.0f, dinv[3];
      C y[3], s = {0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float D = base + cc * (Sv[q] - Tv[q] * Tv[q]);
        dinv[q] = D > 0.0f ? __fdividef(1.0f, D) : 0.0f;
        y[q] = C{rv[q].x * dinv[q], rv[q].y * dinv[q]};
        tdt += Tv[q] * Tv[q] * dinv[q];
        s.x += Tv[q] * y[q].x;
        s.y += Tv[q] * y[q].y;
      }
      const float f = __fdividef(cc, 1.0f + cc * tdt);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float g = f * Tv[q] * dinv[q];
        const C zq = C{(y[q].x - g * s.x) * inv_vol, (y[q].y - g * s.y) * inv_vol};
        if (valid) rz_part += wgt * (rv[q].x * zq.x + rv[q].y * zq.y);
        el(q, kz) = zq;
      }
    }
  }

#pragma unroll 1
  for (int q = 0; q < 3; ++q) inverse(q);
  fence_proxy_async_smem();                    // the tile's writes, visible to the copies
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) tma_store_4d(&map, kx0, ky, 0, q, tile + q * TILE);
    bulk_commit_and_wait();
  }
  double out;
  if (block_sum_last((double)rz_part, V.partial, V.counter, blockIdx.y * gridDim.x + blockIdx.x,
                     gridDim.x * gridDim.y, out))
    cg_after_precond(*S, out);
}

// ---------------------------------------------------------------------------- x inverse
// block (pair tile, z, component): the half spectra of rows y0 + 2l, y0 + 2l + 1 form
// C[k] = A[k] + i B[k] over all k (Hermitian extension); the inverse transform is
// a + i b.  Writes z = s (inverse transform) (s = 1 unscaled), or with PU the new search
// direction p = z + beta p_old (beta = 0 on a solve's first iteration).
template <typename R, bool PUP, int FORM>
__global__ void __launch_bounds__(NT, PUP ? 4 : 2) k_spec_x_inv(Spec<R> V, R* z0, R* z1, R* z2,
                                                                const CgScal* S, PUpd<R> PU) {
  using C = typename CxOf<R>::T;
  if (spec_skip<R>(S)) return;
  const int n = V.nx, ln = ilog2(n), half = n / 2, pb = V.pb, es = pb + 1;
  C* tw = smem_cx<C>();
  C* a = tw + n;
  C* b = a + (size_t)es * n;
  load_roots(tw, V.tw[0], n);
  const int comp = blockIdx.z, z = blockIdx.y, y0 = 2 * V.pb * blockIdx.x;
  const C* W = V.W + (((size_t)comp * V.nz + z) * V.ny + y0) * V.nxp;
  const int total = pb * n;
  for (int i0 = threadIdx.x; i0 < total; i0 += LB * blockDim.x) {
    C A[LB], B[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) {
        const int l = idx >> ln, k = idx & (n - 1);
        const int kk = k <= half ? k : n - k;
        A[u] = __ldg(W + (size_t)(2 * l) * V.nxp + kk);
        B[u] = __ldg(W + (size_t)(2 * l + 1) * V.nxp + kk);
      }
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) {
        const int l = idx >> ln, k = idx & (n - 1);
        C a_ = A[u], b_ = B[u];
        if (k == 0 || k == half) {
          a_.y = (R)0;
          b_.y = (R)0;
        } else if (k > half) {
          a_.y = -a_.y;
          b_.y = -b_.y;
        }
        a[k * es + l] = C{a_.x - b_.y, a_.y + b_.x};
      }
    }
  }
  __syncthreads();
  const C* F = fft_x<+1, FORM>(V.x_inpl != 0, a, b, ln, ilog2(pb), es, tw);
  R* out = comp == 0 ? z0 : (comp == 1 ? z1 : z2);
  const R* pold = nullptr;
  R beta = (R)0;
  if (PUP) {   // selects written out: no indexed copy of the parameter arrays
    const int it = S->it;
    R* const p0 = comp == 0 ? PU.p[0][0] : (comp == 1 ? PU.p[0][1] : PU.p[0][2]);
    R* const p1 = comp == 0 ? PU.p[1][0] : (comp == 1 ? PU.p[1][1] : PU.p[1][2]);
    out = (it & 1) ? p0 : p1;
    if (it > 0) {
      pold = (it & 1) ? p1 : p0;
      beta = (R)S->beta;
    }
  }
  const R* sc = V.s[comp];   // z = s A0^{-1} (s r) with the scaled preconditioner
  const size_t row0 = ((size_t)z * V.ny + y0) * n;
  for (int i0 = threadIdx.x; i0 < total; i0 += LB * blockDim.x) {   // LB loads in flight
    R sa[LB], sb[LB], pa[LB], pbv[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) {
        const size_t o = row0 + (size_t)(2 * (idx >> ln)) * n + (idx & (n - 1));
        sa[u] = sc ? __ldg(sc + o) : (R)1;
        sb[u] = sc ? __ldg(sc + o + n) : (R)1;
        pa[u] = (PUP && pold) ? pold[o] : (R)0;
        pbv[u] = (PUP && pold) ? pold[o + n] : (R)0;
      }
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < total) {
        const int l = idx >> ln, x = idx & (n - 1);
        const size_t o = row0 + (size_t)(2 * l) * n + x;
        const C f = F[x * es + l];
        out[o] = PUP ? f.x * sa[u] + beta * pa[u] : f.x * sa[u];
        out[o + n] = PUP ? f.y * sb[u] + beta * pbv[u] : f.y * sb[u];
      }
    }
  }
}

// ---------------------------------------------------------------------------- tables, means
template <typename R>
__global__ void k_spec_tables(Spec<R> V, double h0, double h1, double h2) {
  using C = typename CxOf<R>::T;
  const int d = blockIdx.y;
  const int n = d == 0 ? V.nx : (d == 1 ? V.ny : V.nz);
  const double h = d == 0 ? h0 : (d == 1 ? h1 : h2);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double s, c, sh, ch;
    sincospi(2.0 * k / n, &s, &c);        // theta = 2 pi k / n
    sincospi((double)k / n, &sh, &ch);    // theta / 2
    V.tw[d][k] = C{(R)c, (R)-s};
    V.S[d][k] = (R)(4.0 * sh * sh / (h * h));
    V.T[d][k] = (R)(s / h);
  }
}

template <bool F32>
__global__ void __launch_bounds__(NT) k_spec_mean(long long n, const double* __restrict__ mu,
                                                  const double* __restrict__ lam,
                                                  const double* __restrict__ eta, double* mean,
                                                  double* partial, unsigned int* counter) {
  // F32 (the mixed precision): a thread's terms summed in FP32 from FP32 values converted on
  // the integer pipes (the means only shape the preconditioner), threads and blocks in FP64;
  // otherwise every term in FP64, as the oracle forms the means
  double acc[3] = {0.0, 0.0, 0.0};
  float fa[3] = {0.0f, 0.0f, 0.0f};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    if (F32) {
      fa[0] += f32_of(mu[e]);
      fa[1] += f32_of(lam[e]);
      fa[2] += f32_of(eta[e]);
    } else {
      acc[0] += mu[e];
      acc[1] += lam[e];
      acc[2] += eta[e];
    }
  }
  if (F32) {
    acc[0] = (double)fa[0];
    acc[1] = (double)fa[1];
    acc[2] = (double)fa[2];
  }
  double out[3];
  if (reduce_indexed<3>(acc, partial, counter, blockIdx.x, gridDim.x, out) && threadIdx.x == 0) {
    mean[0] = out[0] / (double)n;
    mean[1] = out[1] / (double)n;
    mean[2] = out[2] / (double)n;
  }
}

// Diagonal scaling of TG_PRECOND_SPECTRAL_SCALED: s_a = (D0_a / D_a)^{1/2} per node, D_a the
// Jacobi diagonal of the variable-coefficient operator (FP64, or (hi, lo) pairs with the
// double-FP32 residual) and D0_a = eta0 + 2 (lambda0 + 2 mu0) / h_a^2 + 2 mu0 sum_{d != a}
// 1 / h_d^2 that of the constant-coefficient operator.  The FP32 form is evaluated in FP32.
template <typename R>
__global__ void __launch_bounds__(NT) k_spec_scale(long long n, Spec<R> V, Elas E, double ih20,
                                                   double ih21, double ih22) {
  const double mu0 = V.mean[0], lam0 = V.mean[1], eta0 = V.mean[2];
  const double ih2[3] = {ih20, ih21, ih22};
  R d0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double v = eta0;
#pragma unroll
    for (int d = 0; d < 3; ++d) v += 2.0 * (d == a ? lam0 + 2.0 * mu0 : mu0) * ih2[d];
    d0[a] = (R)v;
  }
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R D;
      if (E.df) {
        const float2 h = reinterpret_cast<const float2*>(E.dsum[a])[e];
        D = sizeof(R) == 4 ? (R)h.x : (R)((double)h.x + (double)h.y);
      } else {
        D = (R)E.dsum[a][e];
      }
      V.s[a][e] = sqrt(d0[a] / D);
    }
  }
}

}  // namespace

// Every pass kernel may use up to the device's opt-in shared memory per block, less 1 KB for
// the kernels' static shared memory (the attribute is a limit, not a reservation), so
// contexts of different grid sizes never lower it for one another; V's own needs must fit.
template <typename R>
cudaError_t spec_prepare(const Spec<R>& V) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  optin -= 1024;
  if (spec_smem_x2(V) > (size_t)optin || spec_smem_y(V) > (size_t)optin ||
      spec_smem_z(V) > (size_t)optin)
    return cudaErrorInvalidValue;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  e = cudaFuncSetAttribute(k_spec_x_fwd<R>, A, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_update_xfwd, A, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_x_inv<R, false, 2>, A, optin);
  if constexpr (sizeof(R) == 4) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_x_inv<R, true, 0>, A, optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_x_inv<R, true, 1>, A, optin);
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_y<R, -1>, A, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_y<R, +1>, A, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_z<R>, A, optin);
  if constexpr (sizeof(R) == 4) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_zr<16>, A, optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_zr<8>, A, optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_zr_tma<16>, A, optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_zr_tma<8>, A, optin);
  }
  return e;
}

// W as a 4-D tensor of 8-byte elements (x modes with the row pitch nxp, y, z, component); box:
// ZR_COLS modes x 1 row x all nz planes x 1 component.  The base is 256-byte aligned, the
// strides multiples of 16 bytes (nxp is a multiple of 16 modes), the box's inner extent
// ZR_COLS * 8 = 64 bytes, and the kernel's x coordinates multiples of ZR_COLS (64 bytes).
bool spec_make_zmap(const Spec<float>& V, void* map) {
  if (V.nz != 128 && V.nz != 256) return false;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr)
    return false;
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint64_t dims[4] = {(cuuint64_t)V.nxp, (cuuint64_t)V.ny, (cuuint64_t)V.nz, 3};
  const cuuint64_t row = (cuuint64_t)V.nxp * sizeof(float2);
  const cuuint64_t strides[3] = {row, row * V.ny, row * V.ny * V.nz};
  const cuuint32_t box[4] = {(cuuint32_t)ZR_COLS, 1, (cuuint32_t)V.nz, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  if ((reinterpret_cast<uintptr_t>(V.W) & 15) != 0 || (row & 15) != 0) return false;
  return encode(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, V.W, dims,
                strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename R>
cudaError_t launch_spec_scale(const Geo& G, const Spec<R>& V, const Elas& E, cudaStream_t st) {
  const long long want = (G.nvox + NT - 1) / NT;
  const int blocks = (int)(want < 4096 ? (want > 0 ? want : 1) : 4096);
  TG_TIMED(K_SPEC_SCALE, st,
           k_spec_scale<R><<<blocks, NT, 0, st>>>(G.nvox, V, E, G.ih2[0], G.ih2[1], G.ih2[2]));
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_spec_tables(const Spec<R>& V, const double h[3], cudaStream_t st) {
  const int nmax = max(V.nx, max(V.ny, V.nz));
  k_spec_tables<R><<<dim3((nmax + 127) / 128, 3), 128, 0, st>>>(V, h[0], h[1], h[2]);
  return cudaGetLastError();
}

cudaError_t launch_spec_mean(long long n, const double* mu, const double* lam,
                             const double* eta, double* mean, double* partial,
                             unsigned int* counter, cudaStream_t st, bool fp32_terms) {
  const long long want = (n + NT - 1) / NT;
  const int blocks = (int)(want < 1024 ? (want > 0 ? want : 1) : 1024);
  if (fp32_terms)
    TG_TIMED(K_SPEC_MEAN, st,
             k_spec_mean<true><<<blocks, NT, 0, st>>>(n, mu, lam, eta, mean, partial, counter));
  else
    TG_TIMED(K_SPEC_MEAN, st,
             k_spec_mean<false><<<blocks, NT, 0, st>>>(n, mu, lam, eta, mean, partial, counter));
  return cudaGetLastError();
}

// the z pass: for FP32 and nz = 128 or 256 in registers, from tiles staged by TMA when the
// context made the tensor map (and the pass updates a solve's scalars), else from global
// memory; staged through shared memory otherwise
template <typename R>
void launch_spec_z(const Spec<R>& V, CgScal* S, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    const dim3 g((V.nxh + ZR_COLS - 1) / ZR_COLS, V.ny);
    if (V.zmap != nullptr && S != nullptr && (V.nz == 256 || V.nz == 128)) {
      const CUtensorMap& map = *static_cast<const CUtensorMap*>(V.zmap);
      if (V.nz == 256)
        TG_TIMED(K_SPEC_ZR, st,
                 k_spec_zr_tma<16><<<g, 16 * ZR_COLS, spec_smem_zr_tma<16>(), st>>>(map, V, S));
      else
        TG_TIMED(K_SPEC_ZR, st,
                 k_spec_zr_tma<8><<<g, 8 * ZR_COLS, spec_smem_zr_tma<8>(), st>>>(map, V, S));
      return;
    }
    if (V.nz == 256) {
      TG_TIMED(K_SPEC_ZR, st, k_spec_zr<16><<<g, 16 * ZR_COLS, spec_smem_zr<16>(), st>>>(V, S));
      return;
    }
    if (V.nz == 128) {
      TG_TIMED(K_SPEC_ZR, st, k_spec_zr<8><<<g, 8 * ZR_COLS, spec_smem_zr<8>(), st>>>(V, S));
      return;
    }
  }
  const dim3 gz((V.nxh + V.tz - 1) / V.tz, V.ny);
  TG_TIMED(K_SPEC_Z, st, k_spec_z<R><<<gz, V.nt_z, spec_smem_z(V), st>>>(V, S));
}

template <typename R>
cudaError_t launch_spectral(const Spec<R>& V, const R* const r[3], R* const z[3], CgScal* S,
                            cudaStream_t st, const PUpd<R>* pu) {
  const dim3 gx(V.ny / (2 * V.pb), V.nz, 3);
  const dim3 gy((V.nxh + V.tx - 1) / V.tx, V.nz, 3);
  TG_TIMED(K_SPEC_X_FWD, st,
           k_spec_x_fwd<R><<<gx, NT, spec_smem_x(V), st>>>(V, r[0], r[1], r[2], S));
  TG_TIMED(K_SPEC_Y_FWD, st, k_spec_y<R, -1><<<gy, NT, spec_smem_y(V), st>>>(V, S));
  launch_spec_z(V, S, st);
  TG_TIMED(K_SPEC_Y_INV, st, k_spec_y<R, +1><<<gy, NT, spec_smem_y(V), st>>>(V, S));
  PUpd<R> P = {};
  if constexpr (sizeof(R) == 4) {
    if (pu) {
      P = *pu;
      if (V.x_inpl)
        TG_TIMED(K_SPEC_X_INV_P, st,
                 k_spec_x_inv<R, true, 1><<<gx, NT, spec_smem_x(V), st>>>(V, z[0], z[1], z[2], S, P));
      else
        TG_TIMED(K_SPEC_X_INV_P, st,
                 k_spec_x_inv<R, true, 0><<<gx, NT, spec_smem_x(V), st>>>(V, z[0], z[1], z[2], S, P));
      return cudaGetLastError();
    }
  }
  TG_TIMED(K_SPEC_X_INV, st,
           k_spec_x_inv<R, false, 2><<<gx, NT, spec_smem_x(V), st>>>(V, z[0], z[1], z[2], S, P));
  return cudaGetLastError();
}

// one preconditioned CG iteration's update and preconditioner (mixed precision): the fused
// update + x forward pass, then the remaining four passes
cudaError_t launch_spectral_update(const Spec<float>& V, const Elas32& I, float* const z[3],
                                   cudaStream_t st) {
  const dim3 gx(V.ny / (2 * V.pb), V.nz, 3);
  const dim3 gy((V.nxh + V.tx - 1) / V.tx, V.nz, 3);
  TG_TIMED(K_SPEC_UPDATE_XFWD, st, k_spec_update_xfwd<<<gx, NT, spec_smem_x2(V), st>>>(V, I));
  TG_TIMED(K_SPEC_Y_FWD, st, k_spec_y<float, -1><<<gy, NT, spec_smem_y(V), st>>>(V, I.S));
  launch_spec_z(V, I.S, st);
  TG_TIMED(K_SPEC_Y_INV, st, k_spec_y<float, +1><<<gy, NT, spec_smem_y(V), st>>>(V, I.S));
  PUpd<float> P;   // p = z + beta p_old straight from the last pass
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 3; ++a) P.p[b][a] = I.p[b][a];
  if (V.x_inpl)
    TG_TIMED(K_SPEC_X_INV_P, st,
             k_spec_x_inv<float, true, 1><<<gx, NT, spec_smem_x(V), st>>>(V, z[0], z[1], z[2], I.S, P));
  else
    TG_TIMED(K_SPEC_X_INV_P, st,
             k_spec_x_inv<float, true, 0><<<gx, NT, spec_smem_x(V), st>>>(V, z[0], z[1], z[2], I.S, P));
  return cudaGetLastError();
}

template cudaError_t spec_prepare<float>(const Spec<float>&);
template cudaError_t spec_prepare<double>(const Spec<double>&);
template cudaError_t launch_spec_scale<float>(const Geo&, const Spec<float>&, const Elas&,
                                              cudaStream_t);
template cudaError_t launch_spec_scale<double>(const Geo&, const Spec<double>&, const Elas&,
                                               cudaStream_t);
template cudaError_t launch_spec_tables<float>(const Spec<float>&, const double[3], cudaStream_t);
template cudaError_t launch_spec_tables<double>(const Spec<double>&, const double[3], cudaStream_t);
template cudaError_t launch_spectral<float>(const Spec<float>&, const float* const[3],
                                            float* const[3], CgScal*, cudaStream_t,
                                            const PUpd<float>*);
template cudaError_t launch_spectral<double>(const Spec<double>&, const double* const[3],
                                             double* const[3], CgScal*, cudaStream_t,
                                             const PUpd<double>*);

}  // namespace tg
