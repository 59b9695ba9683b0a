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
//              inverse per mode (with the 1/V normalisation), inverse transform, in place;
//   y inverse  in place;
//   x inverse  the Hermitian half spectra of two rows form one complex line whose inverse
//              transform carries both real rows; writes z and reduces <r, z>.
// The 1-D transforms are Stockham autosort FFTs (radix 4, one radix-2 stage when log2 n is
// odd) ping-ponging between two shared-memory buffers, one barrier per stage.
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

// Transforms nl lines of length n (a power of two).  Element e of line l sits at
// a[l * ls + e * es]; b has the same shape and is scratch.  line_fast: consecutive threads
// take consecutive lines (lines interleaved in memory), else consecutive butterflies of one
// line.  Entry: a loaded and visible to the block.  Returns the buffer holding the result
// (visible to the block).
template <int SGN, typename C>
__device__ C* fft_lines(C* a, C* b, int n, int nl, int ls, int es, bool line_fast,
                        const C* __restrict__ tw) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int Ns = 1; Ns < n;) {
    const int R = ((n / Ns) & 3) == 0 ? 4 : 2;
    const int nb = n / R;               // butterflies per line
    const int ts = n / (Ns * R);        // twiddle table stride of this stage
    const int total = nl * nb;
    for (int it = tid; it < total; it += nthr) {
      int l, j;
      if (line_fast) {
        l = it % nl;
        j = it / nl;
      } else {
        j = it % nb;
        l = it / nb;
      }
      const int k = j % Ns;             // position inside the current sub-transform
      const int d = (j / Ns) * Ns * R + k;
      const C* src = a + (size_t)l * ls;
      C* dst = b + (size_t)l * ls;
      C v0 = src[(size_t)j * es], v1 = src[(size_t)(j + nb) * es];
      if (R == 4) {
        C v2 = src[(size_t)(j + 2 * nb) * es], v3 = src[(size_t)(j + 3 * nb) * es];
        if (k > 0) {
          v1 = cmul(v1, root<SGN>(tw, k * ts));
          v2 = cmul(v2, root<SGN>(tw, 2 * k * ts));
          v3 = cmul(v3, root<SGN>(tw, 3 * k * ts));
        }
        const C a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3);
        const C a3 = rot<SGN>(csub(v1, v3));
        dst[(size_t)d * es] = cadd(a0, a2);
        dst[(size_t)(d + Ns) * es] = cadd(a1, a3);
        dst[(size_t)(d + 2 * Ns) * es] = csub(a0, a2);
        dst[(size_t)(d + 3 * Ns) * es] = csub(a1, a3);
      } else {
        if (k > 0) v1 = cmul(v1, root<SGN>(tw, k * ts));
        dst[(size_t)d * es] = cadd(v0, v1);
        dst[(size_t)(d + Ns) * es] = csub(v0, v1);
      }
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

template <typename C> __device__ __forceinline__ C* smem_cx() {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return reinterpret_cast<C*>(smem_raw);
}

template <typename R>
__device__ __forceinline__ bool spec_skip(const CgScal* S) {
  return S != nullptr && S->status != CG_RUNNING;
}

// ---------------------------------------------------------------------------- x forward
// block (pair tile, z, component): rows y0 .. y0 + 2 pb - 1 of plane z
template <typename R>
__global__ void __launch_bounds__(NT) k_spec_x_fwd(Spec<R> V, const R* __restrict__ r0,
                                                   const R* __restrict__ r1,
                                                   const R* __restrict__ r2, const CgScal* S) {
  using C = typename CxOf<R>::T;
  if (spec_skip<R>(S)) return;
  C* a = smem_cx<C>();
  C* b = a + (size_t)V.pb * V.nx;
  const int comp = blockIdx.z, z = blockIdx.y, y0 = 2 * V.pb * blockIdx.x;
  const R* src = comp == 0 ? r0 : (comp == 1 ? r1 : r2);
  const size_t row0 = ((size_t)z * V.ny + y0) * V.nx;
  const int n = V.nx;
  for (int idx = threadIdx.x; idx < V.pb * n; idx += blockDim.x) {
    const int l = idx / n, x = idx - l * n;
    const size_t o = row0 + (size_t)(2 * l) * n + x;
    a[idx] = C{src[o], src[o + n]};
  }
  __syncthreads();
  const C* F = fft_lines<-1>(a, b, n, V.pb, n, 1, false, V.tw[0]);
  C* W = V.W + (((size_t)comp * V.nz + z) * V.ny + y0) * V.nxp;
  for (int idx = threadIdx.x; idx < V.pb * V.nxh; idx += blockDim.x) {
    const int l = idx / V.nxh, k = idx - l * V.nxh;
    const C f = F[(size_t)l * n + k], g = F[(size_t)l * n + ((n - k) & (n - 1))];
    // row 2l: (f + conj g) / 2;  row 2l+1: (f - conj g) / (2i)
    W[(size_t)(2 * l) * V.nxp + k] = C{(R)0.5 * (f.x + g.x), (R)0.5 * (f.y - g.y)};
    W[(size_t)(2 * l + 1) * V.nxp + k] = C{(R)0.5 * (f.y + g.y), (R)-0.5 * (f.x - g.x)};
  }
}

// ---------------------------------------------------------------------------- y pass
// block (mode-column tile, z, component), in place
template <typename R, int SGN>
__global__ void __launch_bounds__(NT) k_spec_y(Spec<R> V, const CgScal* S) {
  using C = typename CxOf<R>::T;
  if (spec_skip<R>(S)) return;
  C* a = smem_cx<C>();
  C* b = a + (size_t)V.tx * V.ny;
  const int kx0 = blockIdx.x * V.tx, z = blockIdx.y, comp = blockIdx.z;
  const int ncol = min(V.tx, V.nxh - kx0);
  C* W = V.W + ((size_t)comp * V.nz + z) * V.ny * V.nxp + kx0;
  const int tx = V.tx;
  for (int idx = threadIdx.x; idx < tx * V.ny; idx += blockDim.x) {
    const int y = idx / tx, col = idx - y * tx;
    a[idx] = col < ncol ? W[(size_t)y * V.nxp + col] : C{(R)0, (R)0};
  }
  __syncthreads();
  const C* F = fft_lines<SGN>(a, b, V.ny, tx, 1, tx, true, V.tw[1]);
  for (int idx = threadIdx.x; idx < tx * V.ny; idx += blockDim.x) {
    const int y = idx / tx, col = idx - y * tx;
    if (col < ncol) W[(size_t)y * V.nxp + col] = F[idx];
  }
}

// ---------------------------------------------------------------------------- z pass
// block (mode-column tile, ky): the three components' z columns; forward transform, the
// constant-coefficient inverse per mode, inverse transform; in place
template <typename R>
__global__ void __launch_bounds__(NT) k_spec_z(Spec<R> V, const CgScal* S) {
  using C = typename CxOf<R>::T;
  if (spec_skip<R>(S)) return;
  C* a = smem_cx<C>();
  C* b = a + (size_t)3 * V.tz * V.nz;
  const int kx0 = blockIdx.x * V.tz, ky = blockIdx.y;
  const int tz = V.tz, lw = 3 * tz;          // lines: (component, column), interleaved
  const int ncol = min(tz, V.nxh - kx0);
  const size_t plane = (size_t)V.ny * V.nxp, comp_stride = (size_t)V.nz * plane;
  C* W = V.W + (size_t)ky * V.nxp + kx0;
  for (int idx = threadIdx.x; idx < lw * V.nz; idx += blockDim.x) {
    const int kz = idx / lw, rem = idx - kz * lw, comp = rem / tz, col = rem - comp * tz;
    a[idx] = col < ncol ? W[comp * comp_stride + (size_t)kz * plane + col] : C{(R)0, (R)0};
  }
  __syncthreads();
  C* F = fft_lines<-1>(a, b, V.nz, lw, 1, lw, true, V.tw[2]);
  C* other = F == a ? b : a;
  const R mu0 = (R)V.mean[0], lam0 = (R)V.mean[1], eta0 = (R)V.mean[2];
  const R c = lam0 + mu0;
  const R inv_vol = (R)(1.0 / ((double)V.nx * V.ny * V.nz));
  const R Sy = V.S[1][ky], Ty = V.T[1][ky];
  for (int idx = threadIdx.x; idx < tz * V.nz; idx += blockDim.x) {
    const int kz = idx / tz, col = idx - kz * tz;
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
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const R g = f * Tv[q] * dinv[q];
      F[(size_t)kz * lw + q * tz + col] =
          C{(y[q].x - g * s.x) * inv_vol, (y[q].y - g * s.y) * inv_vol};
    }
  }
  __syncthreads();
  const C* G = fft_lines<+1>(F, other, V.nz, lw, 1, lw, true, V.tw[2]);
  for (int idx = threadIdx.x; idx < lw * V.nz; idx += blockDim.x) {
    const int kz = idx / lw, rem = idx - kz * lw, comp = rem / tz, col = rem - comp * tz;
    if (col < ncol) W[comp * comp_stride + (size_t)kz * plane + col] = G[idx];
  }
}

// ---------------------------------------------------------------------------- x inverse
// block (pair tile, z, component): the half spectra of rows y0 + 2l, y0 + 2l + 1 form
// C[k] = A[k] + i B[k] over all k (Hermitian extension); the inverse transform is
// a + i b.  Writes z and accumulates <r, z>; the last block finishes the CG scalars.
template <typename R>
__global__ void __launch_bounds__(NT) k_spec_x_inv(Spec<R> V, const R* __restrict__ r0,
                                                   const R* __restrict__ r1,
                                                   const R* __restrict__ r2, R* z0, R* z1,
                                                   R* z2, CgScal* S) {
  using C = typename CxOf<R>::T;
  if (spec_skip<R>(S)) return;
  C* a = smem_cx<C>();
  C* b = a + (size_t)V.pb * V.nx;
  const int comp = blockIdx.z, z = blockIdx.y, y0 = 2 * V.pb * blockIdx.x;
  const int n = V.nx, half = n / 2;
  const C* W = V.W + (((size_t)comp * V.nz + z) * V.ny + y0) * V.nxp;
  for (int idx = threadIdx.x; idx < V.pb * n; idx += blockDim.x) {
    const int l = idx / n, k = idx - l * n;
    const bool lower = k <= half;
    const int kk = lower ? k : n - k;
    C A = W[(size_t)(2 * l) * V.nxp + kk], B = W[(size_t)(2 * l + 1) * V.nxp + kk];
    if (k == 0 || k == half) {
      A.y = (R)0;
      B.y = (R)0;
    } else if (!lower) {
      A.y = -A.y;
      B.y = -B.y;
    }
    a[idx] = C{A.x - B.y, A.y + B.x};
  }
  __syncthreads();
  const C* F = fft_lines<+1>(a, b, n, V.pb, n, 1, false, V.tw[0]);
  const R* rs = comp == 0 ? r0 : (comp == 1 ? r1 : r2);
  R* zs = comp == 0 ? z0 : (comp == 1 ? z1 : z2);
  const size_t row0 = ((size_t)z * V.ny + y0) * n;
  double acc[1] = {0.0};
  R part = (R)0;
  for (int idx = threadIdx.x; idx < V.pb * n; idx += blockDim.x) {
    const int l = idx / n, x = idx - l * n;
    const size_t o = row0 + (size_t)(2 * l) * n + x;
    const C f = F[idx];
    zs[o] = f.x;
    zs[o + n] = f.y;
    part += rs[o] * f.x + rs[o + n] * f.y;
  }
  acc[0] = (double)part;
  if (S == nullptr) return;
  const int nb = gridDim.x * gridDim.y * gridDim.z;
  const int bl = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  double out[1];
  if (reduce_indexed<1>(acc, V.partial, V.counter, bl, nb, out) && threadIdx.x == 0)
    cg_after_precond(*S, out[0]);
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

__global__ void __launch_bounds__(NT) k_spec_mean(long long n, const double* __restrict__ mu,
                                                  const double* __restrict__ lam,
                                                  const double* __restrict__ eta, double* mean,
                                                  double* partial, unsigned int* counter) {
  double acc[3] = {0.0, 0.0, 0.0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    acc[0] += mu[e];
    acc[1] += lam[e];
    acc[2] += eta[e];
  }
  double out[3];
  if (reduce_indexed<3>(acc, partial, counter, blockIdx.x, gridDim.x, out) && threadIdx.x == 0) {
    mean[0] = out[0] / (double)n;
    mean[1] = out[1] / (double)n;
    mean[2] = out[2] / (double)n;
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
  if (spec_smem_x(V) > (size_t)optin || spec_smem_y(V) > (size_t)optin ||
      spec_smem_z(V) > (size_t)optin)
    return cudaErrorInvalidValue;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  e = cudaFuncSetAttribute(k_spec_x_fwd<R>, A, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_x_inv<R>, A, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_y<R, -1>, A, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_y<R, +1>, A, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spec_z<R>, A, optin);
  return e;
}

template <typename R>
cudaError_t launch_spec_tables(const Spec<R>& V, const double h[3], cudaStream_t st) {
  const int nmax = max(V.nx, max(V.ny, V.nz));
  k_spec_tables<R><<<dim3((nmax + 127) / 128, 3), 128, 0, st>>>(V, h[0], h[1], h[2]);
  return cudaGetLastError();
}

cudaError_t launch_spec_mean(long long n, const double* mu, const double* lam,
                             const double* eta, double* mean, double* partial,
                             unsigned int* counter, cudaStream_t st) {
  const long long want = (n + NT - 1) / NT;
  const int blocks = (int)(want < 1024 ? (want > 0 ? want : 1) : 1024);
  k_spec_mean<<<blocks, NT, 0, st>>>(n, mu, lam, eta, mean, partial, counter);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_spectral(const Spec<R>& V, const R* const r[3], R* const z[3], CgScal* S,
                            cudaStream_t st) {
  const dim3 gx(V.ny / (2 * V.pb), V.nz, 3);
  const dim3 gy((V.nxh + V.tx - 1) / V.tx, V.nz, 3);
  const dim3 gz((V.nxh + V.tz - 1) / V.tz, V.ny);
  k_spec_x_fwd<R><<<gx, NT, spec_smem_x(V), st>>>(V, r[0], r[1], r[2], S);
  k_spec_y<R, -1><<<gy, NT, spec_smem_y(V), st>>>(V, S);
  k_spec_z<R><<<gz, NT, spec_smem_z(V), st>>>(V, S);
  k_spec_y<R, +1><<<gy, NT, spec_smem_y(V), st>>>(V, S);
  k_spec_x_inv<R><<<gx, NT, spec_smem_x(V), st>>>(V, r[0], r[1], r[2], z[0], z[1], z[2], S);
  return cudaGetLastError();
}

template cudaError_t spec_prepare<float>(const Spec<float>&);
template cudaError_t spec_prepare<double>(const Spec<double>&);
template cudaError_t launch_spec_tables<float>(const Spec<float>&, const double[3], cudaStream_t);
template cudaError_t launch_spec_tables<double>(const Spec<double>&, const double[3], cudaStream_t);
template cudaError_t launch_spectral<float>(const Spec<float>&, const float* const[3],
                                            float* const[3], CgScal*, cudaStream_t);
template cudaError_t launch_spectral<double>(const Spec<double>&, const double* const[3],
                                             double* const[3], CgScal*, cudaStream_t);

}  // namespace tg
