// tg_transport.cu -- semi-Lagrangian transport of S1.
//
// Section 3: characteristics X* = x - dt v(x), X = x - dt/2 (v(x) + v(X*)) and the RK2 source
// update nu* = nu(X) + dt g(nu(X)),  nu = nu(X) + dt/2 (g(nu(X)) + g(nu*)), with cubic
// interpolation at X* and X.  p, i, n, g, w obey d_t q + div(q v) = 0, i.e. the source along
// the characteristic is g(q, x) = -q div v(x); f obeys d_t f + grad f . v = 0 (no source).
// Coordinates are kept in index units (X_d = j_d - dt v_d / h_d), interpolation is tricubic
// Lagrange on nodes floor(X) - 1 .. floor(X) + 2 with periodic wrap, and div v is the
// centred-difference divergence.
#include "tg_internal.cuh"

namespace tg {
namespace {

__global__ void __launch_bounds__(NT) k_divergence(Geo G, const double* __restrict__ vx,
                                                   const double* __restrict__ vy,
                                                   const double* __restrict__ vz, double* div) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const Nbr nb = make_nbr(G, i, j, k);
    div[nb.at(0, 0, 0)] = (vx[nb.at(1, 0, 0)] - vx[nb.at(-1, 0, 0)]) * G.inv2h[0] +
                          (vy[nb.at(0, 1, 0)] - vy[nb.at(0, -1, 0)]) * G.inv2h[1] +
                          (vz[nb.at(0, 0, 1)] - vz[nb.at(0, 0, -1)]) * G.inv2h[2];
  }
}

struct Tricubic {
  long long xo[4], yo[4], zo[4];
  double wx[4], wy[4], wz[4];
};

// cubic Lagrange basis on nodes -1, 0, 1, 2 at fractional position t
__device__ __forceinline__ void lagrange4(double t, double w[4]) {
  const double tm1 = t - 1.0, tm2 = t - 2.0, tp1 = t + 1.0;
  w[0] = -t * tm1 * tm2 * (1.0 / 6.0);
  w[1] = tp1 * tm1 * tm2 * 0.5;
  w[2] = -tp1 * t * tm2 * 0.5;
  w[3] = tp1 * t * tm1 * (1.0 / 6.0);
}

__device__ __forceinline__ void axis_setup(double X, int n, long long stride, long long o[4],
                                           double w[4]) {
  const double fl = floor(X);
  long long m = ((long long)fl - 1) % n;
  if (m < 0) m += n;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    o[a] = m * stride;
    m = (m + 1 == n) ? 0 : m + 1;
  }
  lagrange4(X - fl, w);
}

__device__ __forceinline__ void setup(Tricubic& T, const Geo& G, double X, double Y, double Z) {
  axis_setup(X, G.nx, 1, T.xo, T.wx);
  axis_setup(Y, G.ny, G.nx, T.yo, T.wy);
  axis_setup(Z, G.nz, G.nxy, T.zo, T.wz);
}

__device__ __forceinline__ double eval(const Tricubic& T, const double* __restrict__ q) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double sy = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const double* row = q + T.zo[c] + T.yo[b];
      const double sx = T.wx[0] * __ldg(row + T.xo[0]) + T.wx[1] * __ldg(row + T.xo[1]) +
                        T.wx[2] * __ldg(row + T.xo[2]) + T.wx[3] * __ldg(row + T.xo[3]);
      sy += T.wy[b] * sx;
    }
    s += T.wz[c] * sy;
  }
  return s;
}

struct Six {
  const double* a[6];
};
struct Six_out {
  double* a[6];
};

__global__ void __launch_bounds__(NT) k_sl(Geo G, double dt, double3 dt_h,
                                           const double* __restrict__ vx,
                                           const double* __restrict__ vy,
                                           const double* __restrict__ vz,
                                           const double* __restrict__ div, Six qin, Six_out qout) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    const double v0x = vx[c], v0y = vy[c], v0z = vz[c];
    Tricubic T;
    setup(T, G, i - v0x * dt_h.x, j - v0y * dt_h.y, k - v0z * dt_h.z);
    const double vsx = eval(T, vx), vsy = eval(T, vy), vsz = eval(T, vz);
    setup(T, G, i - 0.5 * (v0x + vsx) * dt_h.x, j - 0.5 * (v0y + vsy) * dt_h.y,
          k - 0.5 * (v0z + vsz) * dt_h.z);
    const double dX = eval(T, div);
    const double dx = div[c];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const double qX = eval(T, qin.a[s]);
      const double gX = -qX * dX;
      const double qs = qX + dt * gX;
      const double gs = -qs * dx;
      qout.a[s][c] = qX + 0.5 * dt * (gX + gs);
    }
    qout.a[5][c] = eval(T, qin.a[5]);
  }
}

}  // namespace

cudaError_t launch_divergence(const Geo& G, const double* const v[3], double* div, cudaStream_t st) {
  TG_TIMED(K_DIVERGENCE, st,
           k_divergence<<<G.grid, dim3(BX, BY), 0, st>>>(G, v[0], v[1], v[2], div));
  return cudaGetLastError();
}

cudaError_t launch_sl_advect(const Geo& G, double dt, const double* const v[3], const double* div,
                             const double* const qin[6], double* const qout[6], cudaStream_t st) {
  Six a;
  Six_out b;
  for (int s = 0; s < 6; ++s) {
    a.a[s] = qin[s];
    b.a[s] = qout[s];
  }
  const double3 dth = make_double3(dt / G.h[0], dt / G.h[1], dt / G.h[2]);
  TG_TIMED(K_SL, st,
           k_sl<<<G.grid, dim3(BX, BY), 0, st>>>(G, dt, dth, v[0], v[1], v[2], div, a, b));
  return cudaGetLastError();
}

}  // namespace tg
