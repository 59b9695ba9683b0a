// tg_diagnostics.cu -- the mass-effect diagnostics of Section 3.
//
// Per node, from the displacement u and the Lame coefficients (centred differences for
// grad u, as in the operator's mixed terms):
//   T = lambda tr(E) I + 2 mu E,  E = (grad u + grad u^T) / 2            (Eq. e:hook)
//   tr T, and the in-plane maximum shear stress sqrt(((T_xx - T_yy)/2)^2 + T_xy^2)
//                                                                       (Eq. e:princ_stress)
//   J = det(I + grad u)                                                 (Eq. e:jacobian)
// and the summaries the paper's mass-effect study reports: the extremes of J, the L2 norm of
// J - 1, the extremes of tr T, the largest shear, and d_max, the largest periodic distance
// from the tumor seed of a node whose displacement reaches a threshold.  Summaries are
// combined per block and then, by the last block, in block order (min, max and sums of
// squares; deterministic).
#include "tg_internal.cuh"

namespace tg {
namespace {

constexpr int NQ = 7;   // jac_min, jac_max, sum (J-1)^2, tr_min, tr_max, tau_max, d_max

__device__ __forceinline__ void combine(double (&a)[NQ], const double (&b)[NQ]) {
  a[0] = fmin(a[0], b[0]);
  a[1] = fmax(a[1], b[1]);
  a[2] += b[2];
  a[3] = fmin(a[3], b[3]);
  a[4] = fmax(a[4], b[4]);
  a[5] = fmax(a[5], b[5]);
  a[6] = fmax(a[6], b[6]);
}

__device__ __forceinline__ void identity(double (&a)[NQ]) {
  a[0] = INFINITY;
  a[1] = -INFINITY;
  a[2] = 0.0;
  a[3] = INFINITY;
  a[4] = -INFINITY;
  a[5] = 0.0;
  a[6] = 0.0;
}

__global__ void __launch_bounds__(NT) k_diagnostics(Geo G, DiagArgs A) {
  double acc[NQ];
  identity(acc);
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i < G.nx && j < G.ny) {
    const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
    for (int k = k0; k < k1; ++k) {
      const Nbr nb = make_nbr(G, i, j, k);
      const long long c = nb.at(0, 0, 0);
      double D[3][3];   // D[a][d] = d u_a / d x_d
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double* u = A.u[a];
        D[a][0] = (u[nb.at(1, 0, 0)] - u[nb.at(-1, 0, 0)]) * G.inv2h[0];
        D[a][1] = (u[nb.at(0, 1, 0)] - u[nb.at(0, -1, 0)]) * G.inv2h[1];
        D[a][2] = (u[nb.at(0, 0, 1)] - u[nb.at(0, 0, -1)]) * G.inv2h[2];
      }
      const double mu = A.mu[c], lam = A.lam[c];
      const double trE = D[0][0] + D[1][1] + D[2][2];
      const double txx = lam * trE + 2.0 * mu * D[0][0];
      const double tyy = lam * trE + 2.0 * mu * D[1][1];
      const double tzz = lam * trE + 2.0 * mu * D[2][2];
      const double txy = mu * (D[0][1] + D[1][0]);
      const double tr = txx + tyy + tzz;
      const double hx = 0.5 * (txx - tyy);
      const double tau = sqrt(hx * hx + txy * txy);
      const double f00 = 1.0 + D[0][0], f11 = 1.0 + D[1][1], f22 = 1.0 + D[2][2];
      const double jac = f00 * (f11 * f22 - D[1][2] * D[2][1]) -
                         D[0][1] * (D[1][0] * f22 - D[1][2] * D[2][0]) +
                         D[0][2] * (D[1][0] * D[2][1] - f11 * D[2][0]);
      if (A.out[0]) A.out[0][c] = tr;
      if (A.out[1]) A.out[1][c] = tau;
      if (A.out[2]) A.out[2][c] = jac;
      const double u0 = A.u[0][c], u1 = A.u[1][c], u2 = A.u[2][c];
      double dist = 0.0;
      if (sqrt(u0 * u0 + u1 * u1 + u2 * u2) >= A.threshold) {
        const int q[3] = {i, j, k};
        double r2 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          double x = q[d] * G.h[d] - A.seed[d];
          x -= A.L[d] * floor(x / A.L[d] + 0.5);   // nearest periodic image
          r2 += x * x;
        }
        dist = sqrt(r2);
      }
      const double v[NQ] = {jac, jac, (jac - 1.0) * (jac - 1.0), tr, tr, tau, dist};
      combine(acc, v);
    }
  }
  // block: warp shuffles, then warps in order
  __shared__ double sh[NQ][NWARP];
  __shared__ bool am_last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    double o[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) o[q] = __shfl_down_sync(0xffffffffu, acc[q], off);
    combine(acc, o);
  }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[q][warp] = acc[q];
  __syncthreads();
  const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int nb = gridDim.x * gridDim.y * gridDim.z;
  if (tid == 0) {
    double s[NQ];
    identity(s);
    for (int w = 0; w < NWARP; ++w) {
      double t[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) t[q] = sh[q][w];
      combine(s, t);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) A.partial[(size_t)b * NQ + q] = s[q];
    __threadfence();
    am_last = atomicAdd(A.counter, 1u) == (unsigned int)(nb - 1);
  }
  __syncthreads();
  if (!am_last || tid != 0) return;
  __threadfence();
  double s[NQ];
  identity(s);
  for (int k = 0; k < nb; ++k) {
    double t[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = __ldcg(A.partial + (size_t)k * NQ + q);
    combine(s, t);
  }
  const double vol = G.h[0] * G.h[1] * G.h[2];
  A.result[0] = s[0];
  A.result[1] = s[1];
  A.result[2] = sqrt(vol * s[2]);
  A.result[3] = s[3];
  A.result[4] = s[4];
  A.result[5] = s[5];
  A.result[6] = s[6];
  *A.counter = 0u;
}

}  // namespace

cudaError_t launch_diagnostics(const Geo& G, const DiagArgs& A, cudaStream_t st) {
  k_diagnostics<<<G.grid, dim3(BX, BY), 0, st>>>(G, A);
  return cudaGetLastError();
}

}  // namespace tg
