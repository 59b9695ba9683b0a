// tg_internal.cuh -- shared device helpers and host-side launch declarations of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tg.h"
#include "tg_fpconv.cuh"

namespace tg {

// Thread block of every grid-shaped kernel: 32 x 8 threads over (x, y), marching a chunk of
// z planes.  x is the contiguous axis, so a warp reads 32 consecutive values of a row.
constexpr int BX = 32;
constexpr int BY = 8;
constexpr int NT = BX * BY;
constexpr int NWARP = NT / 32;

// ------------------------------------------------------------------ optional kernel timing
// Kernels that the timing of tg_set_timing reports one by one.  Every launch site of the step
// and the solves brackets its kernel with TG_TIMED; when the calling host thread has a hook
// installed (a context with timing on), the hook records CUDA events before and after the
// launch on the launch's own stream.  Without a hook the bracket is one thread-local load.
enum KernelId : int {
  K_DIFF_FACES, K_DIFF_DIAG, K_TO_F32, K_DIVERGENCE, K_SL, K_SL32,
  K_CN_INIT, K_CN_MATVEC, K_CN_UPDATE, K_CN_PUPDATE,
  K_CN_IR_RESIDUAL, K_CN_IR_RESIDUAL_DF, K_CN32_PUPDATE, K_CN32_MATVEC, K_CN32_UPDATE,
  K_CN_IR_CORRECT, K_CN32_NEUMANN, K_DIFF_NODE_DF, K_DIFF_FACES_DF, K_REACT, K_LAME, K_ELAS_COEF, K_ELAS_COEF_DF, K_ELAS32_COEF, K_DF_PACK3,
  K_ELAS_EXTRAPOLATE, K_SPEC_MEAN, K_SPEC_SCALE, K_ELAS_IR_RESIDUAL, K_ELAS_IR_RESIDUAL_DF,
  K_ELAS32_SCALE_R, K_SPEC_X_FWD, K_SPEC_Y_FWD, K_SPEC_Z, K_SPEC_ZR, K_SPEC_Y_INV,
  K_SPEC_X_INV, K_SPEC_X_INV_P, K_ELAS32_MATVEC, K_ELAS32_UPDATE, K_ELAS32_MATVEC_SPEC,
  K_ELAS32_UPDATE_SPEC, K_SPEC_UPDATE_XFWD, K_ELAS_IR_CORRECT, K_ELAS_IR_FINISH,
  K_ELAS_INIT, K_ELAS_INIT_SPEC, K_ELAS_MATVEC, K_ELAS_UPDATE, K_ELAS_PUPDATE, K_ELAS_UPDATE_SPEC,
  K_ELAS_PUPDATE_SPEC, K_ELAS_FINISH, K_OX_PREP, K_OX_INIT, K_OX_MATVEC, K_OX_UPDATE,
  K_OX_PUPDATE, K_OX_FINISH, K_SL32_PACK, K_LAME_DF,
  K_COUNT
};

struct KHook {
  void (*pre)(void* self, cudaStream_t st);
  void (*post)(void* self, int kid, cudaStream_t st);
  void* self;
};
extern thread_local const KHook* tg_khook;

#define TG_TIMED(kid, st, ...)                          \
  do {                                                  \
    const ::tg::KHook* h_ = ::tg::tg_khook;             \
    if (h_) h_->pre(h_->self, (st));                    \
    __VA_ARGS__;                                        \
    if (h_) h_->post(h_->self, (kid), (st));            \
  } while (0)

struct Geo {
  int nx, ny, nz;
  long long nxy, nvox;
  double h[3];
  double ih2[3];        // 1 / h_d^2
  double inv2h[3];      // 1 / (2 h_d)
  double s_cross[3][3]; // 1 / (4 h_a h_d)
  int zc;               // z planes per block
  dim3 grid;            // (ceil(nx/BX), ceil(ny/BY), ceil(nz/zc))
  int nblocks;
};

// Device-side state of one CG solve (one right-hand side).
enum CgStatus : int {
  CG_RUNNING = 0,
  CG_CONVERGED = 1,
  CG_NONFINITE = 2,
  CG_MAXIT = 3,
  CG_ZERO_RHS = 4,
  CG_TIMEOUT = 5     // a bounded device-side wait gave up (the solve's kernels return at once)
};

struct CgScal {
  double rz;     // <r, D^{-1} r>
  double rr;     // <r, r>
  double bb;     // <rhs, rhs>
  double pq;     // <p, A p>
  double alpha;
  double beta;
  double rtol;
  double scale;  // inner solves of a refinement: the right-hand side was multiplied by it
  int it;
  int maxit;
  int status;
  int pad;
};

// Periodic neighbour offsets of node (i, j, k): X[o+1], Y[o+1], Z[o+1] for o in {-1, 0, 1};
// the linear index of (i + ox, j + oy, k + oz) is Z[oz+1] + Y[oy+1] + X[ox+1].
struct Nbr {
  long long X[3], Y[3], Z[3];
  __device__ __forceinline__ long long at(int ox, int oy, int oz) const {
    return Z[oz + 1] + Y[oy + 1] + X[ox + 1];
  }
};

__device__ __forceinline__ Nbr make_nbr(const Geo& g, int i, int j, int k) {
  Nbr n;
  n.X[0] = (i == 0) ? g.nx - 1 : i - 1;
  n.X[1] = i;
  n.X[2] = (i + 1 == g.nx) ? 0 : i + 1;
  n.Y[0] = (long long)((j == 0) ? g.ny - 1 : j - 1) * g.nx;
  n.Y[1] = (long long)j * g.nx;
  n.Y[2] = (long long)((j + 1 == g.ny) ? 0 : j + 1) * g.nx;
  n.Z[0] = (long long)((k == 0) ? g.nz - 1 : k - 1) * g.nxy;
  n.Z[1] = (long long)k * g.nxy;
  n.Z[2] = (long long)((k + 1 == g.nz) ? 0 : k + 1) * g.nxy;
  return n;
}

// offset vector with s_a along axis A and s_d along axis D
template <int A, int D>
__device__ __forceinline__ long long at2(const Nbr& n, int sa, int sd) {
  int o[3] = {0, 0, 0};
  o[A] += sa;
  o[D] += sd;
  return n.at(o[0], o[1], o[2]);
}

template <int A>
__device__ __forceinline__ long long at1(const Nbr& n, int s) {
  int o[3] = {0, 0, 0};
  o[A] += s;
  return n.at(o[0], o[1], o[2]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int block_linear() {
  return (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
}

__device__ __forceinline__ int block_count() { return gridDim.x * gridDim.y * gridDim.z; }

// Block-level sum of NV values, written to partial[b][NV] for work item b of nb; the last item
// to finish sums all partials in item order (deterministic) and returns true in every thread
// of that block, with the totals in out[] valid in thread 0.  counter is reset by the last.
template <int NV>
__device__ bool reduce_indexed(double (&v)[NV], double* partial, unsigned int* counter, int b,
                               int nb, double (&out)[NV]) {
  __shared__ double sh[NV][NWARP];
  __shared__ bool am_last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) sh[q][warp] = s;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int w = 0; w < NWARP; ++w) s += sh[q][w];
      partial[(size_t)b * NV + q] = s;
    }
    __threadfence();
    unsigned int ticket = atomicAdd(counter, 1u);
    am_last = (ticket == (unsigned int)(nb - 1));
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  for (int k = tid; k < nb; k += NT) {
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += __ldcg(partial + (size_t)k * NV + q);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = warp_sum(acc[q]);
    if (lane == 0) sh[q][warp] = s;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int w = 0; w < NWARP; ++w) s += sh[q][w];
      out[q] = s;
    }
    *counter = 0u;
  }
  __syncthreads();
  return true;
}

// the same over the blocks of a launch
template <int NV>
__device__ bool reduce_last_block(double (&v)[NV], double* partial, unsigned int* counter,
                                  double (&out)[NV]) {
  return reduce_indexed<NV>(v, partial, counter, block_linear(), block_count(), out);
}

// Convergence decision after an update (same order of tests as a textbook PCG loop:
// converged, non-finite, iteration limit).
__device__ __forceinline__ void cg_after_update(CgScal& S, double rz_new, double rr) {
  S.it += 1;
  S.rr = rr;
  if (!isfinite(rr)) {
    S.status = CG_NONFINITE;
  } else if (sqrt(rr) <= S.rtol * sqrt(S.bb)) {
    S.status = CG_CONVERGED;
  } else if (S.it >= S.maxit) {
    S.status = CG_MAXIT;
  } else {
    S.beta = rz_new / S.rz;
    S.rz = rz_new;
  }
}

// With a preconditioner applied in separate kernels the update decides convergence from
// <r, r> alone and the preconditioner's last kernel supplies <r, z> and beta.
__device__ __forceinline__ void cg_after_update_rr(CgScal& S, double rr) {
  S.it += 1;
  S.rr = rr;
  if (!isfinite(rr)) {
    S.status = CG_NONFINITE;
  } else if (sqrt(rr) <= S.rtol * sqrt(S.bb)) {
    S.status = CG_CONVERGED;
  } else if (S.it >= S.maxit) {
    S.status = CG_MAXIT;
  }
}

__device__ __forceinline__ void cg_after_precond(CgScal& S, double rz_new) {
  if (!isfinite(rz_new)) {
    S.status = CG_NONFINITE;
    return;
  }
  S.beta = (S.it == 0) ? 0.0 : rz_new / S.rz;
  S.rz = rz_new;
}

// a solve left out of a masked launch: finished, with nothing done
__device__ __forceinline__ void cg_skip(CgScal& S) {
  S.it = 0;
  S.bb = 0.0;
  S.rr = 0.0;
  S.status = CG_CONVERGED;
}

__device__ __forceinline__ void cg_after_init(CgScal& S, double bb, double rr, double rz) {
  S.bb = bb;
  S.rr = rr;
  S.rz = rz;
  S.it = 0;
  S.alpha = 0.0;
  S.beta = 0.0;
  if (bb == 0.0) {
    S.status = CG_ZERO_RHS;
  } else if (!isfinite(rr)) {
    S.status = CG_NONFINITE;
  } else if (sqrt(rr) <= S.rtol * sqrt(bb)) {
    S.status = CG_CONVERGED;
  } else if (S.maxit <= 0) {
    S.status = CG_MAXIT;
  } else {
    S.status = CG_RUNNING;
  }
}

// Parameters the kernels need, derived once per call on the host.
struct DevParams {
  double k_g, k_w, k_f, k_scale;
  double rho_g, rho_w, rho_i_frac;
  double alpha0, beta0, gamma, sigma_b, o_hyp, o_inv, o_heal, o_mit;
  double delta_s, delta_p, inv_eps_H;
  double cmu[5], clam[5], eta[5];   // per-species Lame and screening weights (Eq. e:lame)
  double zeta;
  double delta_e, delta_half, delta_l;
};

// ----------------------------------------------------------------------------- FP32 buffers

struct F32Copy {   // up to ten FP64 -> FP32 array conversions in one pass
  const double* src[10];
  float* dst[10];
  int count;
};

struct Elas32 {    // inner FP32 elasticity solve of the mixed precision
  float* mu;
  float* lam;
  float* eta;
  float* dinv[3];
  float* e[3];     // correction (CG iterate)
  float* r[3];
  float* p[2][3];  // search direction, double-buffered: iteration k reads p[k&1], writes p[~k&1]
  float* q[3];
  const float* z[3];  // z = P r of a plain preconditioner application (the spectral CG itself
                      // takes p from the preconditioner's last pass)
  CgScal* S;
  double* partial;
  unsigned int* counter;
};

// FP32 transport.  Its inputs are FP32 copies interleaved per voxel, so that one 16-byte load
// brings four of the values a stencil tap needs: v4 = (v_x, v_y, v_z, 0),
// qa = (p, i, n, div_h v), qb = (g, w, f, 0).  The outputs go to the FP64 state.
struct Sl32 {
  float4* v4;
  float4* qa;
  float4* qb;
  double* out[6];
};

// ---------------------------------------------------------------- diagnostics (Section 3)
struct DiagArgs {
  const double* u[3];
  const double* mu;
  const double* lam;
  double* out[3];          // tr T, max shear, det(I + grad u); entries may be null
  double seed[3];          // tumor seed (physical coordinates)
  double L[3];             // box lengths (periodic distances)
  double threshold;        // |u| reaching it counts for d_max
  double* partial;         // 7 per block
  unsigned int* counter;
  double* result;          // 7 doubles (device)
};
cudaError_t launch_diagnostics(const Geo&, const DiagArgs&, cudaStream_t st);

// ---------------------------------------------------------------- spectral preconditioner
// Section 3: the elasticity solve is preconditioned by the exact inverse of the operator with
// constant coefficients (the domain means of mu, lambda, eta).  For the finite-difference
// operator on the periodic grid that inverse is diagonal in the discrete Fourier basis: one
// 3x3 real symmetric system per wave vector, diagonal plus rank one (Sherman-Morrison).
// Grid sizes are powers of two.  W holds the half spectrum (kx = 0 .. nx/2) of the three
// components after the x transform, rows padded to nxp modes.
template <typename R> struct CxOf;
template <> struct CxOf<float> { using T = float2; };
template <> struct CxOf<double> { using T = double2; };

template <typename R>
struct Spec {
  using C = typename CxOf<R>::T;
  int nx, ny, nz, nxh, nxp;   // grid; x modes kept (nx/2 + 1); row pitch of W in modes
  int pb, tx, tz;             // row pairs per x-pass block; mode columns per y / z block
  int nt_z;                   // threads of a z-pass block
  int x_inpl;                 // the x passes other than the fused update pass transform in
                              // place in one line buffer (every stage's butterflies at most
                              // one per thread of a block)
  C* W;                       // 3 components x nz x ny x nxp
  C* tw[3];                   // exp(-2 pi i k / n_d), k < n_d
  R* S[3];                    // 4 sin^2(theta_k / 2) / h_d^2, theta_k = 2 pi k / n_d
  R* T[3];                    // sin(theta_k) / h_d
  R* s[3];                    // diagonal scaling s = (D0 / D)^{1/2} per component (null:
                              // the unscaled preconditioner)
  double* mean;               // mu0, lambda0, eta0 (device)
  double* partial;            // per-block partial sums (x inverse pass, means)
  unsigned int* counter;
  int nb_partial;             // capacity of partial, in doubles
  const void* zmap;           // host: TMA tensor map of W for the FP32 z pass (null: none)
};

// The CG p-update fused into the x inverse pass (mixed precision): the pass writes the new
// search direction p = z + beta p_old instead of z, into the buffer of the two that the
// iteration's operator kernel reads (they alternate with the iteration count S->it).
template <typename R>
struct PUpd {
  R* p[2][3];
};

// shared memory of each pass (bytes): the line length's twiddles and two line buffers
template <typename R> size_t spec_smem_x(const Spec<R>& V) {   // lines padded to pb + 1
  return (1 + (V.x_inpl ? 1 : 2) * ((size_t)V.pb + 1)) * V.nx * sizeof(typename CxOf<R>::T);
}
template <typename R> size_t spec_smem_x2(const Spec<R>& V) {   // always two line buffers
  return (1 + 2 * ((size_t)V.pb + 1)) * V.nx * sizeof(typename CxOf<R>::T);
}
// a y transform of at most two stages (n <= 256) stages through one buffer only
__host__ __device__ inline int spec_y_buffers(int ny) {
  int ln = 0;
  while ((1 << ln) < ny) ++ln;
  return ((ln & 3) ? 1 : 0) + (ln >> 2) <= 2 ? 1 : 2;
}
template <typename R> size_t spec_smem_y(const Spec<R>& V) {
  return (1 + (size_t)spec_y_buffers(V.ny) * V.tx) * V.ny * sizeof(typename CxOf<R>::T);
}
template <typename R> size_t spec_smem_z(const Spec<R>& V) {
  return (1 + 2 * (size_t)3 * V.tz) * V.nz * sizeof(typename CxOf<R>::T);
}

// ----------------------------------------------------------------------------- launches
// All return cudaGetLastError() after queueing on `st`.

// S0: diffusion faces (scaled by dt/(2 h_d^2)), Jacobi diagonal of the CN operator, rho.
cudaError_t launch_diff_coef(const Geo&, const DevParams&, double dt, const double* g,
                             const double* w, const double* f, double* const Kf[3], double* dsum,
                             double* dinv, double* rho, cudaStream_t st,
                             double* const Kfdf[3] = nullptr);   // (hi, lo) pairs, optional

struct Cn3 {   // three simultaneous CN solves sharing one operator
  double* x[3];
  double* r[3];
  double* p[3];
  double* q[3];
  const double* Kf[3];
  const double* dsum;
  const double* dinv;
  CgScal* S;           // 3 entries
  double* partial;
  unsigned int* counter;
  // double-FP32 residual of the mixed precision (df != 0): (hi, lo) pairs of the fields and
  // of the faces; the right-hand sides in p are then pairs as well
  int df;
  float2* xdf[3];
  const float2* Kfdf[3];
};
cudaError_t launch_cn_init(const Geo&, const Cn3&, cudaStream_t st, int mask = 7);
cudaError_t launch_cn_iter(const Geo&, const Cn3&, cudaStream_t st);

// Mixed precision S2: iterative refinement around three FP32 CN solves.  The FP64 side keeps
// the fields (Cn3::x), the right-hand sides (stored in Cn3::p) and the residuals; the FP32
// side solves A e = r with Jacobi PCG on FP32 faces, the diagonal rebuilt from the faces.
struct Cn32 {
  float* e[3];
  float* r[3];
  float* p[3];
  float* q[3];
  float* z[3];         // preconditioned residual of the polynomial preconditioner (null: Jacobi)
  float* palt[3];      // with z: the second search-direction buffer (iteration k writes
                       // p[k & 1 ? p : palt], reading the other)
  const float* Kf[3];
  const float* dinv;
  const float* dmax;   // the CN diagonal's maximum (for the polynomial's weights), or null
  CgScal* S;           // 3 inner solves
  double* partial;
  unsigned int* counter;
};
// FP64 residual r = rhs - A x (init: rhs = x + dt/2 D_h x is formed and stored first), its
// FP32 copy, e = 0, and the outer test / inner start per right-hand side (Sout: 3 entries)
cudaError_t launch_cn_ir_residual(const Geo&, const Cn3&, const Cn32&, CgScal* Sout, bool init,
                                  double tau_min, int max_sweeps, int mask, cudaStream_t st);
// One inner iteration.  With I.z set the iteration is preconditioned by the Neumann series of
// the Jacobi splitting (launch_cn32_neumann, solves r0 and r1, -1 for none) and begins with
// it: z = M r, <r, z>; p = z + beta p; q = A p; e, r updated (convergence from |r|).
// partial_capacity: doubles the reduction buffer holds.
cudaError_t launch_cn32_iter(const Geo&, const Cn32&, cudaStream_t st, int r0 = -1,
                             int r1 = -1, long long partial_capacity = 0);
cudaError_t launch_cn_ir_correct(const Geo&, const Cn3&, const Cn32&, int mask, cudaStream_t st);

// The oxygen solve of the mixed precision in double-FP32 arithmetic (tg_cn_ox.cu): the FP64
// path's Jacobi-CG iterates, carried as (hi, lo) FP32 pairs.
struct OxDf {
  const float2* Kf[3];   // face pairs a_d,j (written in S0 for the double-FP32 residuals)
  float2* dd;            // CN diagonal 1 + sum of the six faces
  float2* di;            // its inverse
  float2* x;             // CG iterate
  float2* r;
  float2* p;
  float2* q;
  double* o;             // the oxygen field: start, and the result
  CgScal* S;             // the solve's scalars
  double* partial;
  unsigned int* counter;
};
// prep (diagonal pairs, x = o) and the CG start; one iteration; o = x
cudaError_t launch_ox_start(const Geo&, const OxDf&, cudaStream_t st);
cudaError_t launch_ox_iter(const Geo&, const OxDf&, cudaStream_t st);
cudaError_t launch_ox_finish(const Geo&, const OxDf&, cudaStream_t st);

// SL (S1)
cudaError_t launch_divergence(const Geo&, const double* const v[3], double* div, cudaStream_t st);
cudaError_t launch_sl_advect(const Geo&, double dt, const double* const v[3], const double* div,
                             const double* const qin[6], double* const qout[6], cudaStream_t st);

// S2 fix-up + S3-S5 (fp32_rates: the mixed precision's FP32 rate arithmetic; single: the
// single-species model, c in p)
cudaError_t launch_react(const Geo&, const DevParams&, double dt, const double* rho,
                         const double* i_dag, double* p, double* i, double* n, double* g,
                         double* w, double* o, double* l, bool fp32_rates, bool single,
                         cudaStream_t st);

// S6 coefficients
cudaError_t launch_lame(const Geo&, const DevParams&, const double* p, const double* i,
                        const double* n, const double* g, const double* w, const double* f,
                        const double* bg, double* mu, double* lam, double* eta, cudaStream_t st);
// the same in double-FP32 for the double-FP32 residual: FP64 mu, lambda, eta, their FP32
// copies, the (hi, lo) pairs of mu and lambda, and the pairs of s = p + n for the force
cudaError_t launch_lame_df(const Geo&, const DevParams&, const double* p, const double* i,
                           const double* n, const double* g, const double* w, const double* f,
                           const double* bg, double* mu, double* lam, double* eta, float* mu32,
                           float* lam32, float* eta32, float2* mudf, float2* lamdf, float2* sdf,
                           cudaStream_t st);

struct Elas {
  const double* mu;
  const double* lam;
  const double* eta;
  double* F[3];      // face (lambda + 2 mu) / h_d^2 between j and j + e_d
  double* G[3];      // face mu / h_d^2
  double* dsum[3];   // Jacobi diagonal per component
  double* dinv[3];   // its inverse, formed only with Jacobi preconditioning (jacobi != 0)
  double* b[3];      // force (or caller's rhs when b_external)
  double* du[3];     // CG iterate: increment of u
  double* r[3];
  double* p[3];
  double* q[3];
  double* u[3];      // displacement (in: u^n, out: u^{n+1})
  double* v[3];      // velocity (written when dt > 0)
  double* vp[3];     // velocity at the previous step's start (the quadratic extrapolation's
                     // history; a step's finish stores v^n there before writing v^{n+1})
  double* z[3];      // spectral preconditioner output (null with Jacobi)
  // double-FP32 residual of the mixed precision (df != 0): F, G and dsum then hold (hi, lo)
  // FP32 pairs instead of FP64 values, and udf, mudf, lamdf the pairs of u, mu and lambda
  int df;
  int jacobi;        // 0 with the spectral preconditioner: dinv (FP64 and FP32) is not used
  float2* udf[3];
  float2* mudf;
  float2* lamdf;
  CgScal* S;
  double* partial;
  unsigned int* counter;
};

// Double-FP32 numbers (Df) and the FP64 <-> FP32 conversions on the integer pipes come from
// tg_fpconv.cuh; the storage forms here.
__device__ __forceinline__ Df df_of(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 df_pack(double x) {
  const Df d = df_split(x);
  return make_float2(d.hi, d.lo);
}

// S0 of the mixed precision with double-FP32 residuals: node K pairs (Kn, scratch), rho, the
// face pairs, the FP32 faces and the FP32 inverse CN diagonal (no FP64 faces)
cudaError_t launch_diff_coef_df(const Geo&, const DevParams&, double dt, const double* g,
                                const double* w, const double* f, float2* Kn, double* rho,
                                float2* const Kfdf[3], float* const Kf32[3], float* dinv32,
                                float* dmax, cudaStream_t st);

// 4 h_A h_D [ d_D(mu d_A u_D) + d_A(lambda d_D u_D) ] at the centre node (centred differences)
template <int A, int D>
__device__ __forceinline__ double elas_mixed64(const Nbr& nb, const double* __restrict__ xd,
                                              const double* __restrict__ mu,
                                              const double* __restrict__ lam) {
  const double epp = xd[at2<A, D>(nb, +1, +1)];  // c + e_A + e_D
  const double epm = xd[at2<A, D>(nb, -1, +1)];  // c - e_A + e_D
  const double emp = xd[at2<A, D>(nb, +1, -1)];  // c + e_A - e_D
  const double emm = xd[at2<A, D>(nb, -1, -1)];  // c - e_A - e_D
  return mu[at1<D>(nb, +1)] * (epp - epm) - mu[at1<D>(nb, -1)] * (emp - emm) +
         lam[at1<A>(nb, +1)] * (epp - emp) - lam[at1<A>(nb, -1)] * (epm - emm);
}

// component A of (eta I - L_h) x at node c, from the stored FP64 faces and diagonal
template <int A>
__device__ __forceinline__ double elas_row64(const Geo& G, const Nbr& nb, long long c,
                                             const Elas& E, const double* const x[3]) {
  constexpr int D1 = (A + 1) % 3, D2 = (A + 2) % 3;
  const double* __restrict__ xa = x[A];
  const double* __restrict__ CA = E.F[A];
  const double* __restrict__ C1 = E.G[D1];
  const double* __restrict__ C2 = E.G[D2];
  double v = E.dsum[A][c] * xa[c];
  v -= CA[c] * xa[at1<A>(nb, 1)] + CA[at1<A>(nb, -1)] * xa[at1<A>(nb, -1)];
  v -= C1[c] * xa[at1<D1>(nb, 1)] + C1[at1<D1>(nb, -1)] * xa[at1<D1>(nb, -1)];
  v -= C2[c] * xa[at1<D2>(nb, 1)] + C2[at1<D2>(nb, -1)] * xa[at1<D2>(nb, -1)];
  v -= G.s_cross[A][D1] * elas_mixed64<A, D1>(nb, x[D1], E.mu, E.lam);
  v -= G.s_cross[A][D2] * elas_mixed64<A, D2>(nb, x[D2], E.mu, E.lam);
  return v;
}

cudaError_t launch_elas_coef(const Geo&, const DevParams&, const Elas&, const double* p,
                             const double* n, bool force, cudaStream_t st);
// the same as (hi, lo) pairs from the node pairs E.mudf, E.lamdf (E.df) and the pairs sdf of
// s = p + n, all written by launch_lame_df; I.dinv if E.jacobi
cudaError_t launch_elas_coef_df(const Geo&, const DevParams&, const Elas&, const Elas32& I,
                                const float2* sdf, bool force, cudaStream_t st);
cudaError_t launch_elas_init(const Geo&, const Elas&, bool rhs_is_minus_b, cudaStream_t st);
cudaError_t launch_elas_matvec(const Geo&, const Elas&, cudaStream_t st);
cudaError_t launch_elas_update(const Geo&, const Elas&, cudaStream_t st);   // update + p-update
cudaError_t launch_elas_init_spec(const Geo&, const Elas&, bool rhs_is_minus_b, cudaStream_t st);
cudaError_t launch_elas_update_spec(const Geo&, const Elas&, cudaStream_t st);
cudaError_t launch_elas_pupdate_spec(const Geo&, const Elas&, cudaStream_t st);
cudaError_t launch_elas_finish(const Geo&, const Elas&, double inv_dt, bool zero_rhs,
                               int extrap, cudaStream_t st);

// mixed precision (tg_mixed.cu)
cudaError_t launch_to_f32(long long n, const F32Copy& c, cudaStream_t st);
constexpr int ELAS32_NODES = 1, ELAS32_DINV = 2, ELAS32_U = 4;
cudaError_t launch_elas32_coef(const Geo&, const Elas&, const Elas32&, cudaStream_t st,
                              int parts = ELAS32_NODES | ELAS32_DINV | ELAS32_U);
cudaError_t launch_df_pack3(const Geo&, const double* const b[3], double* const out[3],
                            cudaStream_t st);
cudaError_t launch_elas_ir_residual(const Geo&, const Elas&, const Elas32&, CgScal* Sout,
                                    bool minus_b, double tau_min, cudaStream_t st);
cudaError_t launch_elas32_matvec(const Geo&, const Elas32&, cudaStream_t st);
cudaError_t launch_elas32_update(const Geo&, const Elas32&, cudaStream_t st);
cudaError_t launch_elas_ir_correct(const Geo&, const Elas&, const Elas32&, cudaStream_t st);
cudaError_t launch_elas_extrapolate(const Geo&, const Elas&, double dt, bool quadratic,
                                    cudaStream_t st);
cudaError_t launch_elas_ir_finish(const Geo&, const Elas&, double inv_dt, bool zero_rhs,
                                  cudaStream_t st);
// S1 of the mixed precision: the interleaved FP32 inputs (div_h v formed in FP64 and rounded),
// then the transport.  Both need nvox < 2^31 (32-bit voxel offsets).
cudaError_t launch_sl32_pack(const Geo&, const double* const v[3], const double* const q[6],
                             const Sl32&, cudaStream_t st);
cudaError_t launch_sl32(const Geo&, double dt, const Sl32&, cudaStream_t st);

// spectral preconditioner: one-time tables, per-solve means, z = A0^{-1} r with <r, z>
// finishing the CG scalars in S (S may be null: plain application)
template <typename R>
cudaError_t launch_spec_tables(const Spec<R>&, const double h[3], cudaStream_t st);
template <typename R>
cudaError_t spec_prepare(const Spec<R>&);   // shared-memory limits of the pass kernels
// V.s = (D0 / D)^{1/2} from E.dsum and the means (TG_PRECOND_SPECTRAL_SCALED)
template <typename R>
cudaError_t launch_spec_scale(const Geo&, const Spec<R>& V, const Elas& E, cudaStream_t st);
// the domain means of mu, lambda, eta; fp32_terms: each thread's terms summed in FP32 (the
// mixed precision), else every term in FP64
cudaError_t launch_spec_mean(long long n, const double* mu, const double* lam,
                             const double* eta, double* mean, double* partial,
                             unsigned int* counter, cudaStream_t st, bool fp32_terms);
template <typename R>
cudaError_t launch_spectral(const Spec<R>&, const R* const r[3], R* const z[3], CgScal* S,
                            cudaStream_t st, const PUpd<R>* pu = nullptr);
cudaError_t launch_elas32_matvec_spec(const Geo&, const Elas32&, cudaStream_t st);
cudaError_t launch_spectral_update(const Spec<float>&, const Elas32&, float* const z[3],
                                   cudaStream_t st);
// the TMA tensor map (a CUtensorMap, 128 bytes, 64-byte aligned storage) of the FP32 W for the
// z pass with nz = 128 or 256; false if the grid has no such pass or the driver refuses
bool spec_make_zmap(const Spec<float>& V, void* map);
cudaError_t launch_elas32_scale_r(const Geo&, const Elas32&, cudaStream_t st);
cudaError_t launch_elas32_update_spec(const Geo&, const Elas32&, cudaStream_t st);

// ----------------------------------------------------------------------------- batches

struct Consts32 {   // FP32 copies of the grid constants the FP32 operator needs
  float ih2[3];
  float sc[3][3];
};

inline Consts32 make_consts32(const Geo& G) {
  Consts32 K;
  for (int d = 0; d < 3; ++d) K.ih2[d] = (float)G.ih2[d];
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) K.sc[a][d] = (float)G.s_cross[a][d];
  return K;
}

constexpr long long FLAT_GROUPS = 8LL * NT;   // float4 groups per flat work item

struct BSim {       // one simulation of a batch, as the batched kernels see it
  Geo G;            // its grid, with the batch's tile depth
  Consts32 K;
  Elas E;           // FP64 elasticity view (faces, u, force, du)
  Elas32 I;         // FP32 inner solve (I.S: inner CG scalars)
  Cn3 C;            // the three diffusion solves
  CgScal* Sout;     // outer (refinement) scalars of the elasticity solve
  int tile0, ntiles;   // its grid tiles in the batch's tile list
  int item0, nitems;   // its flat ranges in the batch's flat list
  long long n;
  double rtol_elas, rtol_diff;
  int maxit_elas, maxit_diff;
};

struct BatchDev {
  const BSim* sims;
  int nsims;
  const int* tile_sim;   // tile list -> simulation
  const int* item_sim;   // flat list -> simulation
  int ntiles, nitems;
  unsigned int* bar;     // [0] arrivals, [1] generation
  int* err;              // set by a barrier wait that ran out of time
  unsigned long long timeout_ns;
  int maxit;             // bound on the iterations of one persistent solve
  double tau_min;
  int max_sweeps;
};

struct BatchStat {
  int elas_status, elas_sweeps, elas_inner, pad;
  double elas_relres;
  int cn_status[3], cn_it[3];
  double cn_relres[3];
};

int batch_coop_blocks_per_sm(int which);   // 0: diffusion solver, 1: elasticity inner solver
cudaError_t launch_batch_reset(const BatchDev&, cudaStream_t st);
cudaError_t launch_batch_status(const BatchDev&, BatchStat* out, cudaStream_t st);
cudaError_t launch_batch_cn(const BatchDev&, int coop_blocks, cudaStream_t st);
cudaError_t launch_batch_sweep(const BatchDev&, int coop_blocks, cudaStream_t st);
cudaError_t launch_batch_elas_inner(const BatchDev&, int coop_blocks, cudaStream_t st);
cudaError_t launch_batch_residual(const BatchDev&, cudaStream_t st);
cudaError_t launch_batch_force_inner(const BatchDev&, cudaStream_t st);
cudaError_t launch_batch_finish(const BatchDev&, double inv_dt, cudaStream_t st);

// ----------------------------------------------------------------------------- adjoint

struct LamState {   // the caller's adjoint fields (one per state field; bg has none)
  double *p, *i, *n, *g, *w, *f, *o, *l;
  double* u[3];
  double* v[3];
};

struct TapeView {   // forward values of one step, recorded by tg_step
  const double *p, *i, *n, *g, *w, *f, *o, *l;   // state at the step's start
  const double* u[3];
  const double* v[3];
  const double *pdag, *idag, *ndag, *gdag, *wdag, *fplus;   // after transport (S1)
  const double *iddag, *odag, *ldag;                         // after diffusion (S2)
  const double* up[3];                                       // u after the elasticity solve
};

struct AdjView {
  LamState lam;
  double* rhs[3];     // right-hand side of the adjoint elasticity solve
  double* psi[3];     // its solution
  const double* up[3];
  double* LQ[7];      // lambda of the reacted p, i, n, g, w, o, l
  double* LF;         // lambda of f after transport
  double* LD[5];      // lambda of p, i, n, g, w after transport
  double* LCN[3];     // lambda of the CN outputs i, o, l
  double* phi[3];     // adjoint CN solutions
  double* LRHO;       // lambda of the proliferation field
  double* LDEL;       // lambda of div v
  double* LV[3];      // scattered part of lambda_v
  double* grad;       // dJ/dtheta accumulators (5, device)
  double* partial;
  unsigned int* counter;
};

cudaError_t launch_adj_prep(const Geo&, const AdjView&, double inv_dt, cudaStream_t st);
cudaError_t launch_adj_elas_coef(const Geo&, const DevParams&, const AdjView&, const double* mu,
                                 const double* lam, const double* p, const double* n,
                                 double inv_Escale, bool species, cudaStream_t st);
cudaError_t launch_adj_react(const Geo&, const DevParams&, double dt, const AdjView&,
                             const TapeView&, const double* rho, cudaStream_t st);
cudaError_t launch_cn_init_rhs(const Geo&, const Cn3&, const AdjView&, cudaStream_t st);
cudaError_t launch_adj_cn_post(const Geo&, const DevParams&, double dt, const AdjView&,
                               const TapeView&, cudaStream_t st);
cudaError_t launch_adj_sl(const Geo&, double dt, const AdjView&, const TapeView&,
                          const double* div, cudaStream_t st);
cudaError_t launch_adj_div(const Geo&, const AdjView&, cudaStream_t st);

}  // namespace tg
