// tg_api.cu -- the C ABI of tg.h: argument checks, workspace layout, and the host-side
// sequencing of the operator-split step (Section 3) over the kernels of this directory.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <atomic>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "tg_internal.cuh"

using namespace tg;

namespace tg {
thread_local const KHook* tg_khook = nullptr;
}  // namespace tg

namespace {

// ---------------------------------------------------------------------------- workspace
// Every array holds one FP64 value per voxel and starts on a 256-byte boundary.
enum Arr {
  A_KF0, A_KF1, A_KF2, A_DSUM_D, A_DINV_D, A_RHO,
  A_CR0, A_CR1, A_CR2, A_CP0, A_CP1, A_CP2, A_CQ0, A_CQ1, A_CQ2,
  A_IDAG, A_DIV, A_SL0, A_SL1, A_SL2, A_SL3, A_SL4, A_SL5,
  A_MU, A_LAM, A_ETA, A_F0, A_F1, A_F2, A_G0, A_G1, A_G2,
  A_DSUM_E0, A_DSUM_E1, A_DSUM_E2, A_DINV_E0, A_DINV_E1, A_DINV_E2,
  A_B0, A_B1, A_B2, A_DU0, A_DU1, A_DU2, A_ER0, A_ER1, A_ER2, A_EP0, A_EP1, A_EP2,
  A_EQ0, A_EQ1, A_EQ2,
  A_VP0, A_VP1, A_VP2,   // velocity at the previous step's start (quadratic extrapolation)
  // (hi, lo) FP32 pairs of u, mu, lambda for the double-FP32 residual (TG_MIXED only), and of
  // the diffusion faces and fields for the diffusion solves' double-FP32 residual
  A_UDF0, A_UDF1, A_UDF2, A_MUDF, A_LAMDF,
  A_KFDF0, A_KFDF1, A_KFDF2, A_XDF0, A_XDF1, A_XDF2,
  A_COUNT
};

// FP32 arrays of the mixed precision (one FP32 value per voxel each)
enum Arr32 {
  B_MU, B_LAM, B_ETA, B_DINV0, B_DINV1, B_DINV2,
  B_E0, B_E1, B_E2, B_R0, B_R1, B_R2, B_P0, B_P1, B_P2, B_PB0, B_PB1, B_PB2, B_Q0, B_Q1, B_Q2,
  B_SL0, B_SL1, B_SL2, B_SL3, B_SL4, B_SL5, B_SL6, B_SL7, B_SL8, B_SL9, B_SL10, B_SL11,
  B_CKF0, B_CKF1, B_CKF2, B_CDINV,   // FP32 CN faces and Jacobi inverse diagonal
  B_COUNT
};

// arrays of one step's tape (tg_step with a tape records them; tg_adjoint_step reads them)
enum TapeArr {
  T_P, T_I, T_N, T_G, T_W, T_F, T_O, T_L, T_U0, T_U1, T_U2, T_V0, T_V1, T_V2,
  T_PD, T_ID, T_ND, T_GD, T_WD, T_FP, T_IDD, T_OD, T_LD, T_UP0, T_UP1, T_UP2,
  T_COUNT
};

// FP64 scratch of the adjoint (present when the context was created with TG_INIT_ADJOINT)
enum AdjArr {
  C_QP0, C_QP1, C_QP2, C_QP3, C_QP4, C_QP5, C_QP6,
  C_PSI0, C_PSI1, C_PSI2, C_RHS0, C_RHS1, C_RHS2,
  C_LQ0, C_LQ1, C_LQ2, C_LQ3, C_LQ4, C_LQ5, C_LQ6, C_LF,
  C_LD0, C_LD1, C_LD2, C_LD3, C_LD4, C_LCN0, C_LCN1, C_LCN2,
  C_PHI0, C_PHI1, C_PHI2, C_LRHO, C_LDEL, C_LV0, C_LV1, C_LV2,
  C_COUNT
};

constexpr size_t ALIGN = 256;
constexpr int MAX_NV = 9;    // largest number of values reduced by one kernel
// 3 diffusion solves (outer in the mixed precision), elasticity (outer), elasticity inner
// FP32, 3 inner FP32 diffusion solves
constexpr int N_SCAL = 11;   // 3 CN, 2 elasticity, 3 inner CN, 3 concurrent CN
constexpr int MAX_SWEEPS = 64;        // refinement sweeps of one mixed-precision solve
constexpr double TAU_INNER = 1e-4;    // smallest relative reduction asked of an inner solve
// ... of a spectrally preconditioned inner elasticity solve: its few, well-conditioned FP32
// iterations reach 1e-6 without stagnating, so one sweep usually meets the FP64 tolerance
constexpr double TAU_INNER_SPECTRAL = 1e-6;
// Which of the diffusion solves (bits: i, o, l) the mixed precision refines around FP32.
// Oxygen stays FP64: a converged CN solve is fixed only to within its tolerance, and the
// necrotic source h(o) (p + i + g + w) turns an oxygen difference do into a relative
// difference of about (2 / eps_H) do = 200 do in n -- two solvers stopping at different
// points of the same tolerance then differ by ~5e-5 in n (64^3 brain, rtol 1e-8), more than
// the mixed precision's 1e-5.  i and l enter the other fields without such a gain.
constexpr int CN_MIXED_MASK = 0b101;

size_t round_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

bool grid_ok(const tg_grid* g) {
  if (!g) return false;
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] < 4 || g->n[d] > (1 << 20)) return false;
    if (!(g->L[d] > 0.0) || !isfinite(g->L[d])) return false;
  }
  return true;
}

Geo make_geo(const tg_grid* g, int sms) {
  Geo G;
  G.nx = g->n[0];
  G.ny = g->n[1];
  G.nz = g->n[2];
  G.nxy = (long long)G.nx * G.ny;
  G.nvox = G.nxy * G.nz;
  for (int d = 0; d < 3; ++d) {
    G.h[d] = g->L[d] / g->n[d];
    G.ih2[d] = 1.0 / (G.h[d] * G.h[d]);
    G.inv2h[d] = 1.0 / (2.0 * G.h[d]);
  }
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) G.s_cross[a][d] = 1.0 / (4.0 * G.h[a] * G.h[d]);
  const long long gx = (G.nx + BX - 1) / BX, gy = (G.ny + BY - 1) / BY;
  // z chunk so that a launch has about 16 blocks per SM
  const long long target = 16LL * std::max(sms, 1);
  long long zc = (gx * gy * G.nz + target - 1) / target;
  zc = std::max(1LL, std::min(zc, (long long)G.nz));
  G.zc = (int)zc;
  const long long gz = (G.nz + zc - 1) / zc;
  G.grid = dim3((unsigned)gx, (unsigned)gy, (unsigned)gz);
  G.nblocks = (int)(gx * gy * gz);
  return G;
}

// ---------------------------------------------------------------- spectral preconditioner
// Every axis a power of two in [4, 2048]: the FFT passes stage whole lines in shared memory.
bool spectral_precond(int pc) {
  return pc == TG_PRECOND_SPECTRAL || pc == TG_PRECOND_SPECTRAL_SCALED;
}

bool spectral_grid_ok(const Geo& G) {
  for (int n : {G.nx, G.ny, G.nz})
    if (n < 4 || n > 2048 || (n & (n - 1)) != 0) return false;
  return true;
}

int floor_pow2(long long v) {
  int p = 1;
  while ((long long)p * 2 <= v) p *= 2;
  return p;
}

// Line batch sizes of the passes: up to 64 KB of line buffers per block (two ping-pong
// buffers), at most 16 lines (so a radix-16 stage gives 256 threads n/16 butterflies of 16
// lines).  A z block has one thread per radix-16 butterfly of its 3 tz lines.
template <typename R>
void spec_shape(const Geo& G, Spec<R>& V) {
  const long long cs = sizeof(typename CxOf<R>::T);
  V.nx = G.nx;
  V.ny = G.ny;
  V.nz = G.nz;
  V.nxh = G.nx / 2 + 1;
  V.nxp = (V.nxh + 15) / 16 * 16;
  V.pb = std::max(1, std::min(std::min(G.ny / 2, 16), floor_pow2(65536 / (2 * G.nx * cs))));
  V.tx = std::max(1, std::min(16, floor_pow2(65536 / (2 * G.ny * cs))));
  V.tz = std::max(1, std::min(16, floor_pow2(65536 / (6 * G.nz * cs))));
  // in place when each x-pass stage (a radix 2/4/8 stage for ln mod 4, then radix 16) has at
  // most one butterfly per thread of a block
  {
    int ln = 0;
    while ((1 << ln) < G.nx) ++ln;
    const long long first = (long long)V.pb * G.nx >> ((ln & 3) ? (ln & 3) : 4);
    const long long r16 = (long long)V.pb * G.nx >> 4;
    V.x_inpl = std::max(first, r16) <= NT ? 1 : 0;
  }
  const int items = 3 * V.tz * std::max(1, G.nz / 16);
  V.nt_z = std::max(64, std::min(NT, (items + 31) / 32 * 32));
}

// partial sums: one per z-pass block (the <r, z> reduction) and the 1024 x 3 of the mean
// reduction, for the larger of the FP32 and FP64 shapes (the x-pass count is kept as a floor)
int spec_partial_count(const Geo& G) {
  Spec<float> a;
  Spec<double> b;
  spec_shape(G, a);
  spec_shape(G, b);
  const long long na = 3LL * G.nz * (G.ny / (2 * a.pb));
  const long long nb = 3LL * G.nz * (G.ny / (2 * b.pb));
  // the z pass reduces <r, z>: one partial per block
  const long long za = (long long)((a.nxh + a.tz - 1) / a.tz) * G.ny;
  const long long zb = (long long)((b.nxh + b.tz - 1) / b.tz) * G.ny;
  return (int)std::max<long long>(std::max(std::max(na, nb), std::max(za, zb)), 3 * 1024);
}

size_t spec_table_bytes(const Geo& G, size_t real_bytes) {
  const size_t n = (size_t)G.nx + G.ny + G.nz;
  return round_up(n * 2 * real_bytes) + round_up(n * 2 * real_bytes);  // roots; S and T
}

struct Layout {
  size_t arr[A_COUNT];
  size_t arr32[B_COUNT];
  size_t adj[C_COUNT];
  size_t partial, counter, scal, grad;
  size_t partial2, counter2;   // reductions of the oxygen solve running on the side stream
  size_t dmax;                 // the CN diagonal's maximum (mixed S0), one float
  bool spectral;
  size_t sp_w, sp_z32[3], sp_z64[3], sp_s32[3], sp_s64[3], sp_tab32, sp_tab64, sp_mean,
      sp_partial, sp_counter;
  size_t total;
};

Layout layout(const Geo& G, tg_precision prec, bool adjoint = false, bool spectral = false) {
  Layout L;
  size_t off = 0;
  const size_t abytes = round_up((size_t)G.nvox * sizeof(double));
  for (int a = 0; a < A_COUNT; ++a) {
    L.arr[a] = off;
    if (a < A_UDF0 || prec == TG_MIXED) off += abytes;
  }
  const size_t fbytes = round_up((size_t)G.nvox * sizeof(float));
  // FP32 arrays: the mixed precision, and the adjoint's refined elasticity solves
  for (int b = 0; b < B_COUNT; ++b) {
    L.arr32[b] = off;
    if (prec == TG_MIXED || adjoint) off += fbytes;
  }
  for (int c = 0; c < C_COUNT; ++c) {
    L.adj[c] = off;
    if (adjoint) off += abytes;
  }
  L.partial = off;
  off += round_up((size_t)G.nblocks * MAX_NV * sizeof(double));
  L.counter = off;
  off += ALIGN;
  L.scal = off;
  off += round_up(N_SCAL * sizeof(CgScal));
  L.grad = off;
  off += ALIGN;
  L.partial2 = off;
  if (prec == TG_MIXED) off += round_up((size_t)G.nblocks * MAX_NV * sizeof(double));
  L.counter2 = off;
  if (prec == TG_MIXED) off += ALIGN;
  L.dmax = off;
  off += ALIGN;
  // spectral preconditioner: the FP32 form serves the mixed precision and the adjoint's
  // refined solves, the FP64 form the FP64 solves; one half-spectrum buffer serves both
  L.spectral = spectral;
  const bool need32 = spectral && (prec == TG_MIXED || adjoint);
  const bool need64 = spectral && prec == TG_FP64;
  Spec<float> s32;
  spec_shape(G, s32);
  const size_t wmodes = (size_t)3 * G.nz * G.ny * s32.nxp;
  L.sp_w = off;
  if (spectral) off += round_up(wmodes * (need64 ? sizeof(double2) : sizeof(float2)));
  for (int d = 0; d < 3; ++d) {
    L.sp_z32[d] = off;
    if (need32) off += fbytes;
  }
  for (int d = 0; d < 3; ++d) {
    L.sp_z64[d] = off;
    if (need64) off += abytes;
  }
  // the diagonal scaling of TG_PRECOND_SPECTRAL_SCALED (any spectral context may switch to it)
  for (int d = 0; d < 3; ++d) {
    L.sp_s32[d] = off;
    if (need32) off += fbytes;
  }
  for (int d = 0; d < 3; ++d) {
    L.sp_s64[d] = off;
    if (need64) off += abytes;
  }
  L.sp_tab32 = off;
  if (need32) off += spec_table_bytes(G, sizeof(float));
  L.sp_tab64 = off;
  if (need64) off += spec_table_bytes(G, sizeof(double));
  L.sp_mean = off;
  if (spectral) off += ALIGN;
  L.sp_partial = off;
  if (spectral) off += round_up((size_t)spec_partial_count(G) * sizeof(double));
  L.sp_counter = off;
  if (spectral) off += ALIGN;
  L.total = off;
  return L;
}

template <typename R>
Spec<R> spec_view(const Geo& G, const Layout& L, char* ws, size_t tab_off) {
  using C = typename CxOf<R>::T;
  Spec<R> V;
  spec_shape(G, V);
  V.W = (C*)(ws + L.sp_w);
  const int n[3] = {G.nx, G.ny, G.nz};
  const size_t ntot = (size_t)G.nx + G.ny + G.nz;
  C* tw = (C*)(ws + tab_off);
  R* st = (R*)(ws + tab_off + round_up(ntot * sizeof(C)));
  for (int d = 0; d < 3; ++d) {
    V.tw[d] = tw;
    tw += n[d];
    V.S[d] = st;
    st += n[d];
  }
  for (int d = 0; d < 3; ++d) {
    V.T[d] = st;
    st += n[d];
  }
  for (int d = 0; d < 3; ++d) V.s[d] = nullptr;
  V.mean = (double*)(ws + L.sp_mean);
  V.partial = (double*)(ws + L.sp_partial);
  V.counter = (unsigned int*)(ws + L.sp_counter);
  V.nb_partial = spec_partial_count(G);
  V.zmap = nullptr;
  return V;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return sms;
}

bool params_ok(const tg_params* p) {
  if (!p) return false;
  if (p->model != TG_MODEL_MULTISPECIES && p->model != TG_MODEL_SINGLE) return false;
  if (p->precond_elas != TG_PRECOND_JACOBI && p->precond_elas != TG_PRECOND_SPECTRAL &&
      p->precond_elas != TG_PRECOND_SPECTRAL_SCALED)
    return false;
  if (!(p->eps_H > 0.0)) return false;
  if (!(p->o_inv > 0.5 * (p->o_hyp + p->o_inv)) && !(p->o_inv < 0.5 * (p->o_hyp + p->o_inv)))
    return false;  // o_inv == o_mit: the ramp of Eq. e:gog_reac_op is undefined
  if (!(p->rtol_diff >= 0.0) || !(p->rtol_elas >= 0.0)) return false;
  if (p->maxit_diff < 0 || p->maxit_elas < 0) return false;
  for (int s = 0; s < 5; ++s) {
    if (p->nu[s] == 0.5 || p->nu[s] == -1.0) return false;
    if (!isfinite(p->E[s]) || !isfinite(p->nu[s]) || !isfinite(p->eta[s])) return false;
  }
  return true;
}

DevParams make_dev_params(const tg_params* p) {
  DevParams d;
  d.k_g = p->k_g;
  d.k_w = p->k_w;
  d.k_f = p->k_f;
  d.k_scale = p->k_scale;
  d.rho_g = p->rho_g;
  d.rho_w = p->rho_w;
  d.rho_i_frac = p->rho_i_frac;
  d.alpha0 = p->alpha0;
  d.beta0 = p->beta0;
  d.gamma = p->gamma;
  d.sigma_b = p->sigma_b;
  d.o_hyp = p->o_hyp;
  d.o_inv = p->o_inv;
  d.o_heal = p->o_heal;
  d.o_mit = 0.5 * (p->o_hyp + p->o_inv);
  d.delta_s = p->delta_s;
  d.delta_p = p->delta_p;
  d.inv_eps_H = 1.0 / p->eps_H;
  for (int s = 0; s < 5; ++s) {
    const double E = p->E_scale * p->E[s], nu = p->nu[s];
    d.cmu[s] = E / (2.0 * (1.0 + nu));
    d.clam[s] = nu * E / ((1.0 - 2.0 * nu) * (1.0 + nu));
    d.eta[s] = p->eta[s];
  }
  d.zeta = p->zeta;
  d.delta_e = p->delta_e;
  d.delta_half = p->delta_half;
  d.delta_l = p->delta_l;
  return d;
}

__global__ void k_cg_reset(CgScal* S, int count, double rtol, int maxit) {
  const int t = threadIdx.x;
  if (t < count) {
    CgScal s = {};
    s.rtol = rtol;
    s.maxit = maxit;
    s.status = CG_RUNNING;
    S[t] = s;
  }
}

// Per-kernel timing of one context (tg_set_timing).  Each timed launch is bracketed by two
// events on its stream; launches inside a CG solve carry the iteration they belong to and the
// solve's slot, and count only if the solve was still running at that iteration (a host-driven
// solve queues iterations ahead and the ones after convergence return at once).
struct KRec {
  int kid, e0, e1, iter, slot;
};

struct Prof {
  KHook hook;
  std::vector<cudaEvent_t> ev;   // pool, reused every step
  int next;                      // first unused event of the pool
  std::vector<KRec> recs;        // launches of the current step
  std::vector<int> did;          // per solve slot: iterations that did work
  int iter, slot;                // tag of the launches being queued (-1: not in a CG loop)
  cudaStream_t open_st[4];       // stream -> its pending start event
  int open_ev[4];
  double call_ms[K_COUNT];       // this call
  long long call_n[K_COUNT];
  double cum_ms[K_COUNT];        // since timing was switched on
  long long cum_n[K_COUNT];
};

const char* const kKernelNames[K_COUNT] = {
    "k_diff_faces", "k_diff_diag", "k_to_f32", "k_divergence", "k_sl", "k_sl32",
    "k_cn_init", "k_cn_matvec", "k_cn_update", "k_cn_pupdate",
    "k_cn_ir_residual", "k_cn_ir_residual_df", "k_cn32_pupdate", "k_cn32_matvec",
    "k_cn32_update", "k_cn_ir_correct", "k_cn32_neumann", "k_diff_node_df", "k_diff_faces_df",
    "k_react", "k_lame", "k_elas_coef", "k_elas_coef_df",
    "k_elas32_coef", "k_df_pack3", "k_elas_extrapolate", "k_spec_mean", "k_spec_scale",
    "k_elas_ir_residual", "k_elas_ir_residual_df", "k_elas32_scale_r", "k_spec_x_fwd",
    "k_spec_y_fwd", "k_spec_z", "k_spec_zr", "k_spec_y_inv", "k_spec_x_inv", "k_spec_x_inv_p",
    "k_elas32_matvec", "k_elas32_update", "k_elas32_matvec_spec", "k_elas32_update_spec",
    "k_spec_update_xfwd", "k_elas_ir_correct", "k_elas_ir_finish", "k_elas_init",
    "k_elas_init_spec", "k_elas_matvec", "k_elas_update", "k_elas_pupdate", "k_elas_update_spec",
    "k_elas_pupdate_spec", "k_elas_finish", "k_ox_prep", "k_ox_init", "k_ox_matvec",
    "k_ox_update", "k_ox_pupdate", "k_ox_finish", "k_sl32_pack", "k_lame_df"};

}  // namespace

struct tg_ctx {
  Geo G;
  Layout L;
  tg_params prm;
  DevParams dp;
  tg_precision prec;
  tg_state st;
  cudaStream_t stream;
  int device;
  char* ws;
  double* a[A_COUNT];
  float* b32[B_COUNT];   // valid in TG_MIXED only
  double* adj[C_COUNT];  // valid with TG_INIT_ADJOINT only
  bool has_adjoint;
  bool psi_valid;        // the adjoint scratch holds the previous adjoint solution (warm start)
  double* grad;          // 5 device accumulators of dJ/dtheta
  double* tape[T_COUNT]; // tape being recorded by the current step, or null
  double* partial;
  unsigned int* counter;
  CgScal* scal;
  // TG_MIXED: the FP64 oxygen solve of S2 runs on a side stream (created on first use),
  // forked from and joined to the context's stream by events, with its own reductions
  double* partial2;
  unsigned int* counter2;
  float* dmax;   // max over nodes of the CN diagonal 1 + sum of faces, from S0 (mixed)
  cudaStream_t side;
  cudaEvent_t fork_ev, join_ev;
  // the oxygen solve of the mixed step, running on the side stream from S0 on: its first
  // chunk of iterations and profiler slot (ox_begin) until ox_end drives the rest and joins
  bool ox_running;
  int ox_chunk, ox_slot;
  // tg_step_host: the caller's host copies of the state and the copy stream that moves u up
  // during S0-S5 and the species down during S6-S7
  const tg_state* host_in;
  tg_state* host_out;
  cudaStream_t copy;
  cudaEvent_t entry_ev, up_ev[4], s5_ev;
  int broken;
  int prev_it_diff;
  int prev_it_elas;
  int prev_it_inner[2];   // inner FP32 iterations of the first and of later refinement sweeps
  int prev_it_cn_inner[2];  // the same for the mixed precision's diffusion solves
  // profiling: launches queued, and optional event timing of every kernel (tg_set_timing)
  long long launches;
  int timing;
  Prof prof;
  bool df_res;           // the mixed precision's residual in double-FP32 (df_residual_ok)
  bool cn_df;            // ... and that of its diffusion solves (cn_df_ok)
  bool in_batch;         // owned by a batch (its persistent solvers read FP64 faces)
  bool hist_ok;          // the A_VP arrays hold the previous step's starting velocity: the next
                         // step's elasticity solve starts from the quadratic extrapolation
  cudaEvent_t pev[5];    // phase boundaries of a step (created on first use)
  bool pev_ok;
  double t_phase[4];
  // spectral elasticity preconditioner (workspace sized for it when L.spectral)
  Spec<float> sp32;      // FP32 form: mixed precision, adjoint refined solves
  alignas(64) unsigned char zmap32[128];   // TMA tensor map of sp32.W for its z pass
  Spec<double> sp64;     // FP64 form: FP64 solves
  float* z32[3];
  double* z64[3];
  float* s32[3];         // diagonal scaling of TG_PRECOND_SPECTRAL_SCALED
  double* s64[3];
};

namespace {

tg_status fail(tg_ctx* X, tg_status s) {
  if (X && s != TG_OK && s != TG_ERR_ARG) X->broken = 1;
  return s;
}

#define CK(call)                                  \
  do {                                            \
    if ((call) != cudaSuccess) {                  \
      return fail(X, TG_ERR_CUDA);                \
    }                                             \
  } while (0)

tg_status status_of(const CgScal& s) {
  switch (s.status) {
    case CG_CONVERGED:
    case CG_ZERO_RHS: return TG_OK;
    case CG_NONFINITE: return TG_ERR_NONFINITE;
    case CG_MAXIT: return TG_ERR_NOCONV;
    case CG_TIMEOUT: return TG_ERR_TIMEOUT;
    default: return TG_ERR_CUDA;
  }
}

// ---------------------------------------------------------------- per-kernel timing
int prof_event(tg_ctx* X) {
  Prof& P = X->prof;
  if (P.next == (int)P.ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    P.ev.push_back(e);
  }
  return P.next++;
}

int prof_open_index(const Prof& P, cudaStream_t st) {
  for (int k = 0; k < 4; ++k)
    if (P.open_ev[k] >= 0 && P.open_st[k] == st) return k;
  return -1;
}

void prof_pre(void* self, cudaStream_t st) {
  tg_ctx* X = static_cast<tg_ctx*>(self);
  Prof& P = X->prof;
  int k = prof_open_index(P, st);
  if (k < 0)
    for (k = 0; k < 4 && P.open_ev[k] >= 0; ++k) {
    }
  if (k >= 4) return;
  const int e = prof_event(X);
  if (e < 0 || cudaEventRecord(P.ev[e], st) != cudaSuccess) return;
  P.open_st[k] = st;
  P.open_ev[k] = e;
}

void prof_post(void* self, int kid, cudaStream_t st) {
  tg_ctx* X = static_cast<tg_ctx*>(self);
  Prof& P = X->prof;
  const int k = prof_open_index(P, st);
  if (k < 0) return;
  const int e0 = P.open_ev[k];
  P.open_ev[k] = -1;
  const int e = prof_event(X);
  if (e < 0 || cudaEventRecord(P.ev[e], st) != cudaSuccess) return;
  P.recs.push_back({kid, e0, e, P.iter, P.slot});
}

void prof_reset_step(Prof& P) {
  P.next = 0;
  P.recs.clear();
  P.did.clear();
  P.iter = -1;
  P.slot = -1;
  for (int k = 0; k < 4; ++k) P.open_ev[k] = -1;
}

// a CG solve whose iterations are about to be queued: its slot, or -1 with timing off
int prof_open_solve(tg_ctx* X) {
  if (!X->timing) return -1;
  X->prof.did.push_back(INT_MAX);
  return (int)X->prof.did.size() - 1;
}

void prof_iter(tg_ctx* X, int slot, int q) {
  X->prof.slot = slot;
  X->prof.iter = slot >= 0 ? q : -1;
}

void prof_close_solve(tg_ctx* X, int slot, const CgScal* host, int nsolves) {
  X->prof.iter = -1;
  X->prof.slot = -1;
  if (slot < 0) return;
  int did = 0;
  for (int r = 0; r < nsolves; ++r) did = std::max(did, host[r].it);
  X->prof.did[slot] = did;
}

// after a step (its streams synchronised): add the launches that did work, then reuse the pool
void prof_harvest(tg_ctx* X) {
  Prof& P = X->prof;
  for (const KRec& r : P.recs) {
    if (r.iter >= 0 && r.slot >= 0 && r.slot < (int)P.did.size() && r.iter >= P.did[r.slot])
      continue;
    float ms = 0.0f;
    if (cudaEventSynchronize(P.ev[r.e1]) != cudaSuccess) continue;
    if (cudaEventElapsedTime(&ms, P.ev[r.e0], P.ev[r.e1]) != cudaSuccess) continue;
    P.call_ms[r.kid] += ms;
    P.call_n[r.kid] += 1;
    P.cum_ms[r.kid] += ms;
    P.cum_n[r.kid] += 1;
  }
  prof_reset_step(P);
}

// installs the context's timing hook for the calling thread while a call runs
struct HookScope {
  const KHook* saved;
  explicit HookScope(tg_ctx* X) : saved(tg_khook) {
    if (!X->timing) return;
    X->prof.hook = {prof_pre, prof_post, X};
    prof_reset_step(X->prof);
    tg_khook = &X->prof.hook;
  }
  ~HookScope() { tg_khook = saved; }
};

// Queue iterations in chunks and read the device-side flags back between chunks.  Kernels of
// a finished solve return at once, so overshooting a chunk only costs empty launches.
// On stream st; `queued` iterations may already be in flight (then the loop reads the flags
// first).
int first_chunk(int prev) { return prev > 0 ? std::max(1, prev - prev / 8) : 4; }

template <class IterFn>
tg_status drive_cg_loop(tg_ctx* X, cudaStream_t st, IterFn iter, const CgScal* dev, int nsolves,
                        int maxit, int prev, CgScal* host, long long queued, int slot) {
  int chunk = queued > 0 ? 0 : first_chunk(prev);
  const long long first = queued > 0 ? queued : chunk;
  for (;;) {
    for (int c = 0; c < chunk; ++c) {
      prof_iter(X, slot, (int)(queued + c));
      CK(iter((int)(queued + c)));
    }
    queued += chunk;
    CK(cudaMemcpyAsync(host, dev, nsolves * sizeof(CgScal), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool running = false;
    for (int r = 0; r < nsolves; ++r) running |= host[r].status == CG_RUNNING;
    if (!running) return TG_OK;
    if (queued > (long long)maxit + 64) return fail(X, TG_ERR_CUDA);  // flags never settled
    chunk = (queued == first) ? 2 : std::min(chunk * 2, 32);
  }
}

// slot: the timing slot of a solve whose first iterations the caller queued itself (with
// prof_iter tags), or INT_MIN to open one here
template <class IterFn>
tg_status drive_cg_on(tg_ctx* X, cudaStream_t st, IterFn iter, const CgScal* dev, int nsolves,
                      int maxit, int prev, CgScal* host, long long queued = 0,
                      int slot = INT_MIN) {
  if (slot == INT_MIN) slot = prof_open_solve(X);
  const tg_status s = drive_cg_loop(X, st, iter, dev, nsolves, maxit, prev, host, queued, slot);
  prof_close_solve(X, slot, host, nsolves);
  return s;
}

template <class IterFn>
tg_status drive_cg(tg_ctx* X, IterFn iter, const CgScal* dev, int nsolves, int maxit, int prev,
                   CgScal* host) {
  return drive_cg_on(X, X->stream, iter, dev, nsolves, maxit, prev, host);
}

// the single-species model (Eq. e:rd): c is carried in p, only it diffuses
bool single_species(const tg_ctx* X) { return X->prm.model == TG_MODEL_SINGLE; }

Cn3 cn_view(tg_ctx* X) {
  Cn3 C;
  // the diffusing fields: i, o, l (multispecies) or c in the first slot (single species)
  double* xs[3] = {single_species(X) ? X->st.p : X->st.i, X->st.o, X->st.l};
  for (int r = 0; r < 3; ++r) {
    C.x[r] = xs[r];
    C.r[r] = X->a[A_CR0 + r];
    C.p[r] = X->a[A_CP0 + r];
    C.q[r] = X->a[A_CQ0 + r];
    C.Kf[r] = X->a[A_KF0 + r];
  }
  C.dsum = X->a[A_DSUM_D];
  C.dinv = X->a[A_DINV_D];
  C.S = X->scal;
  C.partial = X->partial;
  C.counter = X->counter;
  C.df = X->cn_df ? 1 : 0;
  for (int r = 0; r < 3; ++r) {
    C.xdf[r] = X->cn_df ? reinterpret_cast<float2*>(X->a[A_XDF0 + r]) : nullptr;
    C.Kfdf[r] = X->cn_df ? reinterpret_cast<const float2*>(X->a[A_KFDF0 + r]) : nullptr;
  }
  return C;
}

// the context's elasticity solves use a spectral preconditioner (its workspace has the buffers)
bool spectral_on(const tg_ctx* X) {
  return X->L.spectral && spectral_precond(X->prm.precond_elas);
}

Elas elas_view(tg_ctx* X, double* const u[3], double* const b[3]) {
  Elas E;
  E.mu = X->a[A_MU];
  E.lam = X->a[A_LAM];
  E.eta = X->a[A_ETA];
  for (int d = 0; d < 3; ++d) {
    E.F[d] = X->a[A_F0 + d];
    E.G[d] = X->a[A_G0 + d];
    E.dsum[d] = X->a[A_DSUM_E0 + d];
    E.dinv[d] = X->a[A_DINV_E0 + d];
    E.b[d] = b ? b[d] : X->a[A_B0 + d];
    E.du[d] = X->a[A_DU0 + d];
    E.r[d] = X->a[A_ER0 + d];
    E.p[d] = X->a[A_EP0 + d];
    E.q[d] = X->a[A_EQ0 + d];
    E.u[d] = u[d];
    E.v[d] = X->st.v[d];
    E.vp[d] = X->a[A_VP0 + d];
    E.z[d] = X->z64[d];
    E.udf[d] = reinterpret_cast<float2*>(X->a[A_UDF0 + d]);
  }
  E.df = X->df_res ? 1 : 0;
  E.jacobi = spectral_on(X) ? 0 : 1;
  E.mudf = reinterpret_cast<float2*>(X->a[A_MUDF]);
  E.lamdf = reinterpret_cast<float2*>(X->a[A_LAMDF]);
  E.S = X->scal + 3;
  E.partial = X->partial;
  E.counter = X->counter;
  return E;
}

// The mixed precision's FP64 residual runs in double-FP32 arithmetic when the tolerance allows
// it: its ~48-bit significand resolves residuals down to about 1e-13 of |A||u|, ample for
// rtol_elas >= 1e-10; deeper tolerances, adjoint contexts and batches keep FP64.
constexpr double DF_RTOL_MIN = 1e-10;
bool df_residual_ok(const tg_ctx* X) {
  return X->prec == TG_MIXED && !X->has_adjoint && !X->in_batch &&
         X->prm.rtol_elas >= DF_RTOL_MIN;
}
bool cn_df_ok(const tg_ctx* X) {
  return X->prec == TG_MIXED && !X->has_adjoint && !X->in_batch &&
         X->prm.rtol_diff >= DF_RTOL_MIN;
}

// S2: the three Crank-Nicolson solves (i, o, l) on the faces built by S0.
// mask: bit r set for the fields this call solves (the others are left untouched)
tg_status cn_solve3(tg_ctx* X, tg_stats* stats, int mask = 7) {
  const Cn3 C = cn_view(X);
  k_cg_reset<<<1, 32, 0, X->stream>>>(X->scal, 3, X->prm.rtol_diff, X->prm.maxit_diff);
  CK(cudaGetLastError());
  CK(launch_cn_init(X->G, C, X->stream, mask));
  X->launches += 2;
  CgScal host[3];
  tg_status s = drive_cg(X, [&](int) {
    X->launches += 3;
    return launch_cn_iter(X->G, C, X->stream);
  }, X->scal, 3, X->prm.maxit_diff, X->prev_it_diff, host);
  if (s != TG_OK) return s;
  int itmax = 0;
  for (int r = 0; r < 3; ++r) {
    if (!((mask >> r) & 1)) continue;
    if (host[r].status == CG_ZERO_RHS)
      CK(cudaMemsetAsync(C.x[r], 0, (size_t)X->G.nvox * sizeof(double), X->stream));
    itmax = std::max(itmax, host[r].it);
    if (stats) {
      stats->it_diff[r] = host[r].it;
      stats->relres_diff[r] = host[r].bb > 0.0 ? sqrt(host[r].rr / host[r].bb) : 0.0;
      stats->it_diff_total += host[r].it;
    }
  }
  X->prev_it_diff = itmax;
  for (int r = 0; r < 3; ++r) {
    tg_status e = status_of(host[r]);
    if (e != TG_OK) return fail(X, e);
  }
  return TG_OK;
}

Cn32 cn32_view(tg_ctx* X) {
  Cn32 I;
  for (int r = 0; r < 3; ++r) {   // the elasticity's FP32 CG vectors are free during S2
    I.e[r] = X->b32[B_E0 + r];
    I.r[r] = X->b32[B_R0 + r];
    I.p[r] = X->b32[B_P0 + r];
    I.q[r] = X->b32[B_Q0 + r];
    I.Kf[r] = X->b32[B_CKF0 + r];
  }
  I.dinv = X->b32[B_CDINV];
  I.dmax = X->cn_df ? X->dmax : nullptr;
  for (int r = 0; r < 3; ++r) {
    I.z[r] = nullptr;
    I.palt[r] = X->b32[B_SL0 + r];   // the transport's inputs are free after S1
  }
  I.S = X->scal + 5;
  I.partial = X->partial;
  I.counter = X->counter;
  return I;
}

// S2 in the mixed precision: FP64 residuals around FP32 inner solves (the FP32 faces and
// diagonal were written in S0).  Statistics count inner iterations.  The inner CG of up to two
// solves is preconditioned by the Neumann-series polynomial (launch_cn32_iter), which needs
// about a third of Jacobi's iterations at 256^3; z lives in the elasticity's second p buffer,
// free during S2.
tg_status cn_solve3_mixed(tg_ctx* X, tg_stats* stats, int mask) {
  const Cn3 C = cn_view(X);
  Cn32 I = cn32_view(X);
  int slot[2] = {-1, -1}, nslot = 0;
  for (int r = 0; r < 3; ++r)
    if ((mask >> r) & 1) {
      if (nslot < 2) slot[nslot] = r;
      ++nslot;
    }
  if (nslot <= 2)
    for (int q = 0; q < nslot; ++q) I.z[slot[q]] = X->b32[B_PB0 + slot[q]];
  const long long cap = (long long)X->G.nblocks * MAX_NV;
  k_cg_reset<<<1, 32, 0, X->stream>>>(X->scal, 3, X->prm.rtol_diff, X->prm.maxit_diff);
  CK(cudaGetLastError());
  X->launches += 1;
  int inner_total[3] = {0, 0, 0};
  int sweeps = 0;
  CgScal out[3];
  if (C.df) {   // (hi, lo) pairs of the fields for the first double-FP32 residual
    // only the solved fields are read and only their pairs written: oxygen may be in its own
    // solve on the side stream, whose double-FP32 iterate lives in the oxygen pair array (an
    // unsolved slot repeats the first solved one, the same value to the same address)
    const int f0 = (mask & 1) ? 0 : ((mask & 4) ? 2 : 1);
    auto pick = [&](int r) { return ((mask >> r) & 1) ? r : f0; };
    double* const pk[3] = {reinterpret_cast<double*>(C.xdf[pick(0)]),
                           reinterpret_cast<double*>(C.xdf[pick(1)]),
                           reinterpret_cast<double*>(C.xdf[pick(2)])};
    const double* const src[3] = {C.x[pick(0)], C.x[pick(1)], C.x[pick(2)]};
    CK(launch_df_pack3(X->G, src, pk, X->stream));
    X->launches += 1;
  }
  for (;;) {
    CK(launch_cn_ir_residual(X->G, C, I, X->scal, sweeps == 0, TAU_INNER, MAX_SWEEPS, mask,
                             X->stream));
    X->launches += 1;
    CK(cudaMemcpyAsync(out, X->scal, 3 * sizeof(CgScal), cudaMemcpyDeviceToHost, X->stream));
    CK(cudaStreamSynchronize(X->stream));
    bool any = false;
    for (int r = 0; r < 3; ++r) any |= out[r].status == CG_RUNNING;
    if (!any) break;
    CgScal host[3];
    const int sw = sweeps == 0 ? 0 : 1;
    tg_status st = drive_cg(X, [&](int) {
      X->launches += 3;
      return launch_cn32_iter(X->G, I, X->stream, slot[0], slot[1], cap);
    }, I.S, 3, X->prm.maxit_diff, X->prev_it_cn_inner[sw], host);
    if (st != TG_OK) return st;
    int itmax = 0;
    for (int r = 0; r < 3; ++r) {
      if (out[r].status == CG_RUNNING) inner_total[r] += host[r].it;
      itmax = std::max(itmax, host[r].it);
      if (host[r].status == CG_NONFINITE) return fail(X, TG_ERR_NONFINITE);
    }
    X->prev_it_cn_inner[sw] = itmax;
    CK(launch_cn_ir_correct(X->G, C, I, mask, X->stream));
    X->launches += 1;
    ++sweeps;
  }
  for (int r = 0; r < 3; ++r) {
    if (!((mask >> r) & 1)) continue;
    if (out[r].status == CG_ZERO_RHS)
      CK(cudaMemsetAsync(C.x[r], 0, (size_t)X->G.nvox * sizeof(double), X->stream));
    if (stats) {
      stats->it_diff[r] = inner_total[r];
      stats->relres_diff[r] = out[r].bb > 0.0 ? sqrt(out[r].rr / out[r].bb) : 0.0;
      stats->it_diff_total += inner_total[r];
    }
  }
  for (int r = 0; r < 3; ++r) {
    tg_status e = status_of(out[r]);
    if (e != TG_OK) return fail(X, e);
  }
  return TG_OK;
}

// the mixed precision's double-FP32 oxygen solve: pairs in the FP64 arrays of the oxygen CG
// (free then), the diagonal pairs in those of the FP64 diagonal (S0 copied what the FP32 solves
// need before S2 starts), face pairs from S0; scalars and reductions of the side stream
OxDf ox_view(tg_ctx* X) {
  OxDf O;
  for (int d = 0; d < 3; ++d) O.Kf[d] = reinterpret_cast<const float2*>(X->a[A_KFDF0 + d]);
  O.dd = reinterpret_cast<float2*>(X->a[A_DSUM_D]);
  O.di = reinterpret_cast<float2*>(X->a[A_DINV_D]);
  O.x = reinterpret_cast<float2*>(X->a[A_XDF1]);
  O.r = reinterpret_cast<float2*>(X->a[A_CR1]);
  O.p = reinterpret_cast<float2*>(X->a[A_CP1]);
  O.q = reinterpret_cast<float2*>(X->a[A_CQ1]);
  O.o = X->st.o;
  O.S = X->scal + 9;
  O.partial = X->partial2;
  O.counter = X->counter2;
  return O;
}

// The oxygen solve of the mixed multispecies step runs on a side stream, concurrently with the
// FP32-refined i and l solves on the context's stream.  It follows the FP64 CG's iterates: in
// double-FP32 arithmetic (tg_cn_ox.cu) when the face pairs exist (cn_df), else in FP64, with
// its own CG scalars (scal + 8 .. 10) and reduction buffers.  It needs only the S0 faces and
// o, which the transport does not touch, so it is forked right after S0 (ox_begin): its start
// and first chunk of iterations overlap the transport (L1-bound) and then the i, l solves;
// ox_end drives its remaining iterations, finishes and joins.  OxGuard keeps no side-stream
// work alive past an early return.
struct OxParts {
  Cn3 C;
  OxDf O;
  CgScal* dev;
  int ns;
  bool df;
};

OxParts ox_parts(tg_ctx* X) {
  OxParts P;
  P.df = X->cn_df;
  P.C = cn_view(X);
  P.C.S = X->scal + 8;
  P.C.partial = X->partial2;
  P.C.counter = X->counter2;
  P.C.df = 0;
  P.O = ox_view(X);
  P.dev = P.df ? P.O.S : P.C.S;   // the oxygen entry of the device scalars
  P.ns = P.df ? 1 : 3;
  return P;
}

tg_status ox_begin(tg_ctx* X) {
  constexpr int MASK_O = 7 & ~CN_MIXED_MASK;
  if (!X->side) {   // default priority (the highest measured no better)
    CK(cudaStreamCreateWithFlags(&X->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&X->fork_ev, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&X->join_ev, cudaEventDisableTiming));
  }
  cudaStream_t so = X->side;
  const OxParts P = ox_parts(X);
  CK(cudaEventRecord(X->fork_ev, X->stream));
  CK(cudaStreamWaitEvent(so, X->fork_ev, 0));
  if (X->host_in) CK(cudaStreamWaitEvent(so, X->up_ev[2], 0));   // o is up (tg_step_host)
  X->ox_running = true;
  k_cg_reset<<<1, 32, 0, so>>>(P.dev, P.ns, X->prm.rtol_diff, X->prm.maxit_diff);
  CK(cudaGetLastError());
  CK(P.df ? launch_ox_start(X->G, P.O, so) : launch_cn_init(X->G, P.C, so, MASK_O));
  X->ox_chunk = first_chunk(X->prev_it_diff);
  X->ox_slot = prof_open_solve(X);
  for (int c = 0; c < X->ox_chunk; ++c) {
    prof_iter(X, X->ox_slot, c);
    X->launches += 3;
    CK(P.df ? launch_ox_iter(X->G, P.O, so) : launch_cn_iter(X->G, P.C, so));
  }
  prof_iter(X, -1, -1);
  X->launches += 2 + (P.df ? 1 : 0);
  return TG_OK;
}

tg_status ox_end(tg_ctx* X, tg_stats* stats) {
  cudaStream_t so = X->side;
  const OxParts P = ox_parts(X);
  auto iter = [&](int) -> cudaError_t {
    X->launches += 3;
    return P.df ? launch_ox_iter(X->G, P.O, so) : launch_cn_iter(X->G, P.C, so);
  };
  CgScal host[3];
  tg_status e = drive_cg_on(X, so, iter, P.dev, P.ns, X->prm.maxit_diff, X->prev_it_diff, host,
                            X->ox_chunk, X->ox_slot);
  if (e != TG_OK) return e;
  const CgScal& ho = P.df ? host[0] : host[1];
  if (P.df) {
    CK(launch_ox_finish(X->G, P.O, so));
    X->launches += 1;
  } else if (ho.status == CG_ZERO_RHS) {
    CK(cudaMemsetAsync(P.C.x[1], 0, (size_t)X->G.nvox * sizeof(double), so));
  }
  CK(cudaEventRecord(X->join_ev, so));
  CK(cudaStreamWaitEvent(X->stream, X->join_ev, 0));
  X->ox_running = false;
  X->prev_it_diff = ho.it;
  if (stats) {
    stats->it_diff[1] = ho.it;
    stats->relres_diff[1] = ho.bb > 0.0 ? sqrt(ho.rr / ho.bb) : 0.0;
    stats->it_diff_total += ho.it;
  }
  e = status_of(ho);
  return e == TG_OK ? TG_OK : fail(X, e);
}

// on an early return between ox_begin and ox_end: wait for the side stream's work
struct OxGuard {
  tg_ctx* X;
  ~OxGuard() {
    if (X->ox_running) {
      cudaStreamSynchronize(X->side);
      X->ox_running = false;
    }
  }
};

// The interleaved inputs of the FP32 transport.  The FP32 arrays are consecutive, each at
// least nvox * 4 bytes and 256-byte aligned, so four of them hold one float4 per voxel.
Sl32 sl32_view(tg_ctx* X) {
  tg_state& S = X->st;
  Sl32 T;
  T.v4 = reinterpret_cast<float4*>(X->b32[B_SL0]);
  T.qa = reinterpret_cast<float4*>(X->b32[B_SL4]);
  T.qb = reinterpret_cast<float4*>(X->b32[B_SL8]);
  double* const outs[6] = {S.p, S.i, S.n, S.g, S.w, S.f};
  for (int q = 0; q < 6; ++q) T.out[q] = outs[q];
  return T;
}

Elas32 elas32_view(tg_ctx* X) {
  Elas32 I;
  I.mu = X->b32[B_MU];
  I.lam = X->b32[B_LAM];
  I.eta = X->b32[B_ETA];
  for (int d = 0; d < 3; ++d) {
    I.dinv[d] = X->b32[B_DINV0 + d];
    I.e[d] = X->b32[B_E0 + d];
    I.r[d] = X->b32[B_R0 + d];
    I.p[0][d] = X->b32[B_P0 + d];
    I.p[1][d] = X->b32[B_PB0 + d];
    I.q[d] = X->b32[B_Q0 + d];
    I.z[d] = X->z32[d];
  }
  I.S = X->scal + 4;
  I.partial = X->partial;
  I.counter = X->counter;
  return I;
}

// TG_MIXED elasticity: iterative refinement with an FP64 residual and FP32 inner PCG.
tg_status elas_solve_mixed(tg_ctx* X, double* const u[3], double* const b_ext[3], bool minus_b,
                           double inv_dt, tg_stats* stats) {
  if (X->df_res && b_ext) {   // the double-FP32 residual reads (hi, lo) pairs of the rhs
    double* const packed[3] = {X->a[A_B0], X->a[A_B1], X->a[A_B2]};
    CK(launch_df_pack3(X->G, b_ext, packed, X->stream));
    X->launches += 1;
    b_ext = nullptr;
  }
  const Elas E = elas_view(X, u, b_ext);
  const Elas32 I = elas32_view(X);
  CgScal* Sout = X->scal + 3;
  const size_t bytes = (size_t)X->G.nvox * sizeof(double);
  if (inv_dt > 0.0) {   // a step's solve: start from u extrapolated in time
    CK(launch_elas_extrapolate(X->G, E, 1.0 / inv_dt, X->hist_ok, X->stream));
    X->launches += 1;
  } else {
    for (int d = 0; d < 3; ++d) CK(cudaMemsetAsync(E.du[d], 0, bytes, X->stream));
  }
  k_cg_reset<<<1, 32, 0, X->stream>>>(Sout, 1, X->prm.rtol_elas, X->prm.maxit_elas);
  CK(cudaGetLastError());
  // with the double-FP32 residual the node coefficients came with the faces, and the
  // extrapolation wrote the pairs of a step's starting u; otherwise u is packed here
  if (!(X->df_res && inv_dt > 0.0)) {
    CK(launch_elas32_coef(X->G, E, I, X->stream,
                          X->df_res ? ELAS32_U : ELAS32_NODES | ELAS32_DINV | ELAS32_U));
    X->launches += 1;
  }
  X->launches += 1;
  const bool spec = spectral_on(X);
  Spec<float> V = X->sp32;   // the scaled preconditioner's view carries s
  if (spec) {
    CK(launch_spec_mean(X->G.nvox, E.mu, E.lam, E.eta, V.mean, V.partial, V.counter,
                        X->stream, true));
    X->launches += 1;
    if (X->prm.precond_elas == TG_PRECOND_SPECTRAL_SCALED) {
      for (int d = 0; d < 3; ++d) V.s[d] = X->s32[d];
      CK(launch_spec_scale(X->G, V, E, X->stream));
      X->launches += 1;
    }
  }
  const float* const r32[3] = {I.r[0], I.r[1], I.r[2]};
  int inner_total = 0, sweeps = 0;
  CgScal out;
  for (;;) {
    CK(launch_elas_ir_residual(X->G, E, I, Sout, minus_b, spec ? TAU_INNER_SPECTRAL : TAU_INNER,
                               X->stream));
    X->launches += 1;
    CK(cudaMemcpyAsync(&out, Sout, sizeof(CgScal), cudaMemcpyDeviceToHost, X->stream));
    CK(cudaStreamSynchronize(X->stream));
    if (out.status != CG_RUNNING) break;
    if (sweeps >= MAX_SWEEPS || inner_total >= X->prm.maxit_elas) return fail(X, TG_ERR_NOCONV);
    CK(launch_elas32_scale_r(X->G, I, X->stream));
    X->launches += 1;
    if (spec) {   // p = P r and <r, P r> for the inner solve's first direction
      PUpd<float> pu;
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 3; ++a) pu.p[b][a] = I.p[b][a];
      CK(launch_spectral(V, r32, X->z32, I.S, X->stream, &pu));
      X->launches += 5;
    }
    CgScal host[1];
    const int slot = sweeps == 0 ? 0 : 1;
    tg_status s = drive_cg(X, [&](int) {
      X->launches += spec ? 6 : 2;
      cudaError_t e = spec ? launch_elas32_matvec_spec(X->G, I, X->stream)
                           : launch_elas32_matvec(X->G, I, X->stream);
      if (e != cudaSuccess) return e;
      if (!spec) return launch_elas32_update(X->G, I, X->stream);
      return launch_spectral_update(V, I, X->z32, X->stream);
    }, I.S, 1, X->prm.maxit_elas, X->prev_it_inner[slot], host);
    if (s != TG_OK) return s;
    X->prev_it_inner[slot] = host[0].it;
    inner_total += host[0].it;
    if (host[0].status == CG_NONFINITE) return fail(X, TG_ERR_NONFINITE);
    CK(launch_elas_ir_correct(X->G, E, I, X->stream));
    X->launches += 1;
    ++sweeps;
  }
  if (stats) {
    stats->it_elas = inner_total;
    stats->it_elas_outer = out.it;
    stats->relres_elas = out.bb > 0.0 ? sqrt(out.rr / out.bb) : 0.0;
    stats->it_elas_total += inner_total;
  }
  if (out.status == CG_NONFINITE) return fail(X, TG_ERR_NONFINITE);
  if (out.status == CG_MAXIT) return fail(X, TG_ERR_NOCONV);
  CK(launch_elas_ir_finish(X->G, E, inv_dt, out.status == CG_ZERO_RHS, X->stream));
  X->launches += 1;
  CK(cudaStreamSynchronize(X->stream));
  return TG_OK;
}

// S6 solve on coefficients already built: (eta I - L_h) u = rhs from the given u.
tg_status elas_solve(tg_ctx* X, double* const u[3], double* const b_ext[3], bool minus_b,
                     double inv_dt, tg_stats* stats) {
  if (X->prec == TG_MIXED) return elas_solve_mixed(X, u, b_ext, minus_b, inv_dt, stats);
  const Elas E = elas_view(X, u, b_ext);
  const bool spec = spectral_on(X);
  k_cg_reset<<<1, 32, 0, X->stream>>>(X->scal + 3, 1, X->prm.rtol_elas, X->prm.maxit_elas);
  CK(cudaGetLastError());
  const double* const r64[3] = {E.r[0], E.r[1], E.r[2]};
  if (inv_dt > 0.0) {   // a step's solve: start from u extrapolated in time
    CK(launch_elas_extrapolate(X->G, E, 1.0 / inv_dt, X->hist_ok, X->stream));
    X->launches += 1;
  }
  Spec<double> V = X->sp64;   // the scaled preconditioner's view carries s
  if (spec) {
    CK(launch_spec_mean(X->G.nvox, E.mu, E.lam, E.eta, V.mean, V.partial, V.counter,
                        X->stream, false));
    if (X->prm.precond_elas == TG_PRECOND_SPECTRAL_SCALED) {
      for (int d = 0; d < 3; ++d) V.s[d] = X->s64[d];
      CK(launch_spec_scale(X->G, V, E, X->stream));
      X->launches += 1;
    }
    CK(launch_elas_init_spec(X->G, E, minus_b, X->stream));
    CK(launch_spectral(V, r64, X->z64, E.S, X->stream));
    CK(launch_elas_pupdate_spec(X->G, E, X->stream));
    X->launches += 9;
  } else {
    CK(launch_elas_init(X->G, E, minus_b, X->stream));
    X->launches += 2;
  }
  CgScal host[1];
  tg_status s = drive_cg(X, [&](int) {
    X->launches += spec ? 8 : 3;
    cudaError_t e = launch_elas_matvec(X->G, E, X->stream);
    if (e != cudaSuccess) return e;
    if (!spec) return launch_elas_update(X->G, E, X->stream);
    e = launch_elas_update_spec(X->G, E, X->stream);
    if (e == cudaSuccess) e = launch_spectral(V, r64, X->z64, E.S, X->stream);
    if (e == cudaSuccess) e = launch_elas_pupdate_spec(X->G, E, X->stream);
    return e;
  }, E.S, 1, X->prm.maxit_elas, X->prev_it_elas, host);
  if (s != TG_OK) return s;
  X->prev_it_elas = host[0].it;
  if (stats) {
    stats->it_elas = host[0].it;
    stats->it_elas_outer = 1;
    stats->relres_elas = host[0].bb > 0.0 ? sqrt(host[0].rr / host[0].bb) : 0.0;
    stats->it_elas_total += host[0].it;
  }
  tg_status e = status_of(host[0]);
  if (e != TG_OK) return fail(X, e);
  CK(launch_elas_finish(X->G, E, inv_dt, host[0].status == CG_ZERO_RHS,
                        inv_dt > 0.0 ? (X->hist_ok ? 2 : 1) : 0,
                        X->stream));
  X->launches += 1;
  CK(cudaStreamSynchronize(X->stream));
  return TG_OK;
}

tg_status build_elas_coef(tg_ctx* X, bool force) {
  const tg_state& S = X->st;
  double* const u[3] = {S.u[0], S.u[1], S.u[2]};
  const Elas E = elas_view(X, u, nullptr);
  if (X->df_res) {   // node values and pairs (and s = p + n) first, then faces and force
    const Elas32 I = elas32_view(X);
    float2* const sdf = reinterpret_cast<float2*>(X->a[A_DIV]);   // free in the mixed step
    CK(launch_lame_df(X->G, X->dp, S.p, S.i, S.n, S.g, S.w, S.f, S.bg, X->a[A_MU], X->a[A_LAM],
                      X->a[A_ETA], I.mu, I.lam, I.eta, E.mudf, E.lamdf, sdf, X->stream));
    CK(launch_elas_coef_df(X->G, X->dp, E, I, sdf, force, X->stream));
    X->launches += 2;
    return TG_OK;
  }
  CK(launch_lame(X->G, X->dp, S.p, S.i, S.n, S.g, S.w, S.f, S.bg, X->a[A_MU], X->a[A_LAM],
                 X->a[A_ETA], X->stream));
  CK(launch_elas_coef(X->G, X->dp, E, S.p, S.n, force, X->stream));
  X->launches += 2;
  return TG_OK;
}

void reset_profile(tg_ctx* X) {
  X->launches = 0;
  for (int k = 0; k < K_COUNT; ++k) {
    X->prof.call_ms[k] = 0.0;
    X->prof.call_n[k] = 0;
  }
  for (int q = 0; q < 4; ++q) X->t_phase[q] = 0.0;
}

void fill_profile(tg_ctx* X, tg_stats* stats) {
  const Prof& P = X->prof;
  stats->launches = X->launches;
  stats->t_elas_matvec_ms =
      P.call_ms[K_ELAS_MATVEC] + P.call_ms[K_ELAS32_MATVEC] + P.call_ms[K_ELAS32_MATVEC_SPEC];
  stats->n_elas_matvec =
      P.call_n[K_ELAS_MATVEC] + P.call_n[K_ELAS32_MATVEC] + P.call_n[K_ELAS32_MATVEC_SPEC];
  stats->t_spec_update_ms = P.call_ms[K_SPEC_UPDATE_XFWD];
  stats->n_spec_update = P.call_n[K_SPEC_UPDATE_XFWD];
  for (int q = 0; q < 4; ++q) stats->t_phase_ms[q] = X->t_phase[q];
}

// phase boundary q (0..4) of a step, with timing on
void phase_mark(tg_ctx* X, int q) {
  if (!X->timing) return;
  if (!X->pev_ok) {
    for (int e = 0; e < 5; ++e) {
      if (cudaEventCreate(&X->pev[e]) != cudaSuccess) {
        while (e-- > 0) cudaEventDestroy(X->pev[e]);
        return;
      }
    }
    X->pev_ok = true;
  }
  cudaEventRecord(X->pev[q], X->stream);
}

// after a step with timing on (the stream has been synchronised): add the phase durations
void phase_harvest(tg_ctx* X) {
  if (!X->timing || !X->pev_ok) return;
  if (cudaEventSynchronize(X->pev[4]) != cudaSuccess) return;
  for (int q = 0; q < 4; ++q) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, X->pev[q], X->pev[q + 1]) == cudaSuccess) X->t_phase[q] += ms;
  }
}

// One step of the Section 3 split.
tg_status record(tg_ctx* X, int slot, const double* src) {
  if (X->tape[0] == nullptr) return TG_OK;
  CK(cudaMemcpyAsync(X->tape[slot], src, (size_t)X->G.nvox * sizeof(double),
                     cudaMemcpyDeviceToDevice, X->stream));
  return TG_OK;
}

#define REC(slot, src)                          \
  do {                                          \
    tg_status e_ = record(X, (slot), (src));    \
    if (e_ != TG_OK) return e_;                 \
  } while (0)

tg_status do_step(tg_ctx* X, double dt, tg_stats* stats) {
  const Geo& G = X->G;
  tg_state& S = X->st;
  cudaStream_t s = X->stream;
  const size_t bytes = (size_t)G.nvox * sizeof(double);
  {
    const double* start[14] = {S.p, S.i, S.n, S.g, S.w, S.f, S.o, S.l,
                               S.u[0], S.u[1], S.u[2], S.v[0], S.v[1], S.v[2]};
    for (int q = 0; q < 14; ++q) REC(T_P + q, start[q]);
  }
  // S0: K faces, CN diagonal and rho from the step's start
  if (X->host_in) CK(cudaStreamWaitEvent(s, X->up_ev[0], 0));   // g, w, f are up
  phase_mark(X, 0);
  double* const Kf[3] = {X->a[A_KF0], X->a[A_KF1], X->a[A_KF2]};
  double* const Kfdf[3] = {X->a[A_KFDF0], X->a[A_KFDF1], X->a[A_KFDF2]};
  if (X->prec == TG_MIXED && X->cn_df) {
    // the mixed solves read the faces as pairs and as FP32 values only (the oxygen solve in
    // double-FP32, tg_cn_ox.cu): formed in double-FP32, node K pairs in the FP64 transport
    // scratch (the mixed transport writes the state directly)
    float2* const pairs[3] = {reinterpret_cast<float2*>(Kfdf[0]), reinterpret_cast<float2*>(Kfdf[1]),
                              reinterpret_cast<float2*>(Kfdf[2])};
    float* const f32[3] = {X->b32[B_CKF0], X->b32[B_CKF1], X->b32[B_CKF2]};
    CK(cudaMemsetAsync(X->dmax, 0, sizeof(float), s));
    CK(launch_diff_coef_df(G, X->dp, dt, S.g, S.w, S.f, reinterpret_cast<float2*>(X->a[A_SL0]),
                           X->a[A_RHO], pairs, f32, X->b32[B_CDINV], X->dmax, s));
    X->launches += 2;
  } else {
    CK(launch_diff_coef(G, X->dp, dt, S.g, S.w, S.f, Kf, X->a[A_DSUM_D], X->a[A_DINV_D],
                        X->a[A_RHO], s, X->cn_df ? Kfdf : nullptr));
    X->launches += 1;   // S0 is two kernels (faces, diagonal)
  }
  if (X->prec == TG_MIXED && !X->cn_df) {   // FP32 faces and diagonal of the inner solves
    F32Copy cp;
    const double* src[4] = {Kf[0], Kf[1], Kf[2], X->a[A_DINV_D]};
    for (int q = 0; q < 4; ++q) {
      cp.src[q] = src[q];
      cp.dst[q] = X->b32[B_CKF0 + q];
    }
    cp.count = 4;
    CK(launch_to_f32(G.nvox, cp, s));
    X->launches += 1;
  }
  // the mixed oxygen solve needs only the faces and o: it starts now, beside S1 and S2
  OxGuard ox_guard{X};
  const bool ox_side = X->prec == TG_MIXED && !single_species(X);
  if (ox_side) {
    const tg_status e0 = ox_begin(X);
    if (e0 != TG_OK) return e0;
  }
  // S1: semi-Lagrangian transport with v^n
  if (X->host_in) CK(cudaStreamWaitEvent(s, X->up_ev[1], 0));   // v, p, i, n are up
  const double* const v[3] = {S.v[0], S.v[1], S.v[2]};
  const double* const qin[6] = {S.p, S.i, S.n, S.g, S.w, S.f};
  if (X->prec == TG_MIXED) {
    // interleaved FP32 copies of everything the interpolation gathers, then FP32 transport
    // into the state
    const Sl32 T = sl32_view(X);
    CK(launch_sl32_pack(G, v, qin, T, s));
    CK(launch_sl32(G, dt, T, s));
    X->launches += 2;
  } else {
    CK(launch_divergence(G, v, X->a[A_DIV], s));
    double* const qout[6] = {X->a[A_SL0], X->a[A_SL1], X->a[A_SL2],
                             X->a[A_SL3], X->a[A_SL4], X->a[A_SL5]};
    CK(launch_sl_advect(G, dt, v, X->a[A_DIV], qin, qout, s));
    X->launches += 3;
    double* const dst[6] = {S.p, S.i, S.n, S.g, S.w, S.f};
    for (int q = 0; q < 6; ++q)
      CK(cudaMemcpyAsync(dst[q], qout[q], bytes, cudaMemcpyDeviceToDevice, s));
  }
  {
    const double* sl[6] = {S.p, S.i, S.n, S.g, S.w, S.f};
    for (int q = 0; q < 6; ++q) REC(T_PD + q, sl[q]);
  }
  // S2: Crank-Nicolson diffusion of i, o, l (i after transport kept for the g, w fix-up);
  // single species: of c alone
  if (X->host_in) CK(cudaStreamWaitEvent(s, X->up_ev[2], 0));   // o, l are up
  phase_mark(X, 1);
  const bool single = single_species(X);
  CK(cudaMemcpyAsync(X->a[A_IDAG], single ? S.p : S.i, bytes, cudaMemcpyDeviceToDevice, s));
  tg_status e = TG_OK;
  if (single) {
    e = X->prec == TG_MIXED ? cn_solve3_mixed(X, stats, 1) : cn_solve3(X, stats, 1);
  } else if (X->prec == TG_MIXED) {
    e = cn_solve3_mixed(X, stats, CN_MIXED_MASK);   // i and l; the oxygen runs on the side
    if (e == TG_OK) e = ox_end(X, stats);
  } else {
    e = cn_solve3(X, stats);
  }
  if (e != TG_OK) return e;
  REC(T_IDD, S.i);
  REC(T_OD, S.o);
  REC(T_LD, S.l);
  // S2 fix-up and S3-S5 reactions
  phase_mark(X, 2);
  CK(launch_react(G, X->dp, dt, X->a[A_RHO], X->a[A_IDAG], S.p, S.i, S.n, S.g, S.w, S.o, S.l,
                  X->prec == TG_MIXED, single_species(X), s));
  X->launches += 1;
  if (X->host_out) {   // nothing after S5 changes the species: down during S6-S7
    CK(cudaEventRecord(X->s5_ev, s));
    CK(cudaStreamWaitEvent(X->copy, X->s5_ev, 0));
    double* const dst[9] = {X->host_out->p, X->host_out->i, X->host_out->n, X->host_out->g,
                            X->host_out->w, X->host_out->f, X->host_out->o, X->host_out->l,
                            X->host_out->bg};
    const double* const src[9] = {S.p, S.i, S.n, S.g, S.w, S.f, S.o, S.l, S.bg};
    for (int q = 0; q < 9; ++q)
      CK(cudaMemcpyAsync(dst[q], src[q], bytes, cudaMemcpyDeviceToHost, X->copy));
  }
  if (X->host_in) CK(cudaStreamWaitEvent(s, X->up_ev[3], 0));   // bg and u are up
  // S6-S7: elasticity from the post-reaction state, then v = du / dt
  phase_mark(X, 3);
  e = build_elas_coef(X, true);
  if (e != TG_OK) return e;
  e = elas_solve(X, S.u, nullptr, true, 1.0 / dt, stats);
  if (e != TG_OK) return e;
  X->hist_ok = true;   // the finish kept v^n: the next step may extrapolate quadratically
  phase_mark(X, 4);
  for (int d = 0; d < 3; ++d) REC(T_UP0 + d, S.u[d]);
  phase_harvest(X);
  return TG_OK;
}

AdjView adj_view(tg_ctx* X, const tg_state* lam) {
  AdjView A;
  A.lam.p = lam->p;
  A.lam.i = lam->i;
  A.lam.n = lam->n;
  A.lam.g = lam->g;
  A.lam.w = lam->w;
  A.lam.f = lam->f;
  A.lam.o = lam->o;
  A.lam.l = lam->l;
  for (int d = 0; d < 3; ++d) {
    A.lam.u[d] = lam->u[d];
    A.lam.v[d] = lam->v[d];
    A.rhs[d] = X->adj[C_RHS0 + d];
    A.psi[d] = X->adj[C_PSI0 + d];
    A.up[d] = nullptr;
    A.LCN[d] = X->adj[C_LCN0 + d];
    A.phi[d] = X->adj[C_PHI0 + d];
    A.LV[d] = X->adj[C_LV0 + d];
  }
  for (int q = 0; q < 7; ++q) A.LQ[q] = X->adj[C_LQ0 + q];
  for (int q = 0; q < 5; ++q) A.LD[q] = X->adj[C_LD0 + q];
  A.LF = X->adj[C_LF];
  A.LRHO = X->adj[C_LRHO];
  A.LDEL = X->adj[C_LDEL];
  A.grad = X->grad;
  A.partial = X->partial;
  A.counter = X->counter;
  return A;
}

TapeView tape_view(tg_ctx* X, const void* tape) {
  const char* base = (const char*)tape;
  const size_t stride = round_up((size_t)X->G.nvox * sizeof(double));
  auto at = [&](int q) { return (const double*)(base + (size_t)q * stride); };
  TapeView T;
  T.p = at(T_P);
  T.i = at(T_I);
  T.n = at(T_N);
  T.g = at(T_G);
  T.w = at(T_W);
  T.f = at(T_F);
  T.o = at(T_O);
  T.l = at(T_L);
  for (int d = 0; d < 3; ++d) {
    T.u[d] = at(T_U0 + d);
    T.v[d] = at(T_V0 + d);
    T.up[d] = at(T_UP0 + d);
  }
  T.pdag = at(T_PD);
  T.idag = at(T_ID);
  T.ndag = at(T_ND);
  T.gdag = at(T_GD);
  T.wdag = at(T_WD);
  T.fplus = at(T_FP);
  T.iddag = at(T_IDD);
  T.odag = at(T_OD);
  T.ldag = at(T_LD);
  return T;
}

tg_status read_grad(tg_ctx* X, double grad[5]) {
  double g[5];
  CK(cudaMemcpyAsync(g, X->grad, sizeof(g), cudaMemcpyDeviceToHost, X->stream));
  CK(cudaStreamSynchronize(X->stream));
  for (int k = 0; k < 5; ++k) grad[k] += g[k];
  return TG_OK;
}

// Adjoint of one step (see tg_adjoint.cu for the order and the formulas).
tg_status do_adjoint_step(tg_ctx* X, double dt, const void* tape, const tg_state* lam,
                          double grad[5]) {
  const Geo& G = X->G;
  cudaStream_t s = X->stream;
  const size_t bytes = (size_t)G.nvox * sizeof(double);
  AdjView A = adj_view(X, lam);
  const TapeView T = tape_view(X, tape);
  for (int d = 0; d < 3; ++d) A.up[d] = T.up[d];
  CK(cudaMemsetAsync(X->grad, 0, 5 * sizeof(double), s));
  // S7^T and copies of the incoming lambdas
  CK(launch_adj_prep(G, A, 1.0 / dt, s));
  // recompute the reacted species q+ from the tape (S0 faces and rho come along)
  double* qp[7];
  for (int q = 0; q < 7; ++q) qp[q] = X->adj[C_QP0 + q];
  const double* src[7] = {T.pdag, T.iddag, T.ndag, T.gdag, T.wdag, T.odag, T.ldag};
  for (int q = 0; q < 7; ++q) CK(cudaMemcpyAsync(qp[q], src[q], bytes, cudaMemcpyDeviceToDevice, s));
  double* const Kf[3] = {X->a[A_KF0], X->a[A_KF1], X->a[A_KF2]};
  CK(launch_diff_coef(G, X->dp, dt, T.g, T.w, T.f, Kf, X->a[A_DSUM_D], X->a[A_DINV_D],
                      X->a[A_RHO], s));
  CK(launch_react(G, X->dp, dt, X->a[A_RHO], T.idag, qp[0], qp[1], qp[2], qp[3], qp[4], qp[5],
                  qp[6], X->prec == TG_MIXED, false, s));
  // S6^T: coefficients at q+, adjoint solve, sensitivities
  CK(launch_lame(G, X->dp, qp[0], qp[1], qp[2], qp[3], qp[4], T.fplus, X->st.bg, X->a[A_MU],
                 X->a[A_LAM], X->a[A_ETA], s));
  {
    double* const psi[3] = {A.psi[0], A.psi[1], A.psi[2]};
    const Elas E = elas_view(X, psi, nullptr);
    CK(launch_elas_coef(G, X->dp, E, qp[0], qp[2], false, s));
  }
  X->launches += 7;
  // the previous step's adjoint solution is the starting guess (the solve is differentiated
  // as an exact inverse, so the guess only changes the iteration count)
  if (!X->psi_valid)
    for (int d = 0; d < 3; ++d) CK(cudaMemsetAsync(A.psi[d], 0, bytes, s));
  {
    double* const psi[3] = {A.psi[0], A.psi[1], A.psi[2]};
    double* const rhs[3] = {A.rhs[0], A.rhs[1], A.rhs[2]};
    X->psi_valid = false;
    tg_status e = elas_solve_mixed(X, psi, rhs, false, 0.0, nullptr);
    if (e != TG_OK) return e;
    X->psi_valid = true;
  }
  const double invE = X->prm.E_scale != 0.0 ? 1.0 / X->prm.E_scale : 0.0;
  CK(launch_adj_elas_coef(G, X->dp, A, X->a[A_MU], X->a[A_LAM], qp[0], qp[2], invE, true, s));
  // S5^T, S4^T, S3^T and the fix-up
  CK(launch_adj_react(G, X->dp, dt, A, T, X->a[A_RHO], s));
  X->launches += 2;
  // S2^T: three adjoint Crank-Nicolson solves on the step-start faces
  {
    Cn3 C = cn_view(X);
    for (int r = 0; r < 3; ++r) C.x[r] = A.phi[r];
    k_cg_reset<<<1, 32, 0, s>>>(X->scal, 3, X->prm.rtol_diff, X->prm.maxit_diff);
    CK(cudaGetLastError());
    CK(launch_cn_init_rhs(G, C, A, s));
    X->launches += 2;
    CgScal host[3];
    tg_status e = drive_cg(X, [&](int) {
      X->launches += 3;
      return launch_cn_iter(G, C, s);
    }, X->scal, 3, X->prm.maxit_diff, X->prev_it_diff, host);
    if (e != TG_OK) return e;
    for (int r = 0; r < 3; ++r) {
      tg_status e2 = status_of(host[r]);
      if (e2 != TG_OK) return fail(X, e2);
    }
  }
  CK(launch_adj_cn_post(G, X->dp, dt, A, T, s));
  // S1^T: transport transpose (scatter), then div_h^T
  CK(cudaMemsetAsync(A.LDEL, 0, bytes, s));
  for (int d = 0; d < 3; ++d) CK(cudaMemsetAsync(A.LV[d], 0, bytes, s));
  const double* const v[3] = {T.v[0], T.v[1], T.v[2]};
  CK(launch_divergence(G, v, X->a[A_DIV], s));
  CK(launch_adj_sl(G, dt, A, T, X->a[A_DIV], s));
  CK(launch_adj_div(G, A, s));
  X->launches += 4;
  return read_grad(X, grad);
}

// Views of the spectral buffers and their one-time tables (twiddles, symbol factors).
tg_status spectral_setup(tg_ctx* X) {
  const Layout& L = X->L;
  for (int d = 0; d < 3; ++d) {
    X->z32[d] = nullptr;
    X->z64[d] = nullptr;
    X->s32[d] = nullptr;
    X->s64[d] = nullptr;
  }
  if (!L.spectral) return TG_OK;
  const bool need32 = X->prec == TG_MIXED || X->has_adjoint;
  const bool need64 = X->prec == TG_FP64;
  if (cudaMemsetAsync(X->ws + L.sp_counter, 0, ALIGN, X->stream) != cudaSuccess) return TG_ERR_CUDA;
  if (need32) {
    X->sp32 = spec_view<float>(X->G, L, X->ws, L.sp_tab32);
    for (int d = 0; d < 3; ++d) {
      X->z32[d] = (float*)(X->ws + L.sp_z32[d]);
      X->s32[d] = (float*)(X->ws + L.sp_s32[d]);
    }
    if (spec_prepare(X->sp32) != cudaSuccess) return TG_ERR_CUDA;
    if (launch_spec_tables(X->sp32, X->G.h, X->stream) != cudaSuccess) return TG_ERR_CUDA;
    X->sp32.zmap = spec_make_zmap(X->sp32, X->zmap32) ? X->zmap32 : nullptr;
  }
  if (need64) {
    X->sp64 = spec_view<double>(X->G, L, X->ws, L.sp_tab64);
    for (int d = 0; d < 3; ++d) {
      X->z64[d] = (double*)(X->ws + L.sp_z64[d]);
      X->s64[d] = (double*)(X->ws + L.sp_s64[d]);
    }
    if (spec_prepare(X->sp64) != cudaSuccess) return TG_ERR_CUDA;
    if (launch_spec_tables(X->sp64, X->G.h, X->stream) != cudaSuccess) return TG_ERR_CUDA;
  }
  return TG_OK;
}

}  // namespace

extern "C" {

size_t tg_workspace_bytes(const tg_grid* grid, const tg_params* params, tg_precision prec) {
  if (!grid_ok(grid) || (prec != TG_FP64 && prec != TG_MIXED)) return 0;
  if (params && !params_ok(params)) return 0;
  const Geo G = make_geo(grid, sm_count());
  const bool spectral = params && spectral_precond(params->precond_elas);
  if (spectral && !spectral_grid_ok(G)) return 0;
  return layout(G, prec, false, spectral).total;
}

size_t tg_workspace_bytes_adjoint(const tg_grid* grid, const tg_params* params,
                                  tg_precision prec) {
  if (!grid_ok(grid) || (prec != TG_FP64 && prec != TG_MIXED)) return 0;
  if (params && !params_ok(params)) return 0;
  const Geo G = make_geo(grid, sm_count());
  const bool spectral = params && spectral_precond(params->precond_elas);
  if (spectral && !spectral_grid_ok(G)) return 0;
  return layout(G, prec, true, spectral).total;
}

size_t tg_tape_bytes(const tg_grid* grid) {
  if (!grid_ok(grid)) return 0;
  const size_t v = (size_t)grid->n[0] * grid->n[1] * grid->n[2];
  return (size_t)T_COUNT * round_up(v * sizeof(double));
}

tg_status tg_init(const tg_grid* grid, const tg_params* params, tg_precision prec,
                  const tg_state* state, void* workspace, size_t workspace_bytes,
                  void* cuda_stream, uint32_t flags, tg_ctx** out, tg_stats* stats) {
  if (out) *out = nullptr;
  if (!out || !grid_ok(grid) || !params_ok(params) || !state) return TG_ERR_ARG;
  if (prec != TG_FP64 && prec != TG_MIXED) return TG_ERR_ARG;
  // the adjoint differentiates the multispecies step only
  if ((flags & TG_INIT_ADJOINT) && params->model != TG_MODEL_MULTISPECIES) return TG_ERR_ARG;
  const double* must[] = {state->p, state->i, state->n, state->g, state->w, state->f, state->o,
                          state->l, state->bg, state->u[0], state->u[1], state->u[2],
                          state->v[0], state->v[1], state->v[2]};
  for (const double* q : must)
    if (!q || ((uintptr_t)q & 15u)) return TG_ERR_ARG;
  const Geo G = make_geo(grid, sm_count());
  const bool adjoint = (flags & TG_INIT_ADJOINT) != 0;
  const bool spectral = spectral_precond(params->precond_elas);
  if (spectral && !spectral_grid_ok(G)) return TG_ERR_ARG;
  const Layout L = layout(G, prec, adjoint, spectral);
  if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 || workspace_bytes < L.total)
    return TG_ERR_WORKSPACE;
  tg_ctx* X = new (std::nothrow) tg_ctx();
  if (!X) return TG_ERR_CUDA;
  X->G = G;
  X->L = L;
  X->prm = *params;
  X->dp = make_dev_params(params);
  X->prec = prec;
  X->st = *state;
  X->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&X->device);
  X->ws = (char*)workspace;
  for (int a = 0; a < A_COUNT; ++a) X->a[a] = (double*)(X->ws + L.arr[a]);
  for (int b = 0; b < B_COUNT; ++b)
    X->b32[b] = (prec == TG_MIXED || adjoint) ? (float*)(X->ws + L.arr32[b]) : nullptr;
  X->has_adjoint = adjoint;
  X->df_res = df_residual_ok(X);
  X->cn_df = cn_df_ok(X);
  for (int c = 0; c < C_COUNT; ++c) X->adj[c] = adjoint ? (double*)(X->ws + L.adj[c]) : nullptr;
  X->grad = (double*)(X->ws + L.grad);
  X->partial = (double*)(X->ws + L.partial);
  X->counter = (unsigned int*)(X->ws + L.counter);
  X->scal = (CgScal*)(X->ws + L.scal);
  X->partial2 = (double*)(X->ws + L.partial2);
  X->counter2 = (unsigned int*)(X->ws + L.counter2);
  X->dmax = (float*)(X->ws + L.dmax);
  if (cudaMemsetAsync(X->counter, 0, ALIGN, X->stream) != cudaSuccess ||
      (prec == TG_MIXED && cudaMemsetAsync(X->counter2, 0, ALIGN, X->stream) != cudaSuccess)) {
    tg_free(X);
    return TG_ERR_CUDA;
  }
  if (spectral_setup(X) != TG_OK) {
    tg_free(X);
    return TG_ERR_CUDA;
  }
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!(flags & TG_INIT_KEEP_UV)) {
    const size_t bytes = (size_t)G.nvox * sizeof(double);
    tg_status e = TG_OK;
    for (int d = 0; d < 3 && e == TG_OK; ++d) {
      if (cudaMemsetAsync(X->st.u[d], 0, bytes, X->stream) != cudaSuccess ||
          cudaMemsetAsync(X->st.v[d], 0, bytes, X->stream) != cudaSuccess)
        e = TG_ERR_CUDA;
    }
    if (e == TG_OK) e = build_elas_coef(X, true);
    if (e == TG_OK) e = elas_solve(X, X->st.u, nullptr, true, 0.0, stats);
    if (e != TG_OK) {
      tg_free(X);
      return e;
    }
  }
  if (cudaStreamSynchronize(X->stream) != cudaSuccess) {
    tg_free(X);
    return TG_ERR_CUDA;
  }
  if (stats) fill_profile(X, stats);
  *out = X;
  return TG_OK;
}

// One step with the state in host memory, the copies overlapped with the step (tg.h).
tg_status tg_step_host(tg_ctx* X, const tg_state* in, tg_state* out, double dt,
                       tg_stats* stats) {
  if (!X || !in || !out) return TG_ERR_ARG;
  if (X->broken) return TG_ERR_STATE;
  if (!(dt > 0.0) || !isfinite(dt)) return TG_ERR_ARG;
  CK(cudaSetDevice(X->device));
  if (!X->copy) {
    CK(cudaStreamCreateWithFlags(&X->copy, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&X->entry_ev, cudaEventDisableTiming));
    for (int g = 0; g < 4; ++g) CK(cudaEventCreateWithFlags(&X->up_ev[g], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&X->s5_ev, cudaEventDisableTiming));
  }
  tg_state& S = X->st;
  cudaStream_t s = X->stream;
  const size_t bytes = (size_t)X->G.nvox * sizeof(double);
  // up on the copy stream, after everything already queued on the context's stream, in the
  // order the split reads the fields: S0 (g, w, f), S1 (v, p, i, n), S2 (o, l), S6 (bg, u);
  // the step waits for each group where it first reads it
  CK(cudaEventRecord(X->entry_ev, s));
  CK(cudaStreamWaitEvent(X->copy, X->entry_ev, 0));
  const double* const src[15] = {in->g, in->w, in->f, in->v[0], in->v[1], in->v[2], in->p,
                                 in->i, in->n, in->o, in->l, in->bg, in->u[0], in->u[1],
                                 in->u[2]};
  double* const dst[15] = {S.g, S.w, S.f, S.v[0], S.v[1], S.v[2], S.p, S.i, S.n, S.o, S.l,
                           S.bg, S.u[0], S.u[1], S.u[2]};
  const int group_end[4] = {3, 9, 11, 15};
  for (int g = 0, q = 0; g < 4; ++g) {
    for (; q < group_end[g]; ++q)
      CK(cudaMemcpyAsync(dst[q], src[q], bytes, cudaMemcpyHostToDevice, X->copy));
    CK(cudaEventRecord(X->up_ev[g], X->copy));
  }
  X->host_in = in;
  X->host_out = out;
  tg_status e = tg_step(X, dt, 1, nullptr, stats);
  X->host_in = nullptr;
  X->host_out = nullptr;
  if (e != TG_OK) {
    cudaStreamSynchronize(X->copy);
    return e;
  }
  for (int a = 0; a < 3; ++a) {
    CK(cudaMemcpyAsync(out->u[a], S.u[a], bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->v[a], S.v[a], bytes, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(X->copy));
  CK(cudaStreamSynchronize(s));
  return TG_OK;
}

tg_status tg_step(tg_ctx* X, double dt, int32_t nsteps, void* tape, tg_stats* stats) {
  if (!X) return TG_ERR_ARG;
  if (X->broken) return TG_ERR_STATE;
  if (!(dt > 0.0) || !isfinite(dt) || nsteps < 0) return TG_ERR_ARG;
  if (tape && (nsteps != 1 || ((uintptr_t)tape % ALIGN) != 0)) return TG_ERR_ARG;
  if (tape && single_species(X)) return TG_ERR_ARG;
  if (stats) memset(stats, 0, sizeof(*stats));
  reset_profile(X);
  CK(cudaSetDevice(X->device));
  HookScope hook(X);
  const size_t stride = round_up((size_t)X->G.nvox * sizeof(double));
  for (int q = 0; q < T_COUNT; ++q)
    X->tape[q] = tape ? (double*)((char*)tape + (size_t)q * stride) : nullptr;
  for (int32_t s = 0; s < nsteps; ++s) {
    tg_status e = do_step(X, dt, stats);
    if (e != TG_OK) {
      X->tape[0] = nullptr;
      return fail(X, e);
    }
    if (X->timing) prof_harvest(X);
    if (stats) stats->steps += 1;
  }
  X->tape[0] = nullptr;
  CK(cudaStreamSynchronize(X->stream));
  if (stats) fill_profile(X, stats);
  return TG_OK;
}

tg_status tg_solve_elasticity(tg_ctx* X, double* const rhs[3], double* u[3], tg_stats* stats) {
  if (!X || !u || !u[0] || !u[1] || !u[2]) return TG_ERR_ARG;
  if (rhs && (!rhs[0] || !rhs[1] || !rhs[2])) return TG_ERR_ARG;
  if (X->broken) return TG_ERR_STATE;
  if (stats) memset(stats, 0, sizeof(*stats));
  reset_profile(X);
  CK(cudaSetDevice(X->device));
  HookScope hook(X);
  tg_status e = build_elas_coef(X, rhs == nullptr);
  if (e != TG_OK) return fail(X, e);
  double* const uu[3] = {u[0], u[1], u[2]};
  e = elas_solve(X, uu, rhs, rhs == nullptr, 0.0, stats);
  if (e == TG_OK && X->timing) prof_harvest(X);
  if (e == TG_OK && stats) fill_profile(X, stats);
  return e;
}

tg_status tg_adjoint_step(tg_ctx* X, double dt, const void* tape, tg_state* lam, double grad[5]) {
  if (!X || !tape || !lam || !grad) return TG_ERR_ARG;
  if (X->broken) return TG_ERR_STATE;
  if (!X->has_adjoint) return TG_ERR_WORKSPACE;
  if (!(dt > 0.0) || !isfinite(dt) || ((uintptr_t)tape % ALIGN) != 0) return TG_ERR_ARG;
  const double* must[] = {lam->p, lam->i, lam->n, lam->g, lam->w, lam->f, lam->o, lam->l,
                          lam->u[0], lam->u[1], lam->u[2], lam->v[0], lam->v[1], lam->v[2]};
  for (const double* q : must)
    if (!q) return TG_ERR_ARG;
  reset_profile(X);
  CK(cudaSetDevice(X->device));
  tg_status e = do_adjoint_step(X, dt, tape, lam, grad);
  return e == TG_OK ? TG_OK : fail(X, e);
}

tg_status tg_adjoint_init(tg_ctx* X, double* const lam_u[3], double grad[5]) {
  if (!X || !lam_u || !lam_u[0] || !lam_u[1] || !lam_u[2] || !grad) return TG_ERR_ARG;
  if (X->broken) return TG_ERR_STATE;
  if (!X->has_adjoint) return TG_ERR_WORKSPACE;
  CK(cudaSetDevice(X->device));
  const Geo& G = X->G;
  cudaStream_t s = X->stream;
  tg_state dummy = X->st;
  AdjView A = adj_view(X, &dummy);
  for (int d = 0; d < 3; ++d) A.up[d] = X->st.u[d];
  CK(cudaMemsetAsync(X->grad, 0, 5 * sizeof(double), s));
  tg_status e = build_elas_coef(X, false);
  if (e != TG_OK) return fail(X, e);
  const size_t bytes = (size_t)G.nvox * sizeof(double);
  if (!X->psi_valid)
    for (int d = 0; d < 3; ++d) CK(cudaMemsetAsync(A.psi[d], 0, bytes, s));
  double* const psi[3] = {A.psi[0], A.psi[1], A.psi[2]};
  X->psi_valid = false;
  e = elas_solve_mixed(X, psi, lam_u, false, 0.0, nullptr);
  if (e != TG_OK) return fail(X, e);
  X->psi_valid = true;
  const double invE = X->prm.E_scale != 0.0 ? 1.0 / X->prm.E_scale : 0.0;
  CK(launch_adj_elas_coef(G, X->dp, A, X->a[A_MU], X->a[A_LAM], X->st.p, X->st.n, invE, false, s));
  e = read_grad(X, grad);
  return e == TG_OK ? TG_OK : fail(X, e);
}

tg_status tg_set_params(tg_ctx* X, const tg_params* params) {
  if (!X || !params_ok(params)) return TG_ERR_ARG;
  if (X->broken) return TG_ERR_STATE;
  if (spectral_precond(params->precond_elas) && !X->L.spectral) return TG_ERR_WORKSPACE;
  if (X->has_adjoint && params->model != TG_MODEL_MULTISPECIES) return TG_ERR_ARG;
  X->prm = *params;
  X->df_res = df_residual_ok(X);
  X->cn_df = cn_df_ok(X);
  X->dp = make_dev_params(params);
  X->hist_ok = false;
  return TG_OK;
}

tg_status tg_reset_history(tg_ctx* X) {
  if (!X) return TG_ERR_ARG;
  X->hist_ok = false;
  return TG_OK;
}

tg_status tg_diagnostics(tg_ctx* X, const double seed[3], double u_threshold,
                         double* const fields[3], tg_diag* out) {
  if (!X || !seed || !out || !(u_threshold >= 0.0)) return TG_ERR_ARG;
  if (X->broken) return TG_ERR_STATE;
  CK(cudaSetDevice(X->device));
  const Geo& G = X->G;
  tg_state& S = X->st;
  CK(launch_lame(G, X->dp, S.p, S.i, S.n, S.g, S.w, S.f, S.bg, X->a[A_MU], X->a[A_LAM],
                 X->a[A_ETA], X->stream));
  DiagArgs A;
  for (int d = 0; d < 3; ++d) {
    A.u[d] = S.u[d];
    A.out[d] = fields ? fields[d] : nullptr;
    A.seed[d] = seed[d];
    A.L[d] = G.h[d] * (d == 0 ? G.nx : (d == 1 ? G.ny : G.nz));
  }
  A.mu = X->a[A_MU];
  A.lam = X->a[A_LAM];
  A.threshold = u_threshold;
  A.partial = X->partial;
  A.counter = X->counter;
  A.result = X->grad + 8;   // 7 spare doubles of the reduction area, after the gradient's 5
  CK(launch_diagnostics(G, A, X->stream));
  X->launches += 2;
  double r[7];
  CK(cudaMemcpyAsync(r, A.result, sizeof(r), cudaMemcpyDeviceToHost, X->stream));
  CK(cudaStreamSynchronize(X->stream));
  out->jac_min = r[0];
  out->jac_max = r[1];
  out->jac_dev_l2 = r[2];
  out->trace_min = r[3];
  out->trace_max = r[4];
  out->shear_max = r[5];
  out->d_max = r[6];
  return TG_OK;
}

tg_status tg_set_timing(tg_ctx* X, int32_t enable) {
  if (!X) return TG_ERR_ARG;
  if (enable && !X->timing) {
    for (int k = 0; k < K_COUNT; ++k) {
      X->prof.cum_ms[k] = 0.0;
      X->prof.cum_n[k] = 0;
    }
  }
  X->timing = enable != 0;
  return TG_OK;
}

int32_t tg_kernel_times(const tg_ctx* X, tg_kernel_time* out, int32_t capacity) {
  if (!X || capacity < 0 || (capacity > 0 && !out)) return -1;
  int32_t count = 0;
  for (int k = 0; k < K_COUNT; ++k) {
    if (X->prof.cum_n[k] == 0) continue;
    if (count < capacity) {
      out[count].name = kKernelNames[k];
      out[count].ms = X->prof.cum_ms[k];
      out[count].launches = X->prof.cum_n[k];
    }
    ++count;
  }
  return count;
}

void tg_free(tg_ctx* X) {
  if (!X) return;
  if (X->side) {
    cudaStreamSynchronize(X->side);
    cudaStreamDestroy(X->side);
  }
  if (X->fork_ev) cudaEventDestroy(X->fork_ev);
  if (X->join_ev) cudaEventDestroy(X->join_ev);
  if (X->copy) {
    cudaStreamSynchronize(X->copy);
    cudaStreamDestroy(X->copy);
    cudaEventDestroy(X->entry_ev);
    for (int g = 0; g < 4; ++g) cudaEventDestroy(X->up_ev[g]);
    cudaEventDestroy(X->s5_ev);
  }
  for (cudaEvent_t e : X->prof.ev) cudaEventDestroy(e);
  if (X->pev_ok)
    for (cudaEvent_t e : X->pev) cudaEventDestroy(e);
  delete X;
}

const char* tg_error_string(tg_status s) {
  switch (s) {
    case TG_OK: return "success";
    case TG_ERR_ARG: return "invalid argument";
    case TG_ERR_CUDA: return "CUDA error";
    case TG_ERR_NOCONV: return "CG did not converge within its iteration limit";
    case TG_ERR_NONFINITE: return "non-finite residual";
    case TG_ERR_TIMEOUT: return "device-side wait timed out";
    case TG_ERR_STATE: return "context unusable after an earlier error";
    case TG_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
  }
  return "unknown status";
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Allocation-free elasticity solve (tg_solve_elasticity_static).  Its scratch lives in a
// file-scope device array instead of a caller workspace.  Host code must not use the array's
// name as an address (it is a host-side stand-in); the device address is looked up once per
// device with cudaGetSymbolAddress and cached.
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[TG_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_addr[kMaxDevices] = {};

// device address of g_static_scratch on the current device (set up on first use)
tg_status static_scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return TG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return TG_ERR_CUDA;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return TG_OK;
}

}  // namespace

extern "C" tg_status tg_solve_elasticity_static(const tg_grid* grid, const tg_params* params,
                                                const tg_state* state, double* const rhs[3],
                                                double* u[3], void* cuda_stream,
                                                tg_stats* stats) {
  if (!grid_ok(grid) || !params_ok(params) || !state || !u) return TG_ERR_ARG;
  const double* must[] = {state->p, state->i, state->n, state->g, state->w, state->f, state->bg,
                          u[0], u[1], u[2]};
  for (const double* q : must)
    if (!q || ((uintptr_t)q & 15u)) return TG_ERR_ARG;
  if (rhs && (!rhs[0] || !rhs[1] || !rhs[2])) return TG_ERR_ARG;
  const Geo G = make_geo(grid, sm_count());
  const Layout L = layout(G, TG_FP64);
  if (G.nvox > TG_STATIC_MAX_VOXELS || L.total > (size_t)TG_STATIC_SCRATCH_BYTES)
    return TG_ERR_WORKSPACE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TG_ERR_CUDA;
  void* base = nullptr;
  tg_status e = static_scratch_address(dev, &base);
  if (e != TG_OK) return e;

  // a value-initialised context on the stack over the static scratch (host memory only)
  tg_ctx X{};
  X.G = G;
  X.L = L;
  X.prm = *params;
  X.dp = make_dev_params(params);
  X.prec = TG_FP64;
  X.st = *state;
  X.stream = (cudaStream_t)cuda_stream;
  X.device = dev;
  X.ws = (char*)base;
  for (int a = 0; a < A_COUNT; ++a) X.a[a] = (double*)(X.ws + L.arr[a]);
  X.partial = (double*)(X.ws + L.partial);
  X.counter = (unsigned int*)(X.ws + L.counter);
  X.scal = (CgScal*)(X.ws + L.scal);
  if (stats) memset(stats, 0, sizeof(*stats));
  // the reduction counter must start at zero; the previous call may have left anything
  if (cudaMemsetAsync(X.counter, 0, ALIGN, X.stream) != cudaSuccess) return TG_ERR_CUDA;
  e = build_elas_coef(&X, rhs == nullptr);
  if (e != TG_OK) return e;
  double* const uu[3] = {u[0], u[1], u[2]};
  e = elas_solve(&X, uu, rhs, rhs == nullptr, 0.0, stats);
  if (e == TG_OK && stats) fill_profile(&X, stats);
  return e;
}

// =============================================================================================
// Batches: many simulations of different grids stepped together.  Each simulation keeps its own
// context (state, workspace); the batch adds the tile and flat-range lists that let one launch
// cover all simulations, and runs the solvers as persistent cooperative kernels.  One step is
// captured once in a CUDA graph and replayed.
namespace {

constexpr int BATCH_GRAPH_SWEEPS = 6;   // refinement sweeps inside the step graph
constexpr int BATCH_MAX_SWEEPS = 64;    // total, including sweeps run after the graph
const int kZcCandidates[] = {8, 16, 32, 64};
constexpr unsigned long long kDefaultTimeoutNs = 20ULL * 1000 * 1000 * 1000;   // 20 s

struct BatchArea {
  size_t sims, tile_sim, item_sim, partial, counters, bar, stat, total;
  size_t partial_per_sim;   // doubles
};

Geo geo_with_depth(const Geo& G0, int zc) {
  Geo G = G0;
  G.zc = std::max(1, std::min(zc, G.nz));
  const unsigned gz = (unsigned)((G.nz + G.zc - 1) / G.zc);
  G.grid = dim3(G0.grid.x, G0.grid.y, gz);
  G.nblocks = (int)(G.grid.x * G.grid.y * gz);
  return G;
}

long long flat_items(long long n) {
  const long long g = n / 4;
  return std::max(1LL, (g + FLAT_GROUPS - 1) / FLAT_GROUPS);
}

BatchArea batch_area(int nsims, const tg_grid* grids) {
  BatchArea A;
  long long max_tiles_total = 0, items_total = 0, per_sim = 0;
  for (int s = 0; s < nsims; ++s) {
    const Geo G = make_geo(&grids[s], sm_count());
    const Geo Gmin = geo_with_depth(G, kZcCandidates[0]);
    max_tiles_total += Gmin.nblocks;
    const long long it = flat_items(G.nvox);
    items_total += it;
    per_sim = std::max(per_sim, std::max((long long)Gmin.nblocks, it) * MAX_NV);
  }
  size_t off = 0;
  A.sims = off;
  off += round_up((size_t)nsims * sizeof(BSim));
  A.tile_sim = off;
  off += round_up((size_t)max_tiles_total * sizeof(int));
  A.item_sim = off;
  off += round_up((size_t)items_total * sizeof(int));
  A.partial_per_sim = (size_t)per_sim;
  A.partial = off;
  off += round_up((size_t)nsims * per_sim * sizeof(double));
  A.counters = off;
  off += round_up((size_t)nsims * 64);
  A.bar = off;
  off += ALIGN;
  A.stat = off;
  off += round_up((size_t)nsims * sizeof(BatchStat));
  A.total = off;
  return A;
}

// Enqueue S0, S1 and the copy of i before diffusion for one simulation (mixed precision).
tg_status queue_pre_diffusion(tg_ctx* X, double dt) {
  const Geo& G = X->G;
  tg_state& S = X->st;
  cudaStream_t s = X->stream;
  const size_t bytes = (size_t)G.nvox * sizeof(double);
  double* const Kf[3] = {X->a[A_KF0], X->a[A_KF1], X->a[A_KF2]};
  CK(launch_diff_coef(G, X->dp, dt, S.g, S.w, S.f, Kf, X->a[A_DSUM_D], X->a[A_DINV_D],
                      X->a[A_RHO], s));
  const double* const v[3] = {S.v[0], S.v[1], S.v[2]};
  const double* const qin[6] = {S.p, S.i, S.n, S.g, S.w, S.f};
  const Sl32 T = sl32_view(X);
  CK(launch_sl32_pack(G, v, qin, T, s));
  CK(launch_sl32(G, dt, T, s));
  CK(cudaMemcpyAsync(X->a[A_IDAG], S.i, bytes, cudaMemcpyDeviceToDevice, s));
  return TG_OK;
}

// Enqueue the fix-up and reactions (S2-S5) and the elasticity coefficients for one simulation.
tg_status queue_post_diffusion(tg_ctx* X, double dt) {
  const Geo& G = X->G;
  tg_state& S = X->st;
  cudaStream_t s = X->stream;
  CK(launch_react(G, X->dp, dt, X->a[A_RHO], X->a[A_IDAG], S.p, S.i, S.n, S.g, S.w, S.o, S.l,
                  X->prec == TG_MIXED, single_species(X), s));
  tg_status e = build_elas_coef(X, true);
  if (e != TG_OK) return e;
  double* const u[3] = {S.u[0], S.u[1], S.u[2]};
  const Elas E = elas_view(X, u, nullptr);
  CK(launch_elas32_coef(G, E, elas32_view(X), s));
  CK(launch_elas_extrapolate(G, E, dt, false, s));   // u^n + dt v^n; du = dt v^n
  return TG_OK;
}

}  // namespace

struct tg_batch {
  int nsims;
  cudaStream_t stream;
  int device;
  std::vector<tg_ctx*> ctx;
  char* ws;
  BatchArea area;
  std::vector<BSim> h_sims;
  BSim* d_sims;
  int* d_tile_sim;
  int* d_item_sim;
  double* d_partial;
  unsigned int* d_counters;
  unsigned int* d_bar;
  int* d_err;
  BatchStat* d_stat;
  int zc;
  int coop_cn, coop_el;
  int ntiles, nitems;
  unsigned long long timeout_ns;
  cudaGraphExec_t graph;
  bool graph_ready;
  double graph_dt;
  bool use_graph;
  int broken;
  long long launches;
  // concurrent batches: every member steps through the single-simulation path on its own
  // stream, driven by a pool of host threads
  bool concurrent;
  int nthreads;
  std::vector<cudaStream_t> streams;
};

namespace {

tg_status bfail(tg_batch* B, tg_status s) {
  if (B && s != TG_OK && s != TG_ERR_ARG) B->broken = 1;
  return s;
}

#define BCK(call)                          \
  do {                                     \
    if ((call) != cudaSuccess) {           \
      return bfail(B, TG_ERR_CUDA);        \
    }                                      \
  } while (0)

BatchDev batch_dev(const tg_batch* B, int maxit) {
  BatchDev D;
  D.sims = B->d_sims;
  D.nsims = B->nsims;
  D.tile_sim = B->d_tile_sim;
  D.item_sim = B->d_item_sim;
  D.ntiles = B->ntiles;
  D.nitems = B->nitems;
  D.bar = B->d_bar;
  D.err = B->d_err;
  D.timeout_ns = B->timeout_ns;
  D.maxit = maxit;
  D.tau_min = TAU_INNER;
  D.max_sweeps = BATCH_MAX_SWEEPS;
  return D;
}

int batch_maxit(const tg_batch* B) {
  int m = 0;
  for (const BSim& S : B->h_sims) m = std::max(m, std::max(S.maxit_elas, S.maxit_diff));
  return m;
}

// lay the simulations out as tiles of depth zc; upload the descriptors and lists
tg_status build_tiling(tg_batch* B, int zc) {
  std::vector<int> tile_sim, item_sim;
  B->h_sims.resize(B->nsims);
  for (int s = 0; s < B->nsims; ++s) {
    tg_ctx* X = B->ctx[s];
    BSim& S = B->h_sims[s];
    S.G = geo_with_depth(X->G, zc);
    S.K = make_consts32(S.G);
    double* const u[3] = {X->st.u[0], X->st.u[1], X->st.u[2]};
    S.E = elas_view(X, u, nullptr);
    S.I = elas32_view(X);
    S.C = cn_view(X);
    double* part = B->d_partial + (size_t)s * B->area.partial_per_sim;
    unsigned int* cnt = B->d_counters + (size_t)s * 16;
    S.E.partial = S.I.partial = S.C.partial = part;
    S.E.counter = S.I.counter = S.C.counter = cnt;
    S.Sout = X->scal + 3;
    S.tile0 = (int)tile_sim.size();
    S.ntiles = S.G.nblocks;
    for (int t = 0; t < S.ntiles; ++t) tile_sim.push_back(s);
    S.item0 = (int)item_sim.size();
    S.nitems = (int)flat_items(S.G.nvox);
    for (int t = 0; t < S.nitems; ++t) item_sim.push_back(s);
    S.n = S.G.nvox;
    S.rtol_elas = X->prm.rtol_elas;
    S.rtol_diff = X->prm.rtol_diff;
    S.maxit_elas = X->prm.maxit_elas;
    S.maxit_diff = X->prm.maxit_diff;
  }
  B->zc = zc;
  B->ntiles = (int)tile_sim.size();
  B->nitems = (int)item_sim.size();
  BCK(cudaMemcpyAsync(B->d_sims, B->h_sims.data(), B->h_sims.size() * sizeof(BSim),
                      cudaMemcpyHostToDevice, B->stream));
  BCK(cudaMemcpyAsync(B->d_tile_sim, tile_sim.data(), tile_sim.size() * sizeof(int),
                      cudaMemcpyHostToDevice, B->stream));
  BCK(cudaMemcpyAsync(B->d_item_sim, item_sim.data(), item_sim.size() * sizeof(int),
                      cudaMemcpyHostToDevice, B->stream));
  BCK(cudaMemsetAsync(B->d_counters, 0, (size_t)B->nsims * 64, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  B->graph_ready = false;
  return TG_OK;
}

// everything one step queues before the refinement sweeps that run after the graph
tg_status queue_step(tg_batch* B, double dt) {
  const BatchDev D = batch_dev(B, batch_maxit(B));
  BCK(cudaMemsetAsync(B->d_bar, 0, ALIGN, B->stream));
  BCK(launch_batch_reset(D, B->stream));
  for (tg_ctx* X : B->ctx) {
    tg_status e = queue_pre_diffusion(X, dt);
    if (e != TG_OK) return bfail(B, e);
  }
  BCK(launch_batch_cn(D, B->coop_cn, B->stream));
  for (tg_ctx* X : B->ctx) {
    tg_status e = queue_post_diffusion(X, dt);
    if (e != TG_OK) return bfail(B, e);
  }
  for (int k = 0; k < BATCH_GRAPH_SWEEPS; ++k) BCK(launch_batch_sweep(D, B->coop_el, B->stream));
  BCK(launch_batch_status(D, B->d_stat, B->stream));
  // per simulation: S0 faces and diagonal, divergence, FP32 copies, transport; reactions,
  // Lame, elasticity coefficients, their FP32 copies, the extrapolated start
  B->launches += 2 + 1 + (long long)B->ctx.size() * 10 + 3LL * BATCH_GRAPH_SWEEPS + 1;
  return TG_OK;
}

tg_status capture_step(tg_batch* B, double dt) {
  if (B->graph_ready) {
    cudaGraphExecDestroy(B->graph);
    B->graph_ready = false;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return TG_ERR_CUDA;
  const long long before = B->launches;
  const int broken = B->broken;
  std::vector<int> ctx_broken;
  for (tg_ctx* X : B->ctx) ctx_broken.push_back(X->broken);
  tg_status e = queue_step(B, dt);
  B->launches = before;
  B->broken = broken;                   // a capture that fails only disables the graph
  for (size_t k = 0; k < B->ctx.size(); ++k) B->ctx[k]->broken = ctx_broken[k];
  cudaError_t ce = cudaStreamEndCapture(B->stream, &g);
  if (e != TG_OK || ce != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return e != TG_OK ? e : TG_ERR_CUDA;
  }
  ce = cudaGraphInstantiate(&B->graph, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return TG_ERR_CUDA;
  }
  B->graph_ready = true;
  B->graph_dt = dt;
  return TG_OK;
}

tg_status batch_read_status(tg_batch* B, std::vector<BatchStat>& st) {
  st.resize(B->nsims);
  BCK(cudaMemcpyAsync(st.data(), B->d_stat, B->nsims * sizeof(BatchStat), cudaMemcpyDeviceToHost,
                      B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  return TG_OK;
}

tg_status batch_check_timeout(tg_batch* B) {
  int err = 0;
  BCK(cudaMemcpyAsync(&err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  return err ? bfail(B, TG_ERR_TIMEOUT) : TG_OK;
}

tg_status batch_one_step(tg_batch* B, double dt, tg_batch_stats* stats) {
  if (B->use_graph) {
    if (!B->graph_ready || B->graph_dt != dt) {
      tg_status e = capture_step(B, dt);
      if (e != TG_OK) B->use_graph = false;     // fall back to direct launches
    }
  }
  if (B->use_graph && B->graph_ready) {
    BCK(cudaGraphLaunch(B->graph, B->stream));
    B->launches += 2 + 1 + (long long)B->ctx.size() * 10 + 3LL * BATCH_GRAPH_SWEEPS + 1;
  } else {
    tg_status e = queue_step(B, dt);
    if (e != TG_OK) return e;
  }
  tg_status e = batch_check_timeout(B);
  if (e != TG_OK) return e;
  std::vector<BatchStat> st;
  e = batch_read_status(B, st);
  if (e != TG_OK) return e;
  // refinement sweeps beyond the ones in the graph (rare)
  const BatchDev D = batch_dev(B, batch_maxit(B));
  for (int extra = 0; extra < BATCH_MAX_SWEEPS; ++extra) {
    bool running = false;
    for (const BatchStat& b : st) running |= b.elas_status == CG_RUNNING;
    if (!running) break;
    BCK(cudaMemsetAsync(B->d_bar, 0, ALIGN, B->stream));
    BCK(launch_batch_sweep(D, B->coop_el, B->stream));
    BCK(launch_batch_status(D, B->d_stat, B->stream));
    B->launches += 4;
    e = batch_check_timeout(B);
    if (e != TG_OK) return e;
    e = batch_read_status(B, st);
    if (e != TG_OK) return e;
  }
  for (const BatchStat& b : st) {
    for (int r = 0; r < 3; ++r) {
      if (b.cn_status[r] == CG_NONFINITE) return bfail(B, TG_ERR_NONFINITE);
      if (b.cn_status[r] != CG_CONVERGED && b.cn_status[r] != CG_ZERO_RHS)
        return bfail(B, TG_ERR_NOCONV);
    }
    if (b.elas_status == CG_NONFINITE) return bfail(B, TG_ERR_NONFINITE);
    if (b.elas_status != CG_CONVERGED && b.elas_status != CG_ZERO_RHS)
      return bfail(B, TG_ERR_NOCONV);
  }
  BCK(launch_batch_finish(D, 1.0 / dt, B->stream));
  B->launches += 1;
  BCK(cudaStreamSynchronize(B->stream));
  if (stats) {
    stats->steps += 1;
    for (const BatchStat& b : st) {
      stats->it_elas_total += b.elas_inner;
      stats->sweeps_total += b.elas_sweeps;
      stats->it_diff_total += b.cn_it[0] + b.cn_it[1] + b.cn_it[2];
      stats->it_elas_max = std::max<int64_t>(stats->it_elas_max, b.elas_inner);
      stats->relres_elas_max = std::max(stats->relres_elas_max, b.elas_relres);
    }
  }
  return TG_OK;
}

}  // namespace

extern "C" {

size_t tg_batch_workspace_bytes(int32_t nsims, const tg_grid* grids, tg_precision prec) {
  if (nsims <= 0 || !grids || prec != TG_MIXED) return 0;
  size_t total = 0;
  for (int s = 0; s < nsims; ++s) {
    const size_t b = tg_workspace_bytes(&grids[s], nullptr, prec);
    if (b == 0) return 0;
    total += round_up(b);
  }
  return total + batch_area(nsims, grids).total;
}

tg_status tg_batch_init(int32_t nsims, const tg_grid* grids, const tg_params* params,
                        const tg_state* states, tg_precision prec, void* workspace,
                        size_t workspace_bytes, void* cuda_stream, tg_batch** out) {
  if (out) *out = nullptr;
  if (!out || nsims <= 0 || !grids || !params || !states || prec != TG_MIXED) return TG_ERR_ARG;
  for (int s = 0; s < nsims; ++s)   // the persistent solvers step the multispecies model
    if (params[s].model != TG_MODEL_MULTISPECIES) return TG_ERR_ARG;
  const size_t need = tg_batch_workspace_bytes(nsims, grids, prec);
  if (need == 0) return TG_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 || workspace_bytes < need)
    return TG_ERR_WORKSPACE;
  tg_batch* B = new (std::nothrow) tg_batch();
  if (!B) return TG_ERR_CUDA;
  B->nsims = nsims;
  B->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&B->device);
  B->timeout_ns = kDefaultTimeoutNs;
  B->use_graph = true;
  char* base = (char*)workspace;
  size_t off = 0;
  for (int s = 0; s < nsims; ++s) {
    const size_t b = tg_workspace_bytes(&grids[s], nullptr, prec);
    tg_params ps = params[s];
    ps.precond_elas = TG_PRECOND_JACOBI;   // the persistent batch solvers are Jacobi-PCG
    tg_ctx* X = nullptr;
    tg_status e = tg_init(&grids[s], &ps, prec, &states[s], base + off, b, cuda_stream, 0, &X,
                          nullptr);
    if (e != TG_OK) {
      for (tg_ctx* c : B->ctx) tg_free(c);
      delete B;
      return e;
    }
    X->in_batch = true;      // the batch's persistent residual kernel reads FP64 faces
    X->df_res = false;
    X->cn_df = false;
    B->ctx.push_back(X);
    off += round_up(b);
  }
  B->ws = base + off;
  B->area = batch_area(nsims, grids);
  B->d_sims = (BSim*)(B->ws + B->area.sims);
  B->d_tile_sim = (int*)(B->ws + B->area.tile_sim);
  B->d_item_sim = (int*)(B->ws + B->area.item_sim);
  B->d_partial = (double*)(B->ws + B->area.partial);
  B->d_counters = (unsigned int*)(B->ws + B->area.counters);
  B->d_bar = (unsigned int*)(B->ws + B->area.bar);
  B->d_err = (int*)(B->ws + B->area.bar + 64);
  B->d_stat = (BatchStat*)(B->ws + B->area.stat);
  const int sms = sm_count();
  B->coop_cn = std::max(1, batch_coop_blocks_per_sm(0)) * sms;
  B->coop_el = std::max(1, batch_coop_blocks_per_sm(1)) * sms;
  tg_status e = build_tiling(B, 8);
  if (e != TG_OK) {
    tg_batch_free(B);
    return e;
  }
  *out = B;
  return TG_OK;
}

size_t tg_batch_concurrent_workspace_bytes(int32_t nsims, const tg_grid* grids,
                                           const tg_params* params, tg_precision prec) {
  if (nsims <= 0 || !grids || !params || (prec != TG_MIXED && prec != TG_FP64)) return 0;
  size_t total = 0;
  for (int s = 0; s < nsims; ++s) {
    const size_t b = tg_workspace_bytes(&grids[s], &params[s], prec);
    if (b == 0) return 0;
    total += round_up(b);
  }
  return total;
}

tg_status tg_batch_concurrent_init(int32_t nsims, const tg_grid* grids, const tg_params* params,
                                   const tg_state* states, tg_precision prec, void* workspace,
                                   size_t workspace_bytes, int32_t nthreads, void* cuda_stream,
                                   tg_batch** out) {
  if (out) *out = nullptr;
  if (!out || nsims <= 0 || !grids || !params || !states || nthreads < 0) return TG_ERR_ARG;
  const size_t need = tg_batch_concurrent_workspace_bytes(nsims, grids, params, prec);
  if (need == 0) return TG_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace % ALIGN) != 0 || workspace_bytes < need)
    return TG_ERR_WORKSPACE;
  tg_batch* B = new (std::nothrow) tg_batch();
  if (!B) return TG_ERR_CUDA;
  B->nsims = nsims;
  B->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&B->device);
  B->concurrent = true;
  B->nthreads = nthreads > 0 ? std::min<int>(nthreads, nsims) : std::min<int>(nsims, 8);
  // the callers' work on cuda_stream (the states' upload) comes first
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) {
    delete B;
    return TG_ERR_CUDA;
  }
  char* base = (char*)workspace;
  size_t off = 0;
  for (int s = 0; s < nsims; ++s) {
    cudaStream_t st = nullptr;
    tg_status e = TG_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) e = TG_ERR_CUDA;
    tg_ctx* X = nullptr;
    const size_t b = tg_workspace_bytes(&grids[s], &params[s], prec);
    if (e == TG_OK)
      e = tg_init(&grids[s], &params[s], prec, &states[s], base + off, b, st, 0, &X, nullptr);
    if (e == TG_OK && cudaStreamSynchronize(st) != cudaSuccess) e = TG_ERR_CUDA;
    if (e != TG_OK) {
      if (X) tg_free(X);
      if (st) cudaStreamDestroy(st);
      tg_batch_free(B);
      return e;
    }
    B->streams.push_back(st);
    B->ctx.push_back(X);
    off += round_up(b);
  }
  *out = B;
  return TG_OK;
}

}  // extern "C"

namespace {

// Step the members of a concurrent batch: the host threads take members off one list, largest
// first (a longest-processing-time schedule), and step each through all nsteps before taking
// the next; members share nothing, so the only synchronisation is the list counter.  The
// first failure stops the other threads at their next member.
tg_status batch_concurrent_step(tg_batch* B, double dt, int32_t nsteps, tg_batch_stats* stats) {
  const int n = B->nsims;
  std::vector<int> order(n);
  for (int s = 0; s < n; ++s) order[s] = s;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return B->ctx[a]->G.nvox > B->ctx[b]->G.nvox; });
  std::atomic<int> next{0};
  std::atomic<int> err{TG_OK};
  std::mutex mu;
  tg_batch_stats acc;
  memset(&acc, 0, sizeof(acc));
  auto worker = [&]() {
    if (cudaSetDevice(B->device) != cudaSuccess) {
      err.store(TG_ERR_CUDA);
      return;
    }
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= n || err.load() != TG_OK) return;
      const int s = order[q];
      tg_stats st;
      const tg_status e = tg_step(B->ctx[s], dt, nsteps, nullptr, &st);
      if (e != TG_OK) {
        int expect = TG_OK;
        err.compare_exchange_strong(expect, (int)e);
        return;
      }
      std::lock_guard<std::mutex> lock(mu);
      acc.it_elas_total += st.it_elas_total;
      acc.it_elas_max = std::max<int64_t>(acc.it_elas_max, st.it_elas);
      acc.it_diff_total += st.it_diff_total;
      acc.relres_elas_max = std::max(acc.relres_elas_max, st.relres_elas);
      acc.launches += st.launches;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < B->nthreads; ++t) pool.emplace_back(worker);
  worker();   // the calling thread is one of the pool
  for (std::thread& t : pool) t.join();
  if (err.load() != TG_OK) return (tg_status)err.load();
  if (stats) {
    *stats = acc;
    stats->steps = nsteps;
  }
  return TG_OK;
}

}  // namespace

extern "C" {

tg_status tg_batch_step(tg_batch* B, double dt, int32_t nsteps, tg_batch_stats* stats) {
  if (!B) return TG_ERR_ARG;
  if (B->broken) return TG_ERR_STATE;
  if (!(dt > 0.0) || !isfinite(dt) || nsteps < 0) return TG_ERR_ARG;
  if (stats) memset(stats, 0, sizeof(*stats));
  BCK(cudaSetDevice(B->device));
  if (B->concurrent) {
    const tg_status e = batch_concurrent_step(B, dt, nsteps, stats);
    return e == TG_OK ? e : bfail(B, e);
  }
  B->launches = 0;
  for (int32_t s = 0; s < nsteps; ++s) {
    tg_status e = batch_one_step(B, dt, stats);
    if (e != TG_OK) return bfail(B, e);
  }
  if (stats) {
    stats->launches = B->launches;
    stats->graph = B->use_graph && B->graph_ready ? 1 : 0;
    stats->tile_depth = B->zc;
    stats->coop_blocks = B->coop_el;
  }
  return TG_OK;
}

// Pick the tile depth and the persistent grid size of the elasticity inner solver by timing
// a bounded number of inner iterations on the current state (only scratch arrays change).
tg_status tg_batch_autotune(tg_batch* B, double dt, tg_batch_tune* result) {
  if (!B) return TG_ERR_ARG;
  if (B->broken) return TG_ERR_STATE;
  if (!(dt > 0.0)) return TG_ERR_ARG;
  if (B->concurrent) {   // nothing to tune: the members run the single-simulation kernels
    if (result) memset(result, 0, sizeof(*result));
    return TG_OK;
  }
  BCK(cudaSetDevice(B->device));
  for (tg_ctx* X : B->ctx) {
    tg_status e = build_elas_coef(X, true);
    if (e != TG_OK) return bfail(B, e);
    double* const u[3] = {X->st.u[0], X->st.u[1], X->st.u[2]};
    BCK(launch_elas32_coef(X->G, elas_view(X, u, nullptr), elas32_view(X), B->stream));
  }
  const int sms = sm_count();
  const int max_bps = std::max(1, batch_coop_blocks_per_sm(1));
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  float best = -1.0f;
  int best_zc = B->zc, best_blocks = B->coop_el, n = 0;
  for (int zc : kZcCandidates) {
    tg_status e = build_tiling(B, zc);
    if (e != TG_OK) return e;
    for (int bps = 1; bps <= max_bps; ++bps) {
      const int blocks = bps * sms;
      float ms_best = -1.0f;
      for (int rep = 0; rep < 2; ++rep) {
        BatchDev D = batch_dev(B, batch_maxit(B));
        BCK(cudaMemsetAsync(B->d_bar, 0, ALIGN, B->stream));
        BCK(launch_batch_reset(D, B->stream));
        BCK(launch_batch_residual(D, B->stream));
        BCK(launch_batch_force_inner(D, B->stream));    // u^0 may already solve the system
        D.maxit = 16;                                   // a fixed, short inner run
        BCK(cudaEventRecord(e0, B->stream));
        BCK(launch_batch_elas_inner(D, blocks, B->stream));
        BCK(cudaEventRecord(e1, B->stream));
        BCK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        BCK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms_best < 0.0f || ms < ms_best) ms_best = ms;
      }
      if (result && n < 32) {
        result->zc[n] = zc;
        result->blocks[n] = blocks;
        result->ms[n] = ms_best;
      }
      ++n;
      if (best < 0.0f || ms_best < best) {
        best = ms_best;
        best_zc = zc;
        best_blocks = blocks;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tg_status e = batch_check_timeout(B);
  if (e != TG_OK) return e;
  e = build_tiling(B, best_zc);
  if (e != TG_OK) return e;
  B->coop_el = best_blocks;
  if (result) {
    result->count = std::min(n, 32);
    result->best_zc = best_zc;
    result->best_blocks = best_blocks;
  }
  return TG_OK;
}

tg_status tg_batch_set_timeout(tg_batch* B, uint64_t timeout_ns) {
  if (!B || timeout_ns == 0) return TG_ERR_ARG;
  B->timeout_ns = timeout_ns;
  if (B->graph_ready) {
    cudaGraphExecDestroy(B->graph);
    B->graph_ready = false;
  }
  return TG_OK;
}

void tg_batch_free(tg_batch* B) {
  if (!B) return;
  if (B->graph_ready) cudaGraphExecDestroy(B->graph);
  for (tg_ctx* X : B->ctx) tg_free(X);
  for (cudaStream_t st : B->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  delete B;
}

}  // extern "C"
