// tg_reaction.cu -- the pointwise sub-steps: S2 fix-up of g and w, reactions S3-S5, and the
// Lame / screening mixture of S6.
#include "tg_internal.cuh"

namespace tg {
namespace {

// The rates are evaluated in T: FP64, or FP32 in the mixed precision (the state and its
// Heun update stay FP64; only the rate arithmetic, dominated by exp and divisions, drops to
// FP32, whose relative error ~1e-7 in an increment dt * rate is far below the mixed
// precision's tolerance).
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }

// The rate parameters in FP32, converted once per thread (FP64 -> FP32 conversions run on
// GB300's slow FP64 pipe, so none is left inside the voxel loop).
struct RateParams32 {
  float inv_eps_H, o_inv, o_mit, beta0, sigma_b, rho_i_frac, gamma, o_hyp, alpha0;
  float delta_p, delta_s, o_heal, delta_e, delta_half, delta_l;
  __device__ explicit RateParams32(const DevParams& P)
      : inv_eps_H(f32_of(P.inv_eps_H)), o_inv(f32_of(P.o_inv)), o_mit(f32_of(P.o_mit)),
        beta0(f32_of(P.beta0)), sigma_b(f32_of(P.sigma_b)), rho_i_frac(f32_of(P.rho_i_frac)),
        gamma(f32_of(P.gamma)), o_hyp(f32_of(P.o_hyp)), alpha0(f32_of(P.alpha0)),
        delta_p(f32_of(P.delta_p)), delta_s(f32_of(P.delta_s)), o_heal(f32_of(P.o_heal)),
        delta_e(f32_of(P.delta_e)), delta_half(f32_of(P.delta_half)), delta_l(f32_of(P.delta_l)) {}
};

// smoothed Heaviside H(x) = (1 + tanh(x / eps_H)) / 2, evaluated as 1 / (1 + exp(-2 x / eps_H))
// (the same function; this form keeps full relative accuracy where H is tiny)
template <typename T, typename PP>
__device__ __forceinline__ T heaviside(const PP& P, T x) {
  return (T)1 / ((T)1 + exp_t((T)-2 * x * (T)P.inv_eps_H));
}

// oxygen factor of Eq. e:gog_reac_op / e:gog_reac_inv_op
template <typename T, typename PP>
__device__ __forceinline__ T mitosis_factor(const PP& P, T o) {
  if (o > (T)P.o_inv) return (T)1;
  if (o >= (T)P.o_mit) return (o - (T)P.o_mit) / ((T)P.o_inv - (T)P.o_mit);
  return (T)0;
}

// Sources of Eq. e:p, e:i, e:n, e:gm_wm, e:w at fixed oxygen (h, alpha and the mitosis
// factor depend on o only and are passed in).
template <typename T, typename PP>
__device__ __forceinline__ void species_rates(const PP& P, T rho, T o, T h, T alpha, T mf,
                                              const T y[5], T dy[5]) {
  const T p = y[0], i = y[1], g = y[3], w = y[4];
  const T beta = (T)P.beta0 * heaviside<T>(P, (T)P.sigma_b - p - i) * o;   // Eq. e:beta
  const T R = rho * p * ((T)1 - p) * mf;                                   // Eq. e:gog_reac_op
  const T Rt = (T)P.rho_i_frac * rho * i * ((T)1 - i) * mf;                // Eq. e:gog_reac_inv_op
  const T gw = g + w;
  const T fg = gw > (T)0 ? g / gw : (T)0;
  const T fw = gw > (T)0 ? w / gw : (T)0;
  dy[0] = R - alpha * p + beta * i - h * p;
  dy[1] = Rt + alpha * p - beta * i - h * i;
  dy[2] = h * (p + i + g + w);
  dy[3] = -fg * (R + Rt) - h * g;
  dy[4] = -fw * (R + Rt) - h * w;
}

// Single-species model (Eq. e:rd, Eq. e:reac_op): d_t c = rho c (1 - c), and g, w lose
// what c gains in proportion g : w; c is carried in y[0].
template <typename T>
__device__ __forceinline__ void single_rates(T rho, const T y[5], T dy[5]) {
  const T c = y[0], g = y[3], w = y[4];
  const T R = rho * c * ((T)1 - c);
  const T gw = g + w;
  const T fg = gw > (T)0 ? g / gw : (T)0;
  const T fw = gw > (T)0 ? w / gw : (T)0;
  dy[0] = R;
  dy[1] = (T)0;
  dy[2] = (T)0;
  dy[3] = -fg * R;
  dy[4] = -fw * R;
}

// single: the single-species model -- the CN increment of c (in p) leaves g and w, the
// reaction is the logistic one above, and oxygen and edema are not touched
template <typename T>
__global__ void __launch_bounds__(NT) k_react(Geo G, DevParams P, double dt, int single,
                                              const double* __restrict__ rho,
                                              const double* __restrict__ i_dag, double* p,
                                              double* ii, double* n, double* g, double* w,
                                              double* o, double* l) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    // S2 fix-up: the Crank-Nicolson increment of i comes out of g and w, in proportion (the
    // proportions in T: a relative error of ~1e-7 in them moves g and w by ~1e-7 of the small
    // increment)
    double y[5] = {p[c], ii[c], n[c], g[c], w[c]};
    {
      const double di = (single ? y[0] : y[1]) - i_dag[c];
      const T gw = (T)(y[3] + y[4]);
      const double fg = gw > (T)0 ? (double)((T)y[3] / gw) : 0.0;
      const double fw = gw > (T)0 ? (double)((T)y[4] / gw) : 0.0;
      y[3] = y[3] - di * fg;
      y[4] = y[4] - di * fw;
    }
    // S3: one Heun step with the post-diffusion oxygen and the step-start rho
    const double oo = o[c];
    const T ot = (T)oo, r = (T)rho[c], dtt = (T)dt;
    const T h = (T)P.gamma * heaviside<T>(P, (T)P.o_hyp - ot);     // Eq. e:death
    const T alpha = (T)P.alpha0 * heaviside<T>(P, (T)P.o_inv - ot); // Eq. e:alpha
    const T mf = mitosis_factor<T>(P, ot);
    T yt[5], k1v[5], k2v[5], ys[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) yt[s] = (T)y[s];
    if (single)
      single_rates<T>(r, yt, k1v);
    else
      species_rates<T>(P, r, ot, h, alpha, mf, yt, k1v);
#pragma unroll
    for (int s = 0; s < 5; ++s) ys[s] = yt[s] + dtt * k1v[s];
    if (single)
      single_rates<T>(r, ys, k2v);
    else
      species_rates<T>(P, r, ot, h, alpha, mf, ys, k2v);
#pragma unroll
    for (int s = 0; s < 5; ++s) y[s] = y[s] + 0.5 * dt * (double)(k1v[s] + k2v[s]);
    p[c] = y[0];
    ii[c] = y[1];
    n[c] = y[2];
    g[c] = y[3];
    w[c] = y[4];
    if (single) continue;
    // S4: oxygen, d_t o = -delta_p p + delta_s (o_heal - o)(g + w)   (Eq. e:ox)
    const double gwn = y[3] + y[4];
    const double ko1 = -P.delta_p * y[0] + P.delta_s * (P.o_heal - oo) * gwn;
    const double os = oo + dt * ko1;
    const double ko2 = -P.delta_p * y[0] + P.delta_s * (P.o_heal - os) * gwn;
    o[c] = oo + 0.5 * dt * (ko1 + ko2);
    // S5: edema, d_t l = delta_e i / (i + delta_half) (1 - i) - delta_l l   (Eq. e:edema);
    // the source, a rate like those of S3, in T
    const double l0 = l[c];
    const T it = (T)y[1];
    const double src = (double)((T)P.delta_e * it / (it + (T)P.delta_half) * ((T)1 - it));
    const double kl1 = src - P.delta_l * l0;
    const double ls = l0 + dt * kl1;
    const double kl2 = src - P.delta_l * ls;
    l[c] = l0 + 0.5 * dt * (kl1 + kl2);
  }
}

// The same sub-steps with FP32 rates and no FP64 arithmetic but one addition per updated
// value (the mixed precision).  GB300's FP64 pipe issues ~2 lanes per clock per SM, so the
// FP64 form above is bound by it; here each value's increments over S2-S5 are formed in
// FP32 from the split state and added once to the FP64 state:
//   * S2: the CN increment di = i - i_dag as the double-FP32 difference of the two FP64
//     values (a small difference of nearly equal numbers, exact to FP32's precision), then
//     the shares di g / (g + w), di w / (g + w) in FP32;
//   * S3: Heun's rule on the FP32 rates at the post-S2 state;
//   * S4, S5: Heun's rule for oxygen and edema with FP32 rates.
// g and w take the sum of their S2 and S3 increments.  Every increment carries FP32's
// relative error (~6e-8) of a quantity of size dt * rate, as the FP32 rates already do.
__global__ void __launch_bounds__(NT, 4) k_react_f32(Geo G, DevParams P, float dt, int single,
                                                  const double* __restrict__ rho,
                                                  const double* __restrict__ i_dag, double* p,
                                                  double* ii, double* n, double* g, double* w,
                                                  double* o, double* l) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  const float hdt = 0.5f * dt;
  const RateParams32 Q(P);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    const double y0 = p[c], y1 = ii[c], y2 = n[c], y3 = g[c], y4 = w[c];
    // S2 fix-up
    const float di = df_sub(df_split(single ? y0 : y1), df_split(i_dag[c])).hi;
    float yt[5] = {f32_of(y0), f32_of(y1), f32_of(y2), f32_of(y3), f32_of(y4)};
    const float gw = yt[3] + yt[4];
    const float dg = gw > 0.0f ? -di * (yt[3] / gw) : 0.0f;
    const float dw = gw > 0.0f ? -di * (yt[4] / gw) : 0.0f;
    yt[3] += dg;
    yt[4] += dw;
    // S3: one Heun step with the post-diffusion oxygen and the step-start rho
    const double oo = o[c];
    const float ot = f32_of(oo), r = f32_of(rho[c]);
    const float h = Q.gamma * heaviside<float>(Q, Q.o_hyp - ot);
    const float alpha = Q.alpha0 * heaviside<float>(Q, Q.o_inv - ot);
    const float mf = mitosis_factor<float>(Q, ot);
    float k1v[5], k2v[5], ys[5];
    if (single)
      single_rates<float>(r, yt, k1v);
    else
      species_rates<float>(Q, r, ot, h, alpha, mf, yt, k1v);
#pragma unroll
    for (int s = 0; s < 5; ++s) ys[s] = yt[s] + dt * k1v[s];
    if (single)
      single_rates<float>(r, ys, k2v);
    else
      species_rates<float>(Q, r, ot, h, alpha, mf, ys, k2v);
    float inc[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) inc[s] = hdt * (k1v[s] + k2v[s]);
    inc[3] += dg;
    inc[4] += dw;
    const double p1 = y0 + f64_of(inc[0]), i1 = y1 + f64_of(inc[1]);
    const double g1 = y3 + f64_of(inc[3]), w1 = y4 + f64_of(inc[4]);
    p[c] = p1;
    ii[c] = i1;
    n[c] = y2 + f64_of(inc[2]);
    g[c] = g1;
    w[c] = w1;
    if (single) continue;
    // S4: oxygen, d_t o = -delta_p p + delta_s (o_heal - o)(g + w)   (Eq. e:ox)
    const float pt = f32_of(p1), gwn = f32_of(g1) + f32_of(w1);
    const float dp = Q.delta_p, ds = Q.delta_s, oh = Q.o_heal;
    const float ko1 = -dp * pt + ds * (oh - ot) * gwn;
    const float os = ot + dt * ko1;
    const float ko2 = -dp * pt + ds * (oh - os) * gwn;
    o[c] = oo + f64_of(hdt * (ko1 + ko2));
    // S5: edema, d_t l = delta_e i / (i + delta_half) (1 - i) - delta_l l   (Eq. e:edema)
    const double l0 = l[c];
    const float it = f32_of(i1), lt = f32_of(l0), dl = Q.delta_l;
    const float src = Q.delta_e * it / (it + Q.delta_half) * (1.0f - it);
    const float kl1 = src - dl * lt;
    const float ls = lt + dt * kl1;
    const float kl2 = src - dl * ls;
    l[c] = l0 + f64_of(hdt * (kl1 + kl2));
  }
}

// Eq. e:lame over iota = (p + i + n, g, w, f, bg); eta mixed the same way.
__global__ void __launch_bounds__(NT) k_lame(Geo G, DevParams P, const double* __restrict__ p,
                                             const double* __restrict__ ii,
                                             const double* __restrict__ n,
                                             const double* __restrict__ g,
                                             const double* __restrict__ w,
                                             const double* __restrict__ f,
                                             const double* __restrict__ bg, double* mu,
                                             double* lam, double* eta) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    const double iota[5] = {p[c] + ii[c] + n[c], g[c], w[c], f[c], bg[c]};
    double smu = 0.0, slam = 0.0, seta = 0.0;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      smu += P.cmu[s] * iota[s];
      slam += P.clam[s] * iota[s];
      seta += P.eta[s] * iota[s];
    }
    mu[c] = smu;
    lam[c] = slam;
    eta[c] = seta;
  }
}

// Eq. e:lame in double-FP32 for the mixed precision's double-FP32 residual, in one pass: the
// FP64 mu, lambda, eta (for the preconditioner's domain means and the diagonal), their FP32
// copies for the inner solves, the (hi, lo) pairs of mu and lambda, and the pair of
// s = p + n for the force of the next pass.  The FP64 form above spends 17 FP64 operations
// per voxel, which on GB300's FP64 pipe (~2 lanes per clock per SM) bound it; here only the
// three FP64 outputs take one FP64 addition each.
__global__ void __launch_bounds__(NT) k_lame_df(Geo G, DevParams P, const double* __restrict__ p,
                                                const double* __restrict__ ii,
                                                const double* __restrict__ n,
                                                const double* __restrict__ g,
                                                const double* __restrict__ w,
                                                const double* __restrict__ f,
                                                const double* __restrict__ bg, double* mu,
                                                double* lam, double* eta, float* mu32,
                                                float* lam32, float* eta32, float2* mudf,
                                                float2* lamdf, float2* sdf) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= G.nx || j >= G.ny) return;
  Df cmu[5], clam[5], ceta[5];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    cmu[s] = df_split(P.cmu[s]);
    clam[s] = df_split(P.clam[s]);
    ceta[s] = df_split(P.eta[s]);
  }
  const int k0 = blockIdx.z * G.zc, k1 = min(G.nz, k0 + G.zc);
  for (int k = k0; k < k1; ++k) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    const Df sp = df_split(p[c]), sn = df_split(n[c]);
    const Df iota[5] = {df_add_pos(df_add_pos(sp, df_split(ii[c])), sn), df_split(g[c]), df_split(w[c]),
                        df_split(f[c]), df_split(bg[c])};
    Df smu = {0.0f, 0.0f}, slam = {0.0f, 0.0f}, seta = {0.0f, 0.0f};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      smu = df_add_pos(smu, df_mul(cmu[s], iota[s]));   // positive weights and fractions
      slam = df_add_pos(slam, df_mul(clam[s], iota[s]));
      seta = df_add_pos(seta, df_mul(ceta[s], iota[s]));
    }
    mu[c] = df_value(smu);
    lam[c] = df_value(slam);
    eta[c] = df_value(seta);
    mu32[c] = smu.hi;
    lam32[c] = slam.hi;
    eta32[c] = seta.hi;
    mudf[c] = make_float2(smu.hi, smu.lo);
    lamdf[c] = make_float2(slam.hi, slam.lo);
    const Df sum = df_add(sp, sn);
    sdf[c] = make_float2(sum.hi, sum.lo);
  }
}

}  // namespace

cudaError_t launch_react(const Geo& G, const DevParams& P, double dt, const double* rho,
                         const double* i_dag, double* p, double* i, double* n, double* g,
                         double* w, double* o, double* l, bool fp32_rates, bool single,
                         cudaStream_t st) {
  const int sg = single ? 1 : 0;
  if (fp32_rates)
    TG_TIMED(K_REACT, st,
             k_react_f32<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, (float)dt, sg, rho, i_dag, p, i, n,
                                                          g, w, o, l));
  else
    TG_TIMED(K_REACT, st,
             k_react<double><<<G.grid, dim3(BX, BY), 0, st>>>(G, P, dt, sg, rho, i_dag, p, i, n, g, w, o,
                                                               l));
  return cudaGetLastError();
}

cudaError_t launch_lame(const Geo& G, const DevParams& P, const double* p, const double* i,
                        const double* n, const double* g, const double* w, const double* f,
                        const double* bg, double* mu, double* lam, double* eta, cudaStream_t st) {
  TG_TIMED(K_LAME, st,
           k_lame<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, p, i, n, g, w, f, bg, mu, lam, eta));
  return cudaGetLastError();
}

cudaError_t launch_lame_df(const Geo& G, const DevParams& P, const double* p, const double* i,
                           const double* n, const double* g, const double* w, const double* f,
                           const double* bg, double* mu, double* lam, double* eta, float* mu32,
                           float* lam32, float* eta32, float2* mudf, float2* lamdf, float2* sdf,
                           cudaStream_t st) {
  TG_TIMED(K_LAME_DF, st,
           k_lame_df<<<G.grid, dim3(BX, BY), 0, st>>>(G, P, p, i, n, g, w, f, bg, mu, lam, eta,
                                                      mu32, lam32, eta32, mudf, lamdf, sdf));
  return cudaGetLastError();
}

}  // namespace tg
