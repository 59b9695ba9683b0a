// Host build of the library's conversion and double-FP32 helpers (the same header the CUDA
// kernels include), exported for the CPU tests in tests/test_fpconv.py.
#include "tg_fpconv.cuh"

extern "C" {

void tgc_f32_of(const double* x, float* out, long n) {
  for (long q = 0; q < n; ++q) out[q] = tg::f32_of(x[q]);
}

void tgc_f64_of(const float* x, double* out, long n) {
  for (long q = 0; q < n; ++q) out[q] = tg::f64_of(x[q]);
}

void tgc_f64_of_scaled(const float* x, const double* s, double* out, long n) {
  for (long q = 0; q < n; ++q) out[q] = tg::f64_of_scaled(x[q], s[q]);
}

void tgc_df_split(const double* x, float* hi, float* lo, long n) {
  for (long q = 0; q < n; ++q) {
    const tg::Df d = tg::df_split(x[q]);
    hi[q] = d.hi;
    lo[q] = d.lo;
  }
}

void tgc_df_value(const float* hi, const float* lo, double* out, long n) {
  for (long q = 0; q < n; ++q) out[q] = tg::df_value(tg::Df{hi[q], lo[q]});
}

// tanh of the double-FP32 split of x, returned as hi + lo in FP64
void tgc_df_tanh(const double* x, double* out, long n) {
  for (long q = 0; q < n; ++q) {
    const tg::Df t = tg::df_tanh(tg::df_split(x[q]));
    out[q] = (double)t.hi + (double)t.lo;
  }
}

// x / y and x * y of double-FP32 splits, as hi + lo in FP64
void tgc_df_div_mul(const double* x, const double* y, double* quo, double* prod, long n) {
  for (long q = 0; q < n; ++q) {
    const tg::Df a = tg::df_split(x[q]), b = tg::df_split(y[q]);
    const tg::Df d = tg::df_div(a, b), m = tg::df_mul(a, b);
    quo[q] = (double)d.hi + (double)d.lo;
    prod[q] = (double)m.hi + (double)m.lo;
  }
}

// sum_q x[q] y[q] over rows of m terms as one compensated sum started at b (a residual
// b - sum of products when the products are passed negated), returned as hi + lo in FP64
void tgc_cs_dot(const double* b, const double* x, const double* y, double* out, long rows, long m) {
  for (long r = 0; r < rows; ++r) {
    const tg::Df b0 = tg::df_split(b[r]);
    tg::CSum a = {b0.hi, b0.lo};
    for (long q = 0; q < m; ++q) tg::cs_fma(a, tg::df_split(x[r * m + q]), tg::df_split(y[r * m + q]));
    const tg::Df v = tg::cs_value(a);
    out[r] = (double)v.hi + (double)v.lo;
  }
}

}

