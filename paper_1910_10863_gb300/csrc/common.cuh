// Shared device/host helpers of the pfmbem library: complex arithmetic,
// Gauss-Legendre tables, Bessel-function recurrences.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define PF_HD __host__ __device__ __forceinline__

// ---------------------------------------------------------------- complex
struct cplx {
  double re, im;
};
struct cplxf {
  float re, im;
};

PF_HD cplx mk(double a, double b) { return cplx{a, b}; }
PF_HD cplx operator+(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
PF_HD cplx operator-(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
PF_HD cplx operator-(cplx a) { return cplx{-a.re, -a.im}; }
PF_HD cplx operator*(cplx a, cplx b) { return cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
PF_HD cplx operator*(double s, cplx a) { return cplx{s * a.re, s * a.im}; }
PF_HD cplx operator*(cplx a, double s) { return cplx{s * a.re, s * a.im}; }
PF_HD cplx& operator+=(cplx& a, cplx b) { a.re += b.re; a.im += b.im; return a; }
PF_HD cplx& operator-=(cplx& a, cplx b) { a.re -= b.re; a.im -= b.im; return a; }
PF_HD cplx conj(cplx a) { return cplx{a.re, -a.im}; }
PF_HD cplx mul_i(cplx a) { return cplx{-a.im, a.re}; }          // i * a
PF_HD double abs2(cplx a) { return a.re * a.re + a.im * a.im; }
PF_HD cplx cdiv(cplx a, cplx b) {
  double d = b.re * b.re + b.im * b.im;
  return cplx{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

PF_HD cplxf mkf(float a, float b) { return cplxf{a, b}; }
PF_HD cplxf operator+(cplxf a, cplxf b) { return cplxf{a.re + b.re, a.im + b.im}; }
PF_HD cplxf operator-(cplxf a, cplxf b) { return cplxf{a.re - b.re, a.im - b.im}; }
PF_HD cplxf operator*(cplxf a, cplxf b) { return cplxf{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
PF_HD cplxf operator*(float s, cplxf a) { return cplxf{s * a.re, s * a.im}; }
PF_HD cplxf& operator+=(cplxf& a, cplxf b) { a.re += b.re; a.im += b.im; return a; }
PF_HD cplxf conj(cplxf a) { return cplxf{a.re, -a.im}; }
PF_HD cplxf operator-(cplxf a) { return cplxf{-a.re, -a.im}; }
PF_HD cplxf& operator-=(cplxf& a, cplxf b) { a.re -= b.re; a.im -= b.im; return a; }
PF_HD cplxf operator*(cplxf a, float s) { return cplxf{s * a.re, s * a.im}; }
PF_HD cplxf mul_i(cplxf a) { return cplxf{-a.im, a.re}; }

// conversions between the two precisions
PF_HD cplxf to_f(cplx a) { return cplxf{(float)a.re, (float)a.im}; }
PF_HD cplx to_d(cplxf a) { return cplx{(double)a.re, (double)a.im}; }
PF_HD cplx to_d(cplx a) { return a; }
// The FP32 pair (hi, lo) of an FP64 complex value: hi = fl32(a), lo = fl32(a - hi);
// hi + lo carries about 48 bits of a.
PF_HD cplxf split_lo(cplx a) {
  const float hr = (float)a.re, hi = (float)a.im;
  return cplxf{(float)(a.re - (double)hr), (float)(a.im - (double)hi)};
}
template <class C> PF_HD C from_d(cplx a);
template <> PF_HD cplx from_d<cplx>(cplx a) { return a; }
template <> PF_HD cplxf from_d<cplxf>(cplx a) { return to_f(a); }

// ---------------------------------------------------------------- limits
#define PF_PMAX 128                // largest expansion order
#define PF_NCOEF (2 * PF_PMAX + 1)
#define PF_GLMAX 16                // largest Gauss-Legendre rule in the ladder
#define PF_MAXLEVEL 12

// Gauss-Legendre nodes/weights on [-1, 1] (Newton on P_n, host side).
void gauss_legendre(int n, double* x, double* w);

// J_0..J_N(x) (x >= 0) by Miller's backward recurrence normalised with
// J_0 + 2 sum_k J_2k = 1.  out must hold N + 1 values.
PF_HD void bessel_j_array(double x, int N, double* out) {
  if (x < 1e-300) {
    out[0] = 1.0;
    for (int n = 1; n <= N; ++n) out[n] = 0.0;
    return;
  }
  double big = (double)N > x ? (double)N : x;
  int ns = 2 * (((int)(big + 16.0 + sqrt(40.0 * big))) / 2);   // even start index
  double jp1 = 0.0, j = 1e-250, sum = 0.0;
  const double tx = 2.0 / x;
  for (int n = ns; n > 0; --n) {
    double jm1 = (n * tx) * j - jp1;
    jp1 = j;
    j = jm1;                       // j = J_{n-1} (unnormalised)
    if (n - 1 <= N) out[n - 1] = j;
    if (((n - 1) & 1) == 0 && n - 1 > 0) sum += 2.0 * j;
    if (fabs(j) > 1e250) {         // rescale
      const double s = 1e-250;
      j *= s; jp1 *= s; sum *= s;
      if (n - 1 <= N)
        for (int q = n - 1; q <= N; ++q) out[q] *= s;
    }
  }
  // the loop leaves out[0] = unnormalised J_0
  sum += out[0];
  double inv = 1.0 / sum;
  for (int n = 0; n <= N; ++n) out[n] *= inv;
}

