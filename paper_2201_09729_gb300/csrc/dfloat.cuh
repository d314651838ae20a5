// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers, |lo| <= ulp(hi) / 2, carrying about 46 significant bits.  GB300
// issues 128 FP32 FMAs per clock and SM against 2 FP64 FMAs, so the dense FP64
// products of the Laplacian eigensolver's final phase (Gram matrices X^dag Y and
// rotations X C of the FP64 blocks) run in df on the FP32 units: every loaded value
// is converted once and used in 32 to 64 products.
//
// The error-free transformations are the classical ones (Knuth's two-sum, Dekker's
// fast two-sum, the FMA form of the exact product): s + e = a + b exactly, and
// p + e = a b exactly.  The sums below use the "sloppy" df addition (one two-sum
// on the high parts, the low parts added in FP32), whose error is bounded by a
// few units of 2^-46 of max(|a|, |b|): an absolute bound, which is what sums of
// products over a block of vectors need.  Every FP32 operation is an explicit _rn
// intrinsic so that the compiler cannot contract or reassociate them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct df {
  float hi, lo;
  __host__ __device__ __forceinline__ df() {}
  __device__ __forceinline__ df(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ df(int v) : hi((float)v), lo(0.f) {}
  __device__ __forceinline__ df(float v) : hi(v), lo(0.f) {}
  __device__ __forceinline__ df(double x);
  __device__ __forceinline__ operator double() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return df(s, e);
}
// s + e = a + b exactly for |a| >= |b| (Dekker)
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// FP64 -> df without FP64 arithmetic: hi keeps the top 24 significant bits of the
// double (truncated), lo the next 23 (the dropped 6 bits are below 2^-46 |x|), both
// assembled from the bit pattern; |x| below 2^-126 flushes to zero, below 2^-103
// keeps hi only.
__device__ __forceinline__ df::df(double x) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned sgn = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
  if (E < 897) { hi = 0.f; lo = 0.f; return; }
  if (E > 1150) { hi = __double2float_rn(x); lo = 0.f; return; }
  const unsigned long long mant = (unsigned long long)b & 0xFFFFFFFFFFFFFull;
  const float h = __int_as_float((int)(sgn | ((unsigned)(E - 896) << 23) | (unsigned)(mant >> 29)));
  float l = 0.f;
  if (E >= 920) {
    const unsigned rem = (unsigned)(mant & 0x1FFFFFFFull) >> 6;   // next 23 bits
    const float base = __int_as_float((int)((unsigned)(E - 919) << 23));
    l = __fsub_rn(__int_as_float((int)(((unsigned)(E - 919) << 23) | rem)), base);   // exact (Sterbenz)
    if (sgn) l = -l;
  }
  const df n = df_fast_two_sum(h, l);
  hi = n.hi;
  lo = n.lo;
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator+(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { a = a + b; return a; }
__device__ __forceinline__ df& operator-=(df& a, df b) { a = a - b; return a; }
// a b + c with one normalisation
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  df s = df_two_sum(p, c.hi);
  float e = __fadd_rn(s.lo, pe);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  e = __fadd_rn(e, c.lo);
  return df_fast_two_sum(s.hi, e);
}
