// Field I/O shared by the stencil and the solver: one spinor per (site, rhs)
// in the internal even-odd SoA layouts (see Field in common.cuh).
#pragma once
#include "common.cuh"

template <int P> struct PT { typedef float R; };
template <> struct PT<DLMA_FP64> { typedef double R; };

template <class R> struct Spinor { Cx<R> c[4][3]; };

template <int P>
__device__ __forceinline__ Spinor<typename PT<P>::R> load_spinor(const void* __restrict__ base,
                                                                 const float* __restrict__ scale, int Vh, int i) {
  typedef typename PT<P>::R R;
  Spinor<R> s;
  if (P == DLMA_FP64) {
    const double2* b = (const double2*)base;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 v = __ldg(b + (size_t)k * Vh + i);
      s.c[k / 3][k % 3] = cx<R>((R)v.x, (R)v.y);
    }
  } else if (P == DLMA_FP32) {
    const float4* b = (const float4*)base;
#pragma unroll
    for (int q = 0; q < 6; q++) {
      float4 v = __ldg(b + (size_t)q * Vh + i);
      s.c[(2 * q) / 3][(2 * q) % 3] = cx<R>(v.x, v.y);
      s.c[(2 * q + 1) / 3][(2 * q + 1) % 3] = cx<R>(v.z, v.w);
    }
  } else {
    const uint4* b = (const uint4*)base;
    float sc = __ldg(scale + i);
#pragma unroll
    for (int q = 0; q < 3; q++) {
      uint4 v = __ldg(b + (size_t)q * Vh + i);
      unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int r = 0; r < 4; r++) {
        float2 f = __half22float2(*(__half2*)&w[r]);
        int k = 4 * q + r;
        s.c[k / 3][k % 3] = cx<R>(f.x * sc, f.y * sc);
      }
    }
  }
  return s;
}

template <int P>
__device__ __forceinline__ void store_spinor(void* base, float* scale, int Vh, int i,
                                             const Spinor<typename PT<P>::R>& s) {
  if (P == DLMA_FP64) {
    double2* b = (double2*)base;
#pragma unroll
    for (int k = 0; k < 12; k++) b[(size_t)k * Vh + i] = make_double2(s.c[k / 3][k % 3].re, s.c[k / 3][k % 3].im);
  } else if (P == DLMA_FP32) {
    float4* b = (float4*)base;
#pragma unroll
    for (int q = 0; q < 6; q++) {
      Cx<float> a0 = cx<float>((float)s.c[(2 * q) / 3][(2 * q) % 3].re, (float)s.c[(2 * q) / 3][(2 * q) % 3].im);
      Cx<float> a1 = cx<float>((float)s.c[(2 * q + 1) / 3][(2 * q + 1) % 3].re,
                               (float)s.c[(2 * q + 1) / 3][(2 * q + 1) % 3].im);
      b[(size_t)q * Vh + i] = make_float4(a0.re, a0.im, a1.re, a1.im);
    }
  } else {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++)
      m = fmaxf(m, fmaxf(fabsf((float)s.c[k / 3][k % 3].re), fabsf((float)s.c[k / 3][k % 3].im)));
    // sites below 1e-30 (down to float denormals, whose reciprocal overflows) are flushed to zero
    if (!(m > 1e-30f)) m = 0.f;
    const float inv = m > 0.f ? 1.f / m : 0.f;
    uint4* b = (uint4*)base;
#pragma unroll
    for (int q = 0; q < 3; q++) {
      unsigned w[4];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        int k = 4 * q + r;
        __half2 h = __floats2half2_rn((float)s.c[k / 3][k % 3].re * inv, (float)s.c[k / 3][k % 3].im * inv);
        w[r] = *(unsigned*)&h;
      }
      b[(size_t)q * Vh + i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    scale[i] = m;
  }
}

