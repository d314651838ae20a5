// Spatial covariant Laplacian of Eq. 1 and its low modes, batched over
// timeslices.
//
//   (lap v)(m, t) = -6 v(m) + sum_{j=1..3} [U_j(m,t) v(m+j) + U_j(m-j,t)^dag v(m-j)]
//
// The modes are the N lowest eigenpairs of A = -lap(t) (spectrum in [0, 12]) on
// every timeslice at once, by Chebyshev-filtered subspace iteration on a block
// of m = N + buffer vectors per timeslice.  Each iteration filters the block
// with a degree-d Chebyshev polynomial of A that damps [cut, 12] and then
// diagonalises it per timeslice (Rayleigh-Ritz):
//   G = Y^dag Y, H = Y^dag (A Y)  ->  G = Q diag(g) Q^dag, S = Q g^-1/2,
//   S^dag H S = Z diag(theta) Z^dag,  X <- Y S Z,  A X <- (A Y) S Z,
// with the small m x m eigenproblems solved by parallel cyclic Jacobi in the
// block's precision (smalleig.cuh; one CTA per timeslice).
//
// Precision: phase A runs the whole iteration in FP32 until the residuals reach
// ~1e-5.  Phase B keeps X, A X and the Rayleigh-Ritz in FP64 but still filters
// in FP32, on the residual: with R = A X - X Theta and the filter's scalar
// recurrence s_k(theta), p_k(A) X = X s_k(Theta) + E_k where
//   E_{k+1} = a_k A E_k + b_k E_k + c_k E_{k-1} + a_k R s_k(Theta),  E_0 = 0,
// so the FP32 rounding only touches the (small) E, and Y = X + E_d / s_d (the
// filtered block with every column divided by its own s_d, so that the Gram
// matrix stays well conditioned) is formed in FP64.  Stops when every wanted
// pair has ||A x - theta x|| <= tol max(theta, 1).  For tol >= 1e-11 the FP64
// blocks' Gram matrices and rotations compute in double-float (~46 bits,
// dfloat.cuh) on the FP32 units or, for large blocks, with the split-digit
// products of tcproj.cu on the tensor cores; the matvec and the small problems
// stay FP64.
//
// Block layout (row-major per timeslice): element (t, row r = 3 site + colour,
// column j) of a batch of Tn timeslices at (t * 3 Vs + r) * m + j, so a warp
// reads consecutive columns of one site (coalesced) and shares its links.
#include "common.cuh"
#include "dfloat.cuh"
#include "smalleig.cuh"
#include <algorithm>
#include <math.h>

namespace {

template <class R> struct LinkT;
template <> struct LinkT<double> { typedef double2 T; };
template <> struct LinkT<float> { typedef float4 T; };

__device__ __forceinline__ void load_link3(const double2* __restrict__ U, int k, size_t s, size_t V, Cx<double> u[3][3]) {
#pragma unroll
  for (int q = 0; q < 9; q++) {
    double2 e = __ldg(U + ((size_t)k * 9 + q) * V + s);
    u[q / 3][q % 3] = cx<double>(e.x, e.y);
  }
}
__device__ __forceinline__ void load_link3(const float4* __restrict__ U, int k, size_t s, size_t V, Cx<float> u[3][3]) {
#pragma unroll
  for (int q = 0; q < 3; q++) {
    float4 e = __ldg(U + ((size_t)k * 3 + q) * V + s);
    u[(2 * q) / 3][(2 * q) % 3] = cx<float>(e.x, e.y);
    u[(2 * q + 1) / 3][(2 * q + 1) % 3] = cx<float>(e.z, e.w);
  }
  u[2][0] = conj(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
  u[2][1] = conj(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
  u[2][2] = conj(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
}

// NC adjacent complex entries starting at p (16-byte aligned when NC is even): FP32
// pairs move as one 128-bit access
template <int NC>
__device__ __forceinline__ void ld_cols(const Cx<float>* __restrict__ p, Cx<float> (&v)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; c += 2) {
    const float4 e = *(const float4*)(p + c);
    v[c] = cx<float>(e.x, e.y);
    v[c + 1] = cx<float>(e.z, e.w);
  }
}
template <int NC>
__device__ __forceinline__ void ld_cols(const Cx<double>* __restrict__ p, Cx<double> (&v)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; c++) v[c] = p[c];
}
template <int NC>
__device__ __forceinline__ void st_cols(Cx<float>* p, const Cx<float> (&v)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; c += 2) *(float4*)(p + c) = make_float4(v[c].re, v[c].im, v[c + 1].re, v[c + 1].im);
}
template <int NC>
__device__ __forceinline__ void st_cols(Cx<double>* p, const Cx<double> (&v)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; c++) p[c] = v[c];
}

// storage (R) <-> arithmetic (A) precision: A = R, or A = df for FP64 storage (the
// double-float arithmetic of the FP64 phase, see dfloat.cuh)
template <class A, class R> __device__ __forceinline__ Cx<A> to_a(Cx<R> v) { return cx<A>((A)v.re, (A)v.im); }
template <class R, class A> __device__ __forceinline__ Cx<R> to_s(Cx<A> v) { return cx<R>((R)v.re, (R)v.im); }

// out = alpha_t (A in) + beta_t in + gamma_t prev + alpha_t s[t][j] rin,  A = 6 - hopping = -lap
// (in == nullptr: the stencil and beta terms vanish; prev / rin may be nullptr).
// One thread per (site, NC adjacent columns): the six links of the site are loaded
// (and, in FP32, rebuilt from 12 reals) once for NC columns.  The FP32 form is
// compiled for three blocks per SM (80 registers, a few spilled words: matvec of
// 16^3 x 32, N = 32, 61 -> 56 ms against two blocks), FP64 for two.  The block is
// [t][site][colour][m] with m even, so a pair of FP32 columns is 16-byte aligned.
template <class R, class A, int NC>
__global__ void __launch_bounds__(256, sizeof(A) == 4 ? 3 : 2) k_lap(Geom g, int t0, int Tn, int m, const typename LinkT<R>::T* __restrict__ U,
                                             const Cx<R>* __restrict__ in, const Cx<R>* __restrict__ prev,
                                             const Cx<float>* __restrict__ rin, const double* __restrict__ scol,
                                             Cx<R>* __restrict__ out, const double* __restrict__ coef) {
  // 32-bit index arithmetic (the host keeps Tn Vs m below 2^31): 64-bit divisions
  // would cost more than the stencil's arithmetic
  const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned mg = (unsigned)m / NC;
  const unsigned total = (unsigned)Tn * (unsigned)g.Vs * mg;
  if (e >= total) return;
  const unsigned sl = e / mg;
  const int j0 = (int)(e - sl * mg) * NC;
  const int tl = (int)(sl / (unsigned)g.Vs);
  const int ms = (int)(sl - (unsigned)tl * (unsigned)g.Vs);
  const A alpha = (A)coef[3 * tl], beta = (A)coef[3 * tl + 1], gamma = (A)coef[3 * tl + 2];
  const size_t rowbase = (size_t)tl * g.Vs;
  Cx<A> res[3][NC];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int c = 0; c < NC; c++) res[a][c] = cx<A>(0, 0);
  if (in) {
    const int yz = ms / g.L, x = ms - yz * g.L, z = yz / g.L, y = yz - z * g.L;
    const size_t s = (size_t)(t0 + tl) * g.Vs + ms;
    Cx<A> acc[3][NC];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      Cx<R> v[NC];
      ld_cols<NC>(in + ((rowbase + ms) * 3 + a) * m + j0, v);   // own term, kept for beta
#pragma unroll
      for (int c = 0; c < NC; c++) {
        res[a][c] = to_a<A>(v[c]);
        acc[a][c] = (A)6 * res[a][c];
      }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
      int xf = x, yf = y, zf = z, xb = x, yb = y, zb = z;
      if (k == 0) { xf = x + 1 == g.L ? 0 : x + 1; xb = x == 0 ? g.L - 1 : x - 1; }
      else if (k == 1) { yf = y + 1 == g.L ? 0 : y + 1; yb = y == 0 ? g.L - 1 : y - 1; }
      else { zf = z + 1 == g.L ? 0 : z + 1; zb = z == 0 ? g.L - 1 : z - 1; }
      const int mf = xf + g.L * (yf + g.L * zf), mb = xb + g.L * (yb + g.L * zb);
      Cx<A> uf[3][3], ub[3][3];
      load_link3(U, k, s, (size_t)g.V, uf);
      load_link3(U, k, (size_t)(t0 + tl) * g.Vs + mb, (size_t)g.V, ub);
      Cx<R> vf[3][NC], vb[3][NC];
#pragma unroll
      for (int a = 0; a < 3; a++) {
        ld_cols<NC>(in + ((rowbase + mf) * 3 + a) * m + j0, vf[a]);
        ld_cols<NC>(in + ((rowbase + mb) * 3 + a) * m + j0, vb[a]);
      }
#pragma unroll
      for (int c = 0; c < NC; c++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
          Cx<A> h = cx<A>(0, 0);
#pragma unroll
          for (int b = 0; b < 3; b++) {
            fma_acc(h, uf[a][b], to_a<A>(vf[b][c]));
            fma_conj_acc(h, ub[b][a], to_a<A>(vb[b][c]));
          }
          acc[a][c] = acc[a][c] - h;
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int c = 0; c < NC; c++) res[a][c] = alpha * acc[a][c] + beta * res[a][c];
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const size_t idx = ((rowbase + ms) * 3 + a) * m + j0;
    if (prev) {
      Cx<R> pv[NC];
      ld_cols<NC>(prev + idx, pv);
#pragma unroll
      for (int c = 0; c < NC; c++) res[a][c] = res[a][c] + gamma * to_a<A>(pv[c]);
    }
    if (rin) {
      Cx<float> rv[NC];
      ld_cols<NC>(rin + idx, rv);
#pragma unroll
      for (int c = 0; c < NC; c++) {
        const A f = alpha * (A)scol[(size_t)tl * m + j0 + c];
        res[a][c] = res[a][c] + f * cx<A>((A)rv[c].re, (A)rv[c].im);
      }
    }
    Cx<R> o[NC];
#pragma unroll
    for (int c = 0; c < NC; c++) o[c] = to_s<R>(res[a][c]);
    st_cols<NC>(out + idx, o);
  }
}

// Gram partials: part[t][split][i][j] = sum_{k in chunk} conj(X_t[k][i]) Y_t[k][j]
// herm: the product is hermitian (X^dag X, or Y^dag A Y with A hermitian): only the
// tiles on and above the diagonal are computed, k_gram_reduce mirrors the rest
constexpr int GT = 32, GKS = 32;
template <class R, class A>
__global__ void __launch_bounds__(256) k_gram(const Cx<R>* __restrict__ X, const Cx<R>* __restrict__ Y, int n, int m,
                                              int nsplit, int herm, double2* part) {
  __shared__ Cx<A> xs[GKS][GT + 1];
  __shared__ Cx<A> ys[GKS][GT + 1];
  const int tiles_j = (m + GT - 1) / GT;
  int ti = blockIdx.x / tiles_j, tj = blockIdx.x % tiles_j;
  if (herm) {                 // blockIdx.x enumerates the pairs ti <= tj row by row
    int b = blockIdx.x;
    ti = 0;
    while (b >= tiles_j - ti) { b -= tiles_j - ti; ti++; }
    tj = ti + b;
  }
  const int i0 = ti * GT, j0 = tj * GT;
  const int split = blockIdx.y, t = blockIdx.z;
  const int chunk = (n + nsplit - 1) / nsplit;
  const int k0 = split * chunk, k1 = min(n, k0 + chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4, tid = threadIdx.x;
  const Cx<R>* Xt = X + (size_t)t * n * m;
  const Cx<R>* Yt = Y + (size_t)t * n * m;
  Cx<A> acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) acc[a][b] = cx<A>(0, 0);
  for (int kb = k0; kb < k1; kb += GKS) {
#pragma unroll
    for (int q = 0; q < (GKS * GT) / 256; q++) {
      const int e = tid + 256 * q;
      const int r = e / GT, c = e % GT;
      const int k = kb + r;
      Cx<R> vx = cx<R>(0, 0), vy = cx<R>(0, 0);
      if (k < k1) {
        if (i0 + c < m) vx = Xt[(size_t)k * m + i0 + c];
        if (j0 + c < m) vy = Yt[(size_t)k * m + j0 + c];
      }
      xs[r][c] = to_a<A>(vx);
      ys[r][c] = to_a<A>(vy);
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < GKS; r++) {
      const Cx<A> x0 = xs[r][ty], x1 = xs[r][ty + 16], y0 = ys[r][tx], y1 = ys[r][tx + 16];
      fma_conj_acc(acc[0][0], x0, y0);
      fma_conj_acc(acc[0][1], x0, y1);
      fma_conj_acc(acc[1][0], x1, y0);
      fma_conj_acc(acc[1][1], x1, y1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < m && j < m)
        part[(((size_t)t * nsplit + split) * m + i) * m + j] = make_double2((double)acc[a][b].re, (double)acc[a][b].im);
    }
}

__global__ void k_gram_reduce(const double2* part, int nsplit, int m, int Tn, int herm, double2* G) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)m * m;
  if (e >= per * Tn) return;
  const size_t t = e / per;
  const int i = (int)((e % per) / m), j = (int)(e % m);
  const bool mirror = herm && (i / GT) > (j / GT);    // tile below the diagonal: conj of (j, i)
  const size_t ij = mirror ? (size_t)j * m + i : (size_t)i * m + j;
  double2 s = make_double2(0, 0);
  for (int q = 0; q < nsplit; q++) {
    const double2 v = part[(t * nsplit + q) * per + ij];
    s.x += v.x;
    s.y += v.y;
  }
  if (mirror) s.y = -s.y;
  G[e] = s;
}

// rotation Z_t = X_t C_t (X_t n x m row-major, C_t m x m row-major FP64); 64 x 64 output tiles
constexpr int RT = 64, RL = 16;
template <class R, class A>
__global__ void __launch_bounds__(256) k_rotate(const Cx<R>* __restrict__ X, const double2* __restrict__ Cm, int n,
                                                int m, Cx<R>* __restrict__ Z) {
  __shared__ Cx<A> xs[RT][RL + 1];
  __shared__ Cx<A> cs[RL][RT + 1];
  const int t = blockIdx.z, k0 = blockIdx.x * RT, j0 = blockIdx.y * RT;
  const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
  const Cx<R>* Xt = X + (size_t)t * n * m;
  const double2* C = Cm + (size_t)t * m * m;
  Cx<A> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = cx<A>(0, 0);
  for (int l0 = 0; l0 < m; l0 += RL) {
#pragma unroll
    for (int q = 0; q < (RT * RL) / 256; q++) {
      const int e = tid + 256 * q;
      const int r = e / RL, c = e % RL;
      const int k = k0 + r, l = l0 + c;
      xs[r][c] = (k < n && l < m) ? to_a<A>(Xt[(size_t)k * m + l]) : cx<A>(0, 0);
      const int r2 = e / RT, c2 = e % RT;
      const int l2 = l0 + r2, j2 = j0 + c2;
      double2 cv = (l2 < m && j2 < m) ? C[(size_t)l2 * m + j2] : make_double2(0, 0);
      cs[r2][c2] = cx<A>((A)cv.x, (A)cv.y);
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < RL; l++) {
      Cx<A> xv[4], cv[4];
#pragma unroll
      for (int a = 0; a < 4; a++) xv[a] = xs[tr + 16 * a][l];
#pragma unroll
      for (int b = 0; b < 4; b++) cv[b] = cs[l][tc + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) fma_acc(acc[a][b], xv[a], cv[b]);
    }
    __syncthreads();
  }
  Cx<R>* Zt = Z + (size_t)t * n * m;
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int k = k0 + tr + 16 * a, j = j0 + tc + 16 * b;
      if (k < n && j < m) Zt[(size_t)k * m + j] = to_s<R>(acc[a][b]);
    }
}

// residual norms res[t][j] = ||W_j - theta_j X_j||; optionally R = W - X Theta stored in FP32
template <class R>
__global__ void __launch_bounds__(256) k_resid(const Cx<R>* __restrict__ X, const Cx<R>* __restrict__ W,
                                               const double* __restrict__ theta, int n, int m, double* res,
                                               Cx<float>* Rout) {
  const int t = blockIdx.y;
  const int j = blockIdx.x * 32 + (threadIdx.x & 31), lane = threadIdx.x >> 5;
  R s = 0;   // in the block's precision (FP64 arithmetic is scarce next to an FP32 block)
  if (j < m) {
    const R th = (R)theta[(size_t)t * m + j];
    const size_t base = (size_t)t * n * m;
    for (int k = lane; k < n; k += 8) {
      const size_t idx = base + (size_t)k * m + j;
      const Cx<R> w = W[idx], x = X[idx];
      const R dx = w.re - th * x.re, dy = w.im - th * x.im;
      s += dx * dx + dy * dy;
      if (Rout) Rout[idx] = cx<float>((float)dx, (float)dy);
    }
  }
  __shared__ double red[8][33];
  red[lane][threadIdx.x & 31] = (double)s;
  __syncthreads();
  if (lane == 0 && j < m) {
    double tot = 0;
    for (int q = 0; q < 8; q++) tot += red[q][threadIdx.x];
    res[(size_t)t * m + j] = sqrt(tot);
  }
}

// Y64 = X64 + E32 / s[t][j]  (phase B filter output, column j divided by s_d(theta_j)).
// The division leaves the span, and so the Rayleigh-Ritz, unchanged, but keeps the
// columns of Y at unit scale: X s_d + E has columns from 1 down to 1 / rho, whose
// Gram matrix (condition number up to rho^2) would limit the FP64 Ritz vectors
// near the cut to a few 1e-10.  s_d(theta) >= 1 / rho > 0 on [theta_0, cut].
__global__ void k_combine(const Cx<double>* __restrict__ X, const Cx<float>* __restrict__ E,
                          const double* __restrict__ scol, size_t nm, int m, size_t total, Cx<double>* Y) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const unsigned e32 = (unsigned)e;           // total < 2^31 (checked with the block)
  const int j = (int)(e32 % (unsigned)m);
  const unsigned t = e32 / (unsigned)nm;
  const double sj = scol[t * m + j];
  const Cx<float> ev = E[e];
  const Cx<double> ed = cx<double>((double)ev.re, (double)ev.im);
  // a vanishing s_d (possible only when the cut is pushed below 12 on a block that
  // spans nearly the whole timeslice) keeps the unscaled column
  Y[e] = fabs(sj) > 1e-280 ? X[e] + (1.0 / sj) * ed : sj * X[e] + ed;
}

template <class A, class B> __global__ void k_convert_block(const Cx<A>* in, Cx<B>* out, size_t total) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) out[e] = cx<B>((B)in[e].re, (B)in[e].im);
}

// counter-based start vectors: splitmix64 of (seed, index) -> two uniforms in (-1, 1)
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__global__ void k_random(Cx<float>* X, size_t count, uint64_t seed) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const uint64_t h = splitmix64(seed ^ splitmix64(e));
  const double a = (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  const uint64_t h2 = splitmix64(h);
  const double b = (double)(h2 >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  X[e] = cx<float>((float)a, (float)b);
}

// columns whose Ritz value is marked dropped (>= 1e299) get fresh random entries
template <class R>
__global__ void k_refill(Cx<R>* X, const double* theta, int n, int m, size_t total, uint64_t seed) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int j = e % m;
  const size_t t = e / ((size_t)n * m);
  if (theta[t * m + j] < 1e299) return;
  const uint64_t h = splitmix64(seed ^ splitmix64(e));
  const uint64_t h2 = splitmix64(h);
  X[e] = cx<R>((R)((double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0),
               (R)((double)(h2 >> 11) * (2.0 / 9007199254740992.0) - 1.0));
}

// first N columns of the block -> out [Tn][N][Vs][3] (cache_layout: [N][T][Vs][3] at timeslice t0 + t)
__global__ void k_extract(const Cx<double>* X, int n, int Tn, int m, int N, double2* out, int cache_layout, int T,
                          int t0) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)N * Tn * n;
  if (e >= total) return;
  const size_t r = e % n;
  const size_t rest = e / n;
  const int k = rest % N;
  const int t = rest / N;
  const Cx<double> v = X[((size_t)t * n + r) * m + k];
  const size_t o = cache_layout ? ((size_t)k * T + t0 + t) * n + r : ((size_t)t * N + k) * n + r;
  out[o] = make_double2(v.re, v.im);
}

// the original per-vector layout ([nvec][V][3]) for dlma_apply_laplacian
__global__ void k_lap_canonical(Geom g, const double2* __restrict__ U3, const double2* __restrict__ in, double2* out,
                                int nvec) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (s >= g.V || j >= nvec) return;
  const int x = s % g.L, y = (s / g.L) % g.L, z = (s / (g.L * g.L)) % g.L, t = s / g.Vs;
  const Coord c{x, y, z, t};
  const double2* v = in + (size_t)j * g.V * 3;
  Cx<double> acc[3];
  for (int a = 0; a < 3; a++) {
    const double2 e = v[(size_t)s * 3 + a];
    acc[a] = cx<double>(-6.0 * e.x, -6.0 * e.y);
  }
  for (int k = 0; k < 3; k++) {
    const int nf = nbr_lex(g, c, k + 1, +1), nb = nbr_lex(g, c, k + 1, -1);
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        const double2 uf = U3[((size_t)k * 9 + a * 3 + b) * g.V + s];
        const double2 ub = U3[((size_t)k * 9 + b * 3 + a) * g.V + nb];
        const double2 vf = v[(size_t)nf * 3 + b], vb = v[(size_t)nb * 3 + b];
        fma_acc(acc[a], cx<double>(uf.x, uf.y), cx<double>(vf.x, vf.y));
        fma_conj_acc(acc[a], cx<double>(ub.x, ub.y), cx<double>(vb.x, vb.y));
      }
  }
  double2* o = out + (size_t)j * g.V * 3;
  for (int a = 0; a < 3; a++) o[(size_t)s * 3 + a] = make_double2(acc[a].re, acc[a].im);
}

}  // namespace

// ---------------------------------------------------------------------------
struct Eig {
  dlma_ctx* ctx;
  int t0, Tn, N, m, n, nsplit, degree;
  int df = 0;   // phase B: Gram matrices and rotations in double-float (tol >= 1e-11)
  int tc = 0;   // phase B: Gram matrices and rotations on the tensor cores (tcproj.cu)
  size_t blk;                    // m * Tn * n complex entries per block
  Cx<float> *F0, *F1, *F2, *F3;  // FP32 blocks
  Cx<double> *D0, *D1, *D2;      // FP64 blocks
  double2 *G, *H, *C, *part, *gwork;
  double *theta, *res, *coef, *scol;
  int* dropped;                  // [0] dropped directions of the last small_rr, [1 + 2t + {0,1}] Jacobi sweeps
  bool refilled = false;         // the last fetch refilled dropped columns
  PhaseTimer* pt = nullptr;      // phases: kPhMatvec, kPhOrtho, kPhHost
  double drop_rel;
  uint64_t refill_seed;
  std::vector<double> th, rs;
};

// timing slots of dlma_laplacian_eigs (Table 2's split of the eigensolver time):
// Laplacian applications, orthogonalisation (Gram matrices, small eigenproblems,
// rotations, residuals, block conversions), host-side steps and transfers
constexpr int kPhMatvec = 3, kPhOrtho = 4, kPhHost = 5;
static inline void phase(Eig& E, int p) {
  if (E.pt) E.pt->enter(p);
}

template <class R> static const typename LinkT<R>::T* links(dlma_ctx* ctx);
template <> const double2* links<double>(dlma_ctx* ctx) { return ctx->U3; }
template <> const float4* links<float>(dlma_ctx* ctx) { return ctx->U3f; }

template <class R>
static dlma_status lap(Eig& E, const Cx<R>* in, const Cx<R>* prev, const Cx<float>* rin, const double* scol,
                       Cx<R>* out, const double* coef) {
  dlma_ctx* ctx = E.ctx;
  const size_t total = (size_t)E.Tn * ctx->g.Vs * E.m;
  if (total >= (1ull << 31)) return set_err(ctx, DLMA_ERR_INVALID_ARG, "eigensolver block above 2^31 entries");
  phase(E, kPhMatvec);
  // m is even; FP32: two columns per thread (one 128-bit access per pair, links
  // rebuilt once per pair); FP64 is bound by its arithmetic and keeps one
  // (measured alternatives: four FP32 columns per thread, 145 registers, and a
  // double-float FP64 matvec, 170 registers and a split of every loaded value,
  // were both slower)
  if constexpr (sizeof(R) == 4) {
    k_lap<R, R, 2><<<(unsigned)((total / 2 + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->g, E.t0, E.Tn, E.m, links<R>(ctx), in, prev, rin, scol, out, coef);
  } else {
    k_lap<R, R, 1><<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(ctx->g, E.t0, E.Tn, E.m, links<R>(ctx), in,
                                                                             prev, rin, scol, out, coef);
  }
  CHECK_LAUNCH();
  return DLMA_OK;
}

// out = X^dag Y per timeslice; herm = 1 when the result is hermitian by construction
template <class R> static dlma_status gram(Eig& E, const Cx<R>* X, const Cx<R>* Y, double2* out, int herm) {
  dlma_ctx* ctx = E.ctx;
  const int tj = (E.m + GT - 1) / GT;
  const int tiles = herm ? tj * (tj + 1) / 2 : tj * tj;
  phase(E, kPhOrtho);
  const dim3 grid(tiles, E.nsplit, E.Tn);
  if constexpr (sizeof(R) == 8) {
    if (E.tc)   // G[t][i][j] = sum_k conj(X[k][i]) Y[k][j]: rows = columns of Y, modes = columns of X
      return tc_block_product(ctx, 1, (const double2*)Y, (size_t)E.n * E.m, 1, (size_t)E.m, E.m,
                              (const double2*)X, 0, E.m, E.n, E.Tn, out);
    if (E.df) k_gram<R, df><<<grid, 256, 0, ctx->stream>>>(X, Y, E.n, E.m, E.nsplit, herm, E.part);
    else k_gram<R, R><<<grid, 256, 0, ctx->stream>>>(X, Y, E.n, E.m, E.nsplit, herm, E.part);
  } else {
    k_gram<R, R><<<grid, 256, 0, ctx->stream>>>(X, Y, E.n, E.m, E.nsplit, herm, E.part);
  }
  CHECK_LAUNCH();
  const size_t tot = (size_t)E.m * E.m * E.Tn;
  k_gram_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(E.part, E.nsplit, E.m, E.Tn, herm, out);
  CHECK_LAUNCH();
  return DLMA_OK;
}

template <class R> static dlma_status rotate(Eig& E, const Cx<R>* X, Cx<R>* Z) {
  dlma_ctx* ctx = E.ctx;
  phase(E, kPhOrtho);
  const dim3 grid((E.n + RT - 1) / RT, (E.m + RT - 1) / RT, E.Tn);
  if constexpr (sizeof(R) == 8) {
    if (E.tc)   // Z[t][k][j] = sum_l X[k][l] C[l][j]: rows = rows of X, modes = conj of the columns of C
      return tc_block_product(ctx, 2, (const double2*)X, (size_t)E.n * E.m, (size_t)E.m, 1, E.n, E.C, 1, E.m, E.m,
                              E.Tn, (double2*)Z);
    if (E.df) k_rotate<R, df><<<grid, 256, 0, ctx->stream>>>(X, E.C, E.n, E.m, Z);
    else k_rotate<R, R><<<grid, 256, 0, ctx->stream>>>(X, E.C, E.n, E.m, Z);
  } else {
    k_rotate<R, R><<<grid, 256, 0, ctx->stream>>>(X, E.C, E.n, E.m, Z);
  }
  CHECK_LAUNCH();
  return DLMA_OK;
}

// small Rayleigh-Ritz problems in precision T (float in phase A, double in phase B).
// The orthonormalisation tries the Cholesky route first in both phases; a pivot
// below the precision's floor (an ill-conditioned Gram matrix, as the unscaled
// phase-A block can have) falls back to the Jacobi route inside the kernel.
template <class T> static dlma_status small_rr(Eig& E) {
  dlma_ctx* ctx = E.ctx;
  size_t sm = 0;
  const int place = small_rr_place<T>(E.m, &sm);
  phase(E, kPhOrtho);
  if (sm) CU(cudaFuncSetAttribute(k_small_rr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  CU(cudaMemsetAsync(E.dropped, 0, sizeof(int), ctx->stream));
  const int chol = 1;
  k_small_rr<T><<<E.Tn, 1024, sm, ctx->stream>>>(E.G, E.H, E.m, E.C, E.theta, (Cx<T>*)E.gwork, place, E.dropped,
                                                 E.drop_rel, chol);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// Rayleigh-Ritz of the block Y: W = A Y, then X <- Y C, AX <- W C, residuals (and R = AX - X Theta in FP32)
template <class R>
static dlma_status rayleigh_ritz(Eig& E, Cx<R>* Y, Cx<R>* W, Cx<R>* Xout, Cx<R>* AXout, Cx<float>* Rout,
                                 const double* coef_plain) {
  TRY(lap<R>(E, Y, nullptr, nullptr, nullptr, W, coef_plain));
  TRY(gram<R>(E, Y, Y, E.G, 1));
  TRY(gram<R>(E, Y, W, E.H, 1));
  TRY(small_rr<R>(E));
  TRY(rotate<R>(E, Y, Xout));
  TRY(rotate<R>(E, W, AXout));
  dlma_ctx* ctx = E.ctx;
  phase(E, kPhOrtho);
  k_resid<R><<<dim3((E.m + 31) / 32, E.Tn), 256, 0, ctx->stream>>>(Xout, AXout, E.theta, E.n, E.m, E.res, Rout);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// fetch theta / residuals; returns the worst relative residual over the wanted pairs.
// Dropped directions (buffer columns that fell below the block's rounding level)
// are refilled with random entries in X and get the largest finite Ritz value of
// their timeslice on the host, so the filter's cut stays finite.
template <class R> static dlma_status fetch(Eig& E, double* worst, Cx<R>* X) {
  dlma_ctx* ctx = E.ctx;
  const size_t cnt = (size_t)E.m * E.Tn;
  phase(E, kPhHost);
  CU(cudaMemcpyAsync(E.th.data(), E.theta, sizeof(double) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(E.rs.data(), E.res, sizeof(double) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
  int hdrop = 0;
  CU(cudaMemcpyAsync(&hdrop, E.dropped, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (E.pt) E.pt->collect();
  E.refilled = hdrop != 0;
  if (hdrop) {
    phase(E, kPhOrtho);
    k_refill<R><<<(unsigned)((E.blk + 255) / 256), 256, 0, ctx->stream>>>(X, E.theta, E.n, E.m, E.blk,
                                                                         E.refill_seed++);
    CHECK_LAUNCH();
    for (int t = 0; t < E.Tn; t++) {
      double mx = 0;
      for (int j = 0; j < E.m; j++) {
        const double v = E.th[(size_t)t * E.m + j];
        if (v < 1e299) mx = std::max(mx, v);
      }
      for (int j = 0; j < E.m; j++) {
        double& v = E.th[(size_t)t * E.m + j];
        if (v >= 1e299) { v = mx; E.rs[(size_t)t * E.m + j] = 1.0; }
      }
    }
  }
  double w = 0;
  for (int t = 0; t < E.Tn; t++)
    for (int k = 0; k < E.N; k++) {
      const double r = E.rs[(size_t)t * E.m + k] / std::max(1.0, fabs(E.th[(size_t)t * E.m + k]));
      if (!(r == r)) return set_err(ctx, DLMA_ERR_NONFINITE, "NaN in the eigensolver");
      w = std::max(w, r);
    }
  *worst = w;
  return DLMA_OK;
}

// largest degree (<= dmax) whose amplification across [theta_0, cut] stays below rho on every timeslice
static int safe_degree(const Eig& E, double rho, int dmax) {
  int d = dmax;
  for (int t = 0; t < E.Tn; t++) {
    double a = E.th[(size_t)t * E.m + E.m - 1], a0 = E.th[(size_t)t * E.m];
    const double b = 12.0;
    if (a >= b) a = 0.5 * (a0 + b);
    const double e = 0.5 * (b - a), c = 0.5 * (b + a);
    const double x0 = (c - a0) / e;
    if (x0 > 1.0) d = std::min(d, (int)(acosh(rho) / acosh(x0)));
  }
  return std::max(d, 2);
}

// Chebyshev coefficients of every step (scaled three-term recurrence damping [cut_t, 12],
// normalised at lam0_t): slot 0 = first step, slot k-1 = step k; slot `degree` = plain A.
// With s_k(theta) (the scalar recurrence at each Ritz value) when scol != nullptr.
static void cheb_coefficients(Eig& E, int d, std::vector<double>& hc, std::vector<double>* hs) {
  const int Tn = E.Tn, m = E.m;
  hc.assign((size_t)(E.degree + 1) * 3 * Tn, 0.0);
  if (hs) hs->assign((size_t)(E.degree + 1) * Tn * m, 0.0);
  for (int t = 0; t < Tn; t++) {
    double a = E.th[(size_t)t * m + m - 1], a0 = E.th[(size_t)t * m];
    const double b = 12.0;
    if (a >= b) a = 0.5 * (a0 + b);
    const double e = 0.5 * (b - a), c = 0.5 * (b + a);
    double sigma = e / (a0 - c);
    const double tau = 2.0 / sigma;
    double* c0 = &hc[3 * t];
    c0[0] = sigma / e;
    c0[1] = -c * sigma / e;
    c0[2] = 0.0;
    std::vector<double> sp(m, 1.0), sc(m);
    for (int j = 0; j < m; j++) sc[j] = c0[0] * E.th[(size_t)t * m + j] + c0[1];
    if (hs) {
      for (int j = 0; j < m; j++) (*hs)[(size_t)t * m + j] = 1.0;                    // s_0
      for (int j = 0; j < m; j++) (*hs)[(size_t)Tn * m + (size_t)t * m + j] = sc[j];  // s_1
    }
    for (int k = 2; k <= d; k++) {
      const double sn = 1.0 / (tau - sigma);
      double* ck = &hc[(size_t)(k - 1) * 3 * Tn + 3 * t];
      ck[0] = 2.0 * sn / e;
      ck[1] = -2.0 * c * sn / e;
      ck[2] = -sigma * sn;
      sigma = sn;
      for (int j = 0; j < m; j++) {
        const double th = E.th[(size_t)t * m + j];
        const double nv = ck[0] * th * sc[j] + ck[1] * sc[j] + ck[2] * sp[j];
        sp[j] = sc[j];
        sc[j] = nv;
        if (hs) (*hs)[(size_t)k * Tn * m + (size_t)t * m + j] = nv;
      }
    }
    double* cd = &hc[(size_t)E.degree * 3 * Tn + 3 * t];   // slot of the plain A application
    cd[0] = 1;
    cd[1] = 0;
    cd[2] = 0;
  }
}

static dlma_status eig_batch(dlma_ctx* ctx, int t0, int Tn, int N, double tol, double* lam_out,
                             Cx<double>** Xres, int* m_out, int* iters_out, PhaseTimer* pt) {
  Eig E;
  E.ctx = ctx;
  E.pt = pt;
  E.t0 = t0;
  E.Tn = Tn;
  E.N = N;
  E.n = 3 * ctx->g.Vs;
  int buf = std::max(16, std::min(N, 64));
  int m = N + buf;
  m += m & 1;
  if (m > E.n) m = E.n - (E.n & 1);
  if (m < N) return set_err(ctx, DLMA_ERR_INVALID_ARG, "N too large for the timeslice");
  if (m > kSmallMaxM - 2)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "N + buffer above the eigensolver's limit of %d", kSmallMaxM - 2);
  E.m = m;
  E.degree = 40;            // largest filter degree (phase B); phase A stays below 20
  E.blk = (size_t)m * Tn * E.n;
  if (E.blk >= (1ull << 31)) return set_err(ctx, DLMA_ERR_INVALID_ARG, "eigensolver block above 2^31 entries");
  E.nsplit = std::max(1, std::min(64, (4 * 152) / std::max(1, Tn * ((m + GT - 1) / GT) * ((m + GT - 1) / GT))));
  E.nsplit = std::min(E.nsplit, std::max(1, E.n / 256));
  TRY(workT(ctx, WS_EIG_X, E.blk * 2, &E.F0));
  E.F1 = E.F0 + E.blk;
  TRY(workT(ctx, WS_EIG_Y, E.blk * 2, &E.F2));
  E.F3 = E.F2 + E.blk;
  TRY(workT(ctx, WS_EIG_Y2, E.blk, &E.D0));
  TRY(workT(ctx, WS_EIG_W, E.blk * 2, &E.D1));
  E.D2 = E.D1 + E.blk;
  const size_t mm = (size_t)m * m;
  TRY(workT(ctx, WS_EIG_G, 3 * mm * Tn, &E.G));
  E.H = E.G + mm * Tn;
  E.C = E.H + mm * Tn;
  TRY(workT(ctx, WS_EIG_PART, (size_t)E.nsplit * mm * Tn, &E.part));
  TRY(workT(ctx, WS_EIG_S, 3 * (size_t)m * (m + 1) * Tn, &E.gwork));
  const int d = E.degree;
  double* aux;
  const size_t ncoef = (size_t)(d + 1) * 3 * Tn, nscol = (size_t)(d + 1) * Tn * m;
  TRY(workT(ctx, WS_EIG_AUX, 2 * (size_t)m * Tn + ncoef + nscol + Tn + 16, &aux));
  E.theta = aux;
  E.res = aux + (size_t)m * Tn;
  E.coef = E.res + (size_t)m * Tn;
  E.scol = E.coef + ncoef;
  E.dropped = (int*)(E.scol + nscol);
  E.th.resize((size_t)m * Tn);
  E.rs.resize((size_t)m * Tn);
  E.drop_rel = 1e-10;
  E.refill_seed = 0x7e11ULL + (uint64_t)t0;
  std::vector<double> hc, hs;
  // plain A for the Rayleigh-Ritz W = A Y: coefficient slot d
  hc.assign(ncoef, 0.0);
  for (int t = 0; t < Tn; t++) hc[(size_t)d * 3 * Tn + 3 * t] = 1.0;
  phase(E, kPhHost);
  CU(cudaMemcpyAsync(E.coef, hc.data(), sizeof(double) * ncoef, cudaMemcpyHostToDevice, ctx->stream));
  const double* plain = E.coef + (size_t)d * 3 * Tn;

  // ---- phase A: FP32 ----
  phase(E, kPhOrtho);
  k_random<<<(unsigned)((E.blk + 255) / 256), 256, 0, ctx->stream>>>(E.F1, E.blk, 0x5eed2022ULL + (uint64_t)t0 * 7919ULL);
  CHECK_LAUNCH();
  // three FP32 blocks rotate: p3[0] = Ritz vectors X, p3[1], p3[2] free; F3 holds A X
  Cx<float>* p3[3] = {E.F0, E.F1, E.F2};
  TRY(rayleigh_ritz<float>(E, p3[1], p3[2], p3[0], E.F3, nullptr, plain));
  double worst = 1;
  int it = 0;
  const int maxA = 60, maxB = 40;
  const double switch_tol = std::max(tol, 3e-6);
  double prev_worst = 1e300;
  E.drop_rel = 1e-10;       // FP32 block: Gram eigenvalues below ~1e-10 gmax are rounding noise
  for (; it < maxA; it++) {
    TRY(fetch<float>(E, &worst, p3[0]));
    if (worst <= switch_tol) break;
    // single precision has stopped paying off: hand over to the FP64 phase
    if (it >= 3 && worst > 0.5 * prev_worst) break;
    prev_worst = worst;
    // FP32 filter: keep the amplification across [theta_0, cut] below ~300 so the
    // filtered block stays resolvable in single precision
    const int dA = safe_degree(E, 300.0, 20);
    cheb_coefficients(E, dA, hc, nullptr);
    phase(E, kPhHost);
    CU(cudaMemcpyAsync(E.coef, hc.data(), sizeof(double) * ncoef, cudaMemcpyHostToDevice, ctx->stream));
    Cx<float>*prev = p3[0], *cur = p3[1], *nxt = p3[2];
    TRY(lap<float>(E, prev, nullptr, nullptr, nullptr, cur, E.coef));
    for (int k = 2; k <= dA; k++) {
      TRY(lap<float>(E, cur, prev, nullptr, nullptr, nxt, E.coef + (size_t)(k - 1) * 3 * Tn));
      Cx<float>* t = prev;
      prev = cur;
      cur = nxt;
      nxt = t;
    }
    // cur holds the filtered block; prev and nxt are free (one of them held X)
    TRY(rayleigh_ritz<float>(E, cur, prev, nxt, E.F3, nullptr, plain));
    p3[0] = nxt;
    p3[1] = cur;
    p3[2] = prev;
  }
  Cx<float>* X = p3[0];
  // ---- phase B: FP64 Ritz vectors, FP32 residual-driven filter ----
  // The FP64 blocks' Gram matrices and rotations run in double-float on the FP32
  // units when the tolerance leaves room for its ~2^-46 rounding.
  E.df = ctx->df_eigs && tol >= 1e-11;
  // products of many multiply-adds (n m^2 per timeslice) take the tensor cores
  // (16^3 x 32: orthogonalisation 250 -> 200 ms at N = 64, 617 -> 533 ms at N = 128;
  // 32^3 x 64, N = 96: 5.4 -> 4.4 s); small ones stay in double-float, where the
  // tensor-core launches do not fill the GPU (16^3 x 32, N = 32: 65 against 70 ms).
  // DLMA_EIGS_TC=1 / 0 forces either.
  E.tc = E.df && (double)E.n * E.m * E.m * E.Tn >= 4.0e9;
  if (const char* e = getenv("DLMA_EIGS_TC")) E.tc = E.df && atoi(e) == 1;
  Cx<double> *X64 = E.D0, *W64 = E.D1, *Y64 = E.D2;
  // phase A's last Ritz pairs were not fetched, or hold refilled (random) columns
  const bool rr_first = E.refilled || it >= maxA;
  phase(E, kPhOrtho);
  k_convert_block<float, double><<<(unsigned)((E.blk + 255) / 256), 256, 0, ctx->stream>>>(X, rr_first ? Y64 : X64,
                                                                                           E.blk);
  CHECK_LAUNCH();
  Cx<float>* R32 = E.F3;   // residual R = AX - X Theta
  Cx<float>* Ebuf[3];
  {
    int q = 0;
    Cx<float>* all[4] = {E.F0, E.F1, E.F2, E.F3};
    for (int i = 0; i < 4; i++)
      if (all[i] != R32) Ebuf[q++] = all[i];
  }
  // The filter below needs only R32 = A X - X Theta for the current X and Theta, which
  // hold for phase A's Ritz pairs as they stand: X64 = X, Y64 = A X64, R32.  After a
  // refill the block is first re-diagonalised in FP64.
  E.drop_rel = 1e-24;
  if (rr_first) {
    TRY(rayleigh_ritz<double>(E, Y64, W64, X64, Y64, R32, plain));
  } else {
    TRY(lap<double>(E, X64, nullptr, nullptr, nullptr, Y64, plain));
    phase(E, kPhOrtho);
    k_resid<double><<<dim3((m + 31) / 32, Tn), 256, 0, ctx->stream>>>(X64, Y64, E.theta, E.n, m, E.res, R32);
    CHECK_LAUNCH();
  }
  bool conv = false;
  int itB = 0;
  int dB = d;
  for (; itB < maxB; itB++) {
    TRY(fetch<double>(E, &worst, X64));
    if (worst <= tol) { conv = true; break; }
    dB = safe_degree(E, 1e6, d);
    cheb_coefficients(E, dB, hc, &hs);
    phase(E, kPhHost);
    CU(cudaMemcpyAsync(E.coef, hc.data(), sizeof(double) * ncoef, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(E.scol, hs.data(), sizeof(double) * nscol, cudaMemcpyHostToDevice, ctx->stream));
    // E_1 = a_1 R s_0 ; E_{k+1} = a_k A E_k + b_k E_k + c_k E_{k-1} + a_k R s_k
    Cx<float>*em = nullptr, *ec = Ebuf[0], *en = Ebuf[1], *spare = Ebuf[2];
    TRY(lap<float>(E, nullptr, nullptr, R32, E.scol, ec, E.coef));
    for (int k = 2; k <= dB; k++) {
      TRY(lap<float>(E, ec, em, R32, E.scol + (size_t)(k - 1) * Tn * m, en, E.coef + (size_t)(k - 1) * 3 * Tn));
      Cx<float>* t = em ? em : spare;
      em = ec;
      ec = en;
      en = t;
    }
    // Y = (X s_d + E_d) / s_d column by column
    phase(E, kPhOrtho);
    k_combine<<<(unsigned)((E.blk + 255) / 256), 256, 0, ctx->stream>>>(X64, ec, E.scol + (size_t)dB * Tn * m,
                                                                        (size_t)E.n * m, m, E.blk, Y64);
    CHECK_LAUNCH();
    // Rayleigh-Ritz of Y64: W64 = A Y64; X64 <- Y64 C; AX into W... (use X64 as output: Y64 and W64 are inputs)
    TRY(lap<double>(E, Y64, nullptr, nullptr, nullptr, W64, plain));
    TRY(gram<double>(E, Y64, Y64, E.G, 1));
    TRY(gram<double>(E, Y64, W64, E.H, 1));
    TRY(small_rr<double>(E));
    TRY(rotate<double>(E, Y64, X64));
    TRY(lap<double>(E, X64, nullptr, nullptr, nullptr, Y64, plain));   // A X, fresh (cheaper than W C)
    phase(E, kPhOrtho);
    k_resid<double><<<dim3((m + 31) / 32, Tn), 256, 0, ctx->stream>>>(X64, Y64, E.theta, E.n, m, E.res, R32);
    CHECK_LAUNCH();
  }
  if (!conv) {
    TRY(fetch<double>(E, &worst, X64));
    conv = worst <= tol;
  }
  if (!conv)
    return set_err(ctx, DLMA_ERR_NOT_CONVERGED, "eigensolver at %.3g, not %.3g, after %d + %d iterations", worst, tol,
                   it, itB);
  for (int t = 0; t < Tn; t++)
    for (int k = 0; k < N; k++) lam_out[(size_t)t * N + k] = E.th[(size_t)t * m + k];
  *Xres = X64;
  *m_out = m;
  if (iters_out) { iters_out[0] = it; iters_out[1] = itB; }
  return DLMA_OK;
}

extern "C" dlma_status dlma_apply_laplacian(dlma_ctx* ctx, const double* in, double* out, int nvec, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge) return set_err(ctx, DLMA_ERR_STATE, "no gauge field");
  if (!in || !out || nvec < 1) return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument");
  CU(cudaSetDevice(ctx->device));
  const size_t bytes = (size_t)nvec * ctx->g.V * 3 * 16;
  const double* din;
  TRY(copy_in(ctx, WS_IN, in, bytes, mem, &din));
  double* dout = out;
  if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_OUT, bytes / 8, &dout));
  dim3 grid((ctx->g.V + 127) / 128, nvec);
  k_lap_canonical<<<grid, 128, 0, ctx->stream>>>(ctx->g, ctx->U3, (const double2*)din, (double2*)dout, nvec);
  CHECK_LAUNCH();
  TRY(copy_out(ctx, out, dout, bytes, mem));
  CU(cudaStreamSynchronize(ctx->stream));
  return DLMA_OK;
}

extern "C" dlma_status dlma_laplacian_eigs(dlma_ctx* ctx, int t, int N, double tol, double* evals, double* evecs,
                                           dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge) return set_err(ctx, DLMA_ERR_STATE, "no gauge field");
  if (!evals || N < 1 || t < -1 || t >= ctx->g.T || !(tol > 0) || N > 3 * ctx->g.Vs / 2)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_laplacian_eigs");
  CU(cudaSetDevice(ctx->device));
  const int t0 = t < 0 ? 0 : t, Tn = t < 0 ? ctx->g.T : 1;
  const int n = 3 * ctx->g.Vs;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, ctx->stream));
  Cx<double>* X = nullptr;
  int m = 0, iters[2] = {0, 0};
  PhaseTimer pt(ctx->stream);
  pt.enter(kPhHost);
  dlma_status st = eig_batch(ctx, t0, Tn, N, tol, evals, &X, &m, iters, &pt);
  if (st != DLMA_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
  }
  pt.enter(kPhHost);
  ctx->eig_gen++;
  if (ctx->eig_N != N || !ctx->eig_V) {
    if (ctx->eig_V) cudaFree(ctx->eig_V);
    ctx->eig_V = nullptr;
    ctx->eig_N = 0;
    CU(cudaMalloc(&ctx->eig_V, (size_t)N * ctx->g.T * n * sizeof(double2)));
    ctx->eig_lam.assign((size_t)N * ctx->g.T, 0.0);
    ctx->eig_have.assign(ctx->g.T, 0);
    ctx->eig_N = N;
  }
  const size_t tot = (size_t)N * Tn * n;
  k_extract<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(X, n, Tn, m, N, ctx->eig_V, 1, ctx->g.T, t0);
  CHECK_LAUNCH();
  for (int tt = 0; tt < Tn; tt++) {
    ctx->eig_have[t0 + tt] = 1;
    for (int k = 0; k < N; k++) ctx->eig_lam[(size_t)(t0 + tt) * N + k] = evals[(size_t)tt * N + k];
  }
  if (evecs) {
    const size_t bytes = tot * sizeof(double2);
    double2* dst = (double2*)evecs;
    if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_OUT, tot, &dst));
    k_extract<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(X, n, Tn, m, N, dst, 0, ctx->g.T, t0);
    CHECK_LAUNCH();
    if (mem == DLMA_MEM_HOST) TRY(copy_out(ctx, evecs, (const double*)dst, bytes, mem));
  }
  CU(cudaEventRecord(e1, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  pt.mark(-1);
  CU(cudaStreamSynchronize(ctx->stream));
  pt.collect();
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  for (int i = 0; i < kTimingSlots; i++) ctx->timing[i] = 0;
  ctx->timing[0] = ms;
  ctx->timing[1] = iters[0];
  ctx->timing[2] = iters[1];
  ctx->timing[kPhMatvec] = pt.acc[kPhMatvec];
  ctx->timing[kPhOrtho] = pt.acc[kPhOrtho];
  ctx->timing[kPhHost] = pt.acc[kPhHost];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return DLMA_OK;
}
