// Small dense Rayleigh-Ritz problems of the Laplacian eigensolver, one CTA per
// timeslice: from G = Y^dag Y and H = Y^dag A Y (m x m, hermitian) produce C
// such that Y C are orthonormal Ritz vectors with ascending Ritz values.
//
//   G = Q diag(g) Q^dag (Jacobi),  S = Q diag(g)^-1/2 (directions with tiny g dropped),
//   S^dag H S = Z diag(theta) Z^dag (Jacobi),  C = S Z sorted by theta.
//
// With chol = 1 the orthonormalising S comes from the Cholesky factor instead,
// G = R^dag R, S = R^-1 (about 2 m^3 / 3 operations against three times that per
// Jacobi sweep): for a well-conditioned G, as the FP64 phase of the eigensolver
// produces, it replaces the first Jacobi solve; a pivot at or below the rounding
// level of the largest diagonal falls back to the Jacobi route (the FP32 phase
// tries it too and falls back whenever its block is ill-conditioned).
//
// The eigendecompositions use the parallel cyclic Jacobi method (round-robin
// pairing, m/2 disjoint complex rotations per round).  T = float serves the
// single-precision phase of the eigensolver, T = double its final phase, where
// both matrices arrive nearly diagonal and Jacobi needs two or three sweeps.
#pragma once
#include "common.cuh"

// a pair (p, q) is rotated only if |a_pq| > eps sqrt(|a_pp a_qq|): below that the
// entry is at the rounding level of the precision; a sweep without any rotation ends
// the iteration (the classical threshold Jacobi method)
template <class T> struct SmallPrec;
template <> struct SmallPrec<float> { static constexpr float eps = 1e-6f; };
template <> struct SmallPrec<double> { static constexpr double eps = 1e-15; };

// largest block (columns per timeslice) the small problems take: m/2 rotation
// pairs and m sort keys live in static shared memory
constexpr int kSmallMaxM = 512;

__device__ __forceinline__ int rr_pos(int idx, int r, int m) { return idx == 0 ? 0 : ((idx - 1 + r) % (m - 1)) + 1; }

// Diagonalise the hermitian A [m][m] (row-major with leading dimension ld, in
// place), accumulating the rotations into the columns of V (which holds the
// initial basis).  ld = m + 1 keeps the column updates, where consecutive threads
// walk down a column, free of shared-memory bank conflicts.  Returns the number
// of sweeps.
template <class T>
__device__ int jacobi(Cx<T>* A, Cx<T>* V, int m, int ld, T* rc, T* rs, Cx<T>* re, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int np = m / 2;
  // thread layout of the row / column updates: rows i0 + l ni, pairs k0 + l nk (no
  // integer division per element)
  const int ni = m <= nt ? m : nt, nk = m <= nt ? nt / m : 1;
  const int i0 = tid % ni, k0 = tid / ni;
  const bool upd = k0 < nk;
  __shared__ int pq[2][kSmallMaxM / 2];
  __shared__ int rotated;
  __shared__ double dmax;
  if (tid == 0) {
    double mx = 0;
    for (int i = 0; i < m; i++) mx = fmax(mx, fabs((double)A[i * ld + i].re));
    dmax = mx;
  }
  __syncthreads();
  // entries below this absolute floor are rounding noise even next to tiny diagonals
  const T floor_abs = (T)(1e-4 * (double)SmallPrec<T>::eps * dmax);
  int sweep = 0;
  for (; sweep < 40; sweep++) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < m - 1; r++) {
      for (int k = tid; k < np; k += nt) {
        const int p = rr_pos(k, r, m), q = rr_pos(m - 1 - k, r, m);
        pq[0][k] = p;
        pq[1][k] = q;
        const T a = A[p * ld + p].re, d = A[q * ld + q].re;
        const Cx<T> b = A[p * ld + q];
        const T ab = sqrt(b.re * b.re + b.im * b.im);
        if (!(ab > SmallPrec<T>::eps * sqrt(fabs(a * d)) && ab > floor_abs && ab > (T)1e-300)) {
          rc[k] = 1; rs[k] = 0; re[k] = cx<T>(1, 0);
          continue;
        }
        rotated = 1;
        const T tau = (d - a) / (2 * ab);
        const T tt = (tau >= 0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt(1 + tau * tau));
        const T c = 1 / sqrt(1 + tt * tt);
        rc[k] = c;
        rs[k] = tt * c;
        re[k] = cx<T>(b.re / ab, -b.im / ab);   // e^{-i phi}
      }
      __syncthreads();
      if (upd)
        for (int k = k0; k < np; k += nk) {          // A <- A J, V <- V J (columns p, q)
          const T s = rs[k];
          if (s == (T)0) continue;                     // pair not rotated this round
          const int p = pq[0][k], q = pq[1][k];
          const T c = rc[k];
          const Cx<T> ph = re[k];
          for (int i = i0; i < m; i += ni) {
            const Cx<T> ap = A[i * ld + p], aq = ph * A[i * ld + q];
            A[i * ld + p] = c * ap - s * aq;
            A[i * ld + q] = s * ap + c * aq;
            const Cx<T> vp = V[i * ld + p], vq = ph * V[i * ld + q];
            V[i * ld + p] = c * vp - s * vq;
            V[i * ld + q] = s * vp + c * vq;
          }
        }
      __syncthreads();
      if (upd)
        for (int k = k0; k < np; k += nk) {          // A <- J^dag A (rows p, q)
          const T s = rs[k];
          if (s == (T)0) continue;
          const int p = pq[0][k], q = pq[1][k];
          const T c = rc[k];
          const Cx<T> ph = conj(re[k]);
          for (int j = i0; j < m; j += ni) {
            const Cx<T> ap = A[p * ld + j], aq = ph * A[q * ld + j];
            A[p * ld + j] = c * ap - s * aq;
            A[q * ld + j] = s * ap + c * aq;
          }
        }
      __syncthreads();
    }
    if (!rotated) break;      // every pair below the threshold: converged
    __syncthreads();
  }
  (void)red;
  return sweep + 1;
}

template <class T>
__global__ void __launch_bounds__(1024) k_small_rr(const double2* Gall, const double2* Hall, int m, double2* Call,
                                                  double* theta_all, Cx<T>* gwork, int use_smem, int* dropped,
                                                  double drop_rel, int chol = 0) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int t = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const size_t mm = (size_t)m * m;
  const int ld = m + 1;                  // padded rows of the work matrices
  const size_t ml = (size_t)m * ld;
  Cx<T>*S, *A, *Z;
  if (use_smem) { S = (Cx<T>*)sm_raw; A = S + ml; Z = A + ml; }
  else { S = gwork + 3 * ml * t; A = S + ml; Z = A + ml; }
  __shared__ T rc[kSmallMaxM / 2], rs[kSmallMaxM / 2];
  __shared__ Cx<T> re[kSmallMaxM / 2];
  __shared__ double red[512], lam[kSmallMaxM];
  __shared__ int order[kSmallMaxM];
  const double2* G = Gall + mm * t;
  const double2* H = Hall + mm * t;
  __shared__ int chol_ok;
  int sw_g = 0;
  if (chol) {
    // 1') Cholesky G = R^dag R (R upper, in A), right-looking, then S = R^-1 by columns
    for (size_t e = tid; e < mm; e += nt) A[(e / m) * ld + e % m] = cx<T>((T)G[e].x, (T)G[e].y);
    if (tid == 0) {
      double mx = 0;
      for (int i = 0; i < m; i++) mx = fmax(mx, G[(size_t)i * m + i].x);
      red[0] = mx;
      chol_ok = 1;
    }
    __syncthreads();
    const T floor_piv = (T)(1e4 * (double)SmallPrec<T>::eps * red[0]);
    for (int k = 0; k < m; k++) {
      if (tid == 0) {
        const T d = A[k * ld + k].re;
        if (!(d > floor_piv)) chol_ok = 0;
        A[k * ld + k] = cx<T>(sqrt(d > (T)0 ? d : (T)1), 0);
      }
      __syncthreads();
      if (!chol_ok) break;
      const T inv = (T)1 / A[k * ld + k].re;
      for (int j = k + 1 + tid; j < m; j += nt) A[k * ld + j] = inv * A[k * ld + j];    // row k of R
      __syncthreads();
      // trailing update: A[i][j] -= conj(R[k][i]) R[k][j] for k < i <= j
      const int rem = m - k - 1;
      for (int e = tid; e < rem * rem; e += nt) {
        const int i = k + 1 + e / rem, j = k + 1 + e % rem;
        if (j < i) continue;
        const Cx<T> rki = A[k * ld + i], rkj = A[k * ld + j];
        A[i * ld + j] = A[i * ld + j] - conj(rki) * rkj;
      }
      __syncthreads();
    }
    if (chol_ok) {
      // S = R^-1: column j by back substitution (S upper triangular)
      for (int j = tid; j < m; j += nt) {
        for (int i = m - 1; i >= 0; i--) {
          Cx<T> sum = cx<T>(i == j ? (T)1 : (T)0, 0);
          if (i <= j)
            for (int l = i + 1; l <= j; l++) sum = sum - A[i * ld + l] * S[l * ld + j];
          S[i * ld + j] = i <= j ? (T)1 / A[i * ld + i].re * sum : cx<T>(0, 0);
        }
      }
      __syncthreads();
      for (int i = tid; i < m; i += nt) lam[i] = 1.0;   // no direction dropped
      __syncthreads();
    }
  }
  if (!chol || !chol_ok) {
  // 1) eigen-decomposition of the Gram matrix
  for (size_t e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    A[i * ld + j] = cx<T>((T)G[e].x, (T)G[e].y);
    S[i * ld + j] = cx<T>(i == j ? (T)1 : (T)0, 0);
  }
  __syncthreads();
  sw_g = jacobi<T>(A, S, m, ld, rc, rs, re, red);
  // 2) S <- Q diag(g)^-1/2, dropping directions with g <= drop_rel gmax
  if (tid == 0) {
    double gmax = 0;
    for (int i = 0; i < m; i++) gmax = fmax(gmax, (double)A[i * ld + i].re);
    red[0] = gmax;
  }
  __syncthreads();
  const double gmax = red[0];
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    const double gi = A[i * ld + i].re;
    lam[i] = gi > drop_rel * gmax ? 1.0 / sqrt(gi) : 0.0;
  }
  __syncthreads();
  for (size_t e = tid; e < mm; e += nt) S[(e / m) * ld + e % m] = (T)lam[e % m] * S[(e / m) * ld + e % m];
  __syncthreads();
  }
  // 3) Z <- H S ; A <- S^dag Z  (= S^dag H S)
  for (size_t e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    Cx<T> s = cx<T>(0, 0);
    for (int l = 0; l < m; l++) fma_acc(s, cx<T>((T)H[i * m + l].x, (T)H[i * m + l].y), S[l * ld + j]);
    Z[i * ld + j] = s;
  }
  __syncthreads();
  for (size_t e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    Cx<T> s = cx<T>(0, 0);
    for (int l = 0; l < m; l++) fma_conj_acc(s, S[l * ld + i], Z[l * ld + j]);
    A[i * ld + j] = s;
  }
  __syncthreads();
  for (size_t e = tid; e < mm; e += nt) {   // hermitian part (round-off)
    const int i = e / m, j = e % m;
    if (i < j) {
      const Cx<T> a = A[i * ld + j], b = A[j * ld + i];
      const Cx<T> h = cx<T>((T)0.5 * (a.re + b.re), (T)0.5 * (a.im - b.im));
      A[i * ld + j] = h;
      A[j * ld + i] = conj(h);
    } else if (i == j) {
      A[i * ld + j].im = 0;
    }
  }
  for (size_t e = tid; e < mm; e += nt) Z[(e / m) * ld + e % m] = cx<T>((e / m) == (e % m) ? (T)1 : (T)0, 0);
  __syncthreads();
  const int sw_h = jacobi<T>(A, Z, m, ld, rc, rs, re, red);
  if (tid == 0) { dropped[1 + 2 * t] = sw_g; dropped[2 + 2 * t] = sw_h; }
  // 4) sort ascending.  A dropped direction i has an exactly zero row and column
  //    in S^dag H S, so Jacobi never rotates it and it keeps position i: sort it last.
  for (int i = tid; i < m; i += nt) lam[i] = lam[i] > 0 ? (double)A[i * ld + i].re : 1e300;
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    int rank = 0;
    for (int l = 0; l < m; l++) rank += (lam[l] < lam[i]) || (lam[l] == lam[i] && l < i);
    order[rank] = i;
  }
  __syncthreads();
  // 5) C = S Z[:, order]
  double2* Cout = Call + mm * t;
  for (size_t e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    const int zj = order[j];
    Cx<T> s = cx<T>(0, 0);
    for (int l = 0; l < m; l++) fma_acc(s, S[i * ld + l], Z[l * ld + zj]);
    Cout[e] = make_double2((double)s.re, (double)s.im);
  }
  for (int j = tid; j < m; j += nt) {
    const double v = lam[order[j]];
    theta_all[(size_t)t * m + j] = v;
    if (v > 1e299) atomicAdd(dropped, 1);
  }
}
