// Small dense Rayleigh-Ritz problems of the Laplacian eigensolver, one CTA per
// timeslice: from G = Y^dag Y and H = Y^dag A Y (m x m, hermitian) produce C
// such that Y C are orthonormal Ritz vectors with ascending Ritz values.
//
//   G = R^dag R (Cholesky), S = R^-1,  or for an ill-conditioned G
//   G = Q diag(g) Q^dag (Jacobi), S = Q diag(g)^-1/2 (directions with tiny g dropped);
//   S^dag H S = Z diag(theta) Z^dag (Jacobi),  C = S Z sorted by theta.
//
// The Cholesky route costs about 2 m^3 / 3 operations against three times that per
// Jacobi sweep; a pivot at or below the rounding level of the largest diagonal falls
// back to the Jacobi route (the FP32 phase of the eigensolver tries Cholesky too and
// falls back whenever its block is ill-conditioned).
//
// The eigendecompositions use the parallel cyclic Jacobi method (round-robin
// pairing, m/2 disjoint complex rotations per round).  T = float serves the
// single-precision phase of the eigensolver, T = double its final phase, where
// both matrices arrive nearly diagonal and Jacobi needs two or three sweeps.
//
// Storage.  A matrix being diagonalised is held as its packed upper triangle (row i
// holds columns i..m-1), S column-major.  One Jacobi round transforms every 2 x 2
// block of A — the rows of one rotation pair against the columns of another — in a
// single pass (A <- J^dag A J, no intermediate A J), and rotates the columns of S in
// the same pass, so the accumulated rotations never form a separate Z: S Z is S
// after the last round.  Packed A and S sit in shared memory when they fit (A first:
// it is on the dependent path of every round), else in the global work area.
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

// packed upper triangle of a hermitian m x m matrix: entry (i, j), i <= j, at
// i m - i (i - 1) / 2 + (j - i); the lower triangle is the conjugate
template <class T> struct Herm {
  Cx<T>* a;
  int m;
  __device__ __forceinline__ int off(int i, int j) const { return i * m - ((i * (i - 1)) >> 1) + (j - i); }
  __device__ __forceinline__ Cx<T> get(int i, int j) const { return i <= j ? a[off(i, j)] : conj(a[off(j, i)]); }
  __device__ __forceinline__ void set(int i, int j, Cx<T> v) const {
    if (i <= j) a[off(i, j)] = v;
    else a[off(j, i)] = conj(v);
  }
  __device__ __forceinline__ T diag(int i) const { return a[off(i, i)].re; }
};

// one complex rotation of the pair of values (x_p, x_q):
//   x_p <- c x_p - s e x_q,   x_q <- s x_p + c e x_q
// columns p, q of A J and of S J take e = e^{-i phi} (a_pq = |a_pq| e^{i phi}), rows
// p, q of J^dag A take conj(e)
template <class T> __device__ __forceinline__ void rot2(Cx<T>& xp, Cx<T>& xq, T c, T s, Cx<T> e) {
  const Cx<T> a = xp, b = e * xq;
  xp = c * a - s * b;
  xq = s * a + c * b;
}

// (k, i) = divmod(e, n) for e = e0 + l * step, advanced without a division per step
struct DivWalk {
  int q, r, dq, dr, n;
  __device__ __forceinline__ DivWalk(int e0, int step, int n_) : q(e0 / n_), r(e0 % n_), dq(step / n_), dr(step % n_), n(n_) {}
  __device__ __forceinline__ void next() {
    q += dq;
    r += dr;
    if (r >= n) { r -= n; q++; }
  }
};

// Diagonalise the hermitian A (packed, in place), applying every rotation to the
// columns of V (column-major, leading dimension ld, m rows), which holds the initial
// basis.  Returns the number of sweeps.
template <class T>
__device__ int jacobi(const Herm<T> A, Cx<T>* V, int ld, T* rc, T* rs, Cx<T>* re) {
  const int tid = threadIdx.x, nt = blockDim.x, m = A.m;
  const int np = m / 2;
  __shared__ int pp[kSmallMaxM / 2], qq[kSmallMaxM / 2];
  __shared__ int rotated;
  __shared__ double dmax;
  if (tid == 0) {
    double mx = 0;
    for (int i = 0; i < m; i++) mx = fmax(mx, fabs((double)A.diag(i)));
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
        pp[k] = p;
        qq[k] = q;
        const T a = A.diag(p), d = A.diag(q);
        const Cx<T> b = A.get(p, q);
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
      // A <- J^dag A J by 2 x 2 blocks: rows of pair ka, columns of pair kb, ka <= kb
      // (the blocks below the diagonal are their conjugate transposes)
      for (DivWalk w(tid, nt, np); w.q < np; w.next()) {
        const int ka = w.q, kb = w.r;
        if (ka > kb) continue;
        const T sa = rs[ka], sb = rs[kb];
        if (sa == (T)0 && sb == (T)0) continue;
        const int p1 = pp[ka], q1 = qq[ka], p2 = pp[kb], q2 = qq[kb];
        const T ca = rc[ka], cb = rc[kb];
        const Cx<T> ea = re[ka], eb = re[kb];
        if (ka == kb) {
          Cx<T> x00 = cx<T>(A.diag(p1), 0), x11 = cx<T>(A.diag(q1), 0), x01 = A.get(p1, q1);
          Cx<T> x10 = conj(x01);
          rot2(x00, x01, ca, sa, ea);             // columns
          rot2(x10, x11, ca, sa, ea);
          rot2(x00, x10, ca, sa, conj(ea));       // rows
          rot2(x01, x11, ca, sa, conj(ea));
          A.a[A.off(p1, p1)] = cx<T>(x00.re, 0);
          A.a[A.off(q1, q1)] = cx<T>(x11.re, 0);
          A.set(p1, q1, x01);
        } else {
          Cx<T> x00 = A.get(p1, p2), x01 = A.get(p1, q2), x10 = A.get(q1, p2), x11 = A.get(q1, q2);
          if (sb != (T)0) {
            rot2(x00, x01, cb, sb, eb);
            rot2(x10, x11, cb, sb, eb);
          }
          if (sa != (T)0) {
            rot2(x00, x10, ca, sa, conj(ea));
            rot2(x01, x11, ca, sa, conj(ea));
          }
          A.set(p1, p2, x00);
          A.set(p1, q2, x01);
          A.set(q1, p2, x10);
          A.set(q1, q2, x11);
        }
      }
      // V <- V J (columns p, q; consecutive threads on consecutive rows).  VB items
      // are loaded before any is stored (their columns are disjoint), so a V in global
      // memory costs one round trip per VB items, not per item
      {
        constexpr int VB = sizeof(T) == 4 ? 4 : 1;
        DivWalk w(tid, nt, m);
        while (w.q < np) {
          int op[VB], oq[VB], kk[VB];
          bool on[VB];
#pragma unroll
          for (int u = 0; u < VB; u++) {
            kk[u] = w.q;
            on[u] = w.q < np && rs[w.q] != (T)0;
            op[u] = on[u] ? pp[w.q] * ld + w.r : 0;
            oq[u] = on[u] ? qq[w.q] * ld + w.r : 0;
            w.next();
          }
          Cx<T> x[VB], y[VB];
#pragma unroll
          for (int u = 0; u < VB; u++)
            if (on[u]) { x[u] = V[op[u]]; y[u] = V[oq[u]]; }
#pragma unroll
          for (int u = 0; u < VB; u++)
            if (on[u]) {
              rot2(x[u], y[u], rc[kk[u]], rs[kk[u]], re[kk[u]]);
              V[op[u]] = x[u];
              V[oq[u]] = y[u];
            }
        }
      }
      __syncthreads();
    }
    if (!rotated) break;      // every pair below the threshold: converged
    __syncthreads();
  }
  return sweep + 1;
}

// Work placement of k_small_rr: the packed A (m (m + 1) / 2 entries) and S (m x (m + 1),
// column-major) in dynamic shared memory when the bits are set, else in the global work
// area, which holds 3 m (m + 1) entries per timeslice (S, packed A, the product H S).
enum { kRrShA = 1, kRrShS = 2 };

template <class T>
__global__ void __launch_bounds__(1024) k_small_rr(const double2* Gall, const double2* Hall, int m, double2* Call,
                                                  double* theta_all, Cx<T>* gwork, int place, int* dropped,
                                                  double drop_rel, int chol = 0) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int t = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const size_t mm = (size_t)m * m;
  const int ld = m + 1;                  // leading dimension of S and of H S (odd: no bank conflicts)
  const size_t ml = (size_t)m * ld;
  Cx<T>* gw = gwork + 3 * ml * t;
  Cx<T>* Sm = (place & kRrShS) ? (Cx<T>*)sm_raw + (((size_t)m * (m + 1) / 2 + 1) & ~(size_t)1) : gw;
  const Herm<T> A{(place & kRrShA) ? (Cx<T>*)sm_raw : gw + ml, m};
  Cx<T>* Z = gw + 2 * ml;                // H S, column-major
  __shared__ T rc[kSmallMaxM / 2], rs[kSmallMaxM / 2];
  __shared__ Cx<T> re[kSmallMaxM / 2];
  __shared__ double lam[kSmallMaxM], dsc[kSmallMaxM], gmx;
  __shared__ int order[kSmallMaxM], chol_ok;
  const double2* G = Gall + mm * t;
  const double2* H = Hall + mm * t;
  if (tid == 0) chol_ok = chol;
  __syncthreads();
  // the Cholesky route factors D^-1/2 G D^-1/2 (D = diag G): unit diagonal, so the
  // pivot test measures the angles between the columns, not their lengths, which the
  // filter spreads over many decades
  for (int i = tid; i < m; i += nt) {
    const double g = G[(size_t)i * m + i].x;
    dsc[i] = g > 0 ? 1.0 / sqrt(g) : 0.0;
    if (!(g > 0)) chol_ok = 0;
  }
  __syncthreads();
  int sw_g = 0;
  if (chol_ok) {
    for (DivWalk w(tid, nt, m); w.q < m; w.next())     // packed upper triangle of the scaled G
      if (w.q <= w.r) {
        const double2 g = G[(size_t)w.q * m + w.r];
        const double f = dsc[w.q] * dsc[w.r];
        A.a[A.off(w.q, w.r)] = cx<T>((T)(f * g.x), (T)(f * g.y));
      }
    __syncthreads();
    // 1') Cholesky D^-1/2 G D^-1/2 = R^dag R (R upper, packed in A), right-looking
    const T floor_piv = (T)(1e4 * (double)SmallPrec<T>::eps);
    for (int k = 0; k < m; k++) {
      if (tid == 0) {
        const T d = A.diag(k);
        if (!(d > floor_piv)) chol_ok = 0;
        A.a[A.off(k, k)] = cx<T>(sqrt(d > (T)0 ? d : (T)1), 0);
      }
      __syncthreads();
      if (!chol_ok) break;
      const T inv = (T)1 / A.diag(k);
      for (int j = k + 1 + tid; j < m; j += nt) A.a[A.off(k, j)] = inv * A.a[A.off(k, j)];    // row k of R
      __syncthreads();
      // trailing update: A[i][j] -= conj(R[k][i]) R[k][j] for k < i <= j
      const int rem = m - k - 1;
      if (rem > 0)
        for (DivWalk w(tid, nt, rem); w.q < rem; w.next()) {
          const int i = k + 1 + w.q, j = k + 1 + w.r;
          if (j < i) continue;
          A.a[A.off(i, j)] = A.a[A.off(i, j)] - conj(A.a[A.off(k, i)]) * A.a[A.off(k, j)];
        }
      __syncthreads();
    }
    if (chol_ok) {
      // S = D^-1/2 R^-1 (upper triangular, column-major).  R^-1 right-looking: S <- I,
      // then for k = m-1 .. 0 row k of S is divided by R[k][k] and eliminated from the
      // rows above it (S[i][c] -= R[i][k] S[k][c], i < k <= c)
      for (DivWalk w(tid, nt, m); w.q < m; w.next()) Sm[(size_t)w.q * ld + w.r] = cx<T>(w.q == w.r ? (T)1 : (T)0, 0);
      __syncthreads();
      for (int k = m - 1; k >= 0; k--) {
        const T inv = (T)1 / A.diag(k);
        for (int c = k + tid; c < m; c += nt) Sm[(size_t)c * ld + k] = inv * Sm[(size_t)c * ld + k];
        __syncthreads();
        if (k > 0)
          for (DivWalk w(tid, nt, k); w.q < m - k; w.next()) {
            Cx<T>* sc = Sm + (size_t)(k + w.q) * ld;
            sc[w.r] = sc[w.r] - A.a[A.off(w.r, k)] * sc[k];
          }
        __syncthreads();
      }
      for (DivWalk w(tid, nt, m); w.q < m; w.next()) {
        Cx<T>& sv = Sm[(size_t)w.q * ld + w.r];
        sv = (T)dsc[w.r] * sv;
      }
      for (int i = tid; i < m; i += nt) lam[i] = 1.0;   // no direction dropped
      __syncthreads();
    }
  }
  const bool tri = chol && chol_ok;                    // S upper triangular
  if (!tri) {
    // 1) eigen-decomposition of the Gram matrix (reloaded: a failed Cholesky overwrote it)
    for (DivWalk w(tid, nt, m); w.q < m; w.next()) {
      if (w.q <= w.r) A.a[A.off(w.q, w.r)] = cx<T>((T)G[(size_t)w.q * m + w.r].x, (T)G[(size_t)w.q * m + w.r].y);
      Sm[(size_t)w.q * ld + w.r] = cx<T>(w.q == w.r ? (T)1 : (T)0, 0);
    }
    __syncthreads();
    sw_g = jacobi<T>(A, Sm, ld, rc, rs, re);
    // 2) S <- Q diag(g)^-1/2, dropping directions with g <= drop_rel gmax
    if (tid == 0) {
      double g = 0;
      for (int i = 0; i < m; i++) g = fmax(g, (double)A.diag(i));
      gmx = g;
    }
    __syncthreads();
    for (int i = tid; i < m; i += nt) {
      const double gi = A.diag(i);
      lam[i] = gi > drop_rel * gmx ? 1.0 / sqrt(gi) : 0.0;
    }
    __syncthreads();
    for (DivWalk w(tid, nt, m); w.q < m; w.next()) {
      Cx<T>& s = Sm[(size_t)w.q * ld + w.r];
      s = (T)lam[w.q] * s;
    }
    __syncthreads();
  }
  // 3) Z <- H^dag S (column-major; reading H by columns keeps the loads coalesced) and
  //    A <- the hermitian part of S^dag Z, which is that of S^dag H S (H is hermitian
  //    up to rounding).  An upper triangular S limits the sums to l <= column.
  for (DivWalk w(tid, nt, m); w.q < m; w.next()) {
    const int j = w.q, i = w.r;
    const int lmax = tri ? j : m - 1;
    const Cx<T>* sj = Sm + (size_t)j * ld;
    Cx<T> s = cx<T>(0, 0);
    for (int l = 0; l <= lmax; l++) fma_conj_acc(s, cx<T>((T)H[(size_t)l * m + i].x, (T)H[(size_t)l * m + i].y), sj[l]);
    Z[(size_t)j * ld + i] = s;
  }
  __syncthreads();
  for (DivWalk w(tid, nt, m); w.q < m; w.next()) {
    const int j = w.q, i = w.r;
    if (i > j) continue;
    const Cx<T>*si = Sm + (size_t)i * ld, *sj = Sm + (size_t)j * ld;
    const Cx<T>*zi = Z + (size_t)i * ld, *zj = Z + (size_t)j * ld;
    Cx<T> a = cx<T>(0, 0), b = cx<T>(0, 0);
    const int li = tri ? i : m - 1, lj = tri ? j : m - 1;
    for (int l = 0; l <= li; l++) fma_conj_acc(a, si[l], zj[l]);     // (S^dag Z)[i][j]
    if (i == j) {
      A.a[A.off(i, i)] = cx<T>(a.re, 0);
      continue;
    }
    for (int l = 0; l <= lj; l++) fma_conj_acc(b, sj[l], zi[l]);     // (S^dag Z)[j][i]
    A.a[A.off(i, j)] = cx<T>((T)0.5 * (a.re + b.re), (T)0.5 * (a.im - b.im));
  }
  __syncthreads();
  // 4) S <- S Z: the rotations that diagonalise S^dag H S, applied to S in place
  const int sw_h = jacobi<T>(A, Sm, ld, rc, rs, re);
  if (tid == 0) { dropped[1 + 2 * t] = sw_g; dropped[2 + 2 * t] = sw_h; }
  // 5) sort ascending.  A dropped direction i has an exactly zero row and column
  //    in S^dag H S, so Jacobi never rotates it and it keeps position i: sort it last.
  for (int i = tid; i < m; i += nt) lam[i] = lam[i] > 0 ? (double)A.diag(i) : 1e300;
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    int rank = 0;
    for (int l = 0; l < m; l++) rank += (lam[l] < lam[i]) || (lam[l] == lam[i] && l < i);
    order[rank] = i;
  }
  __syncthreads();
  // 6) C = (S Z)[:, order], row-major
  double2* Cout = Call + mm * t;
  for (DivWalk w(tid, nt, m); w.q < m; w.next()) {
    const Cx<T> s = Sm[(size_t)order[w.q] * ld + w.r];
    Cout[(size_t)w.r * m + w.q] = make_double2((double)s.re, (double)s.im);
  }
  for (int j = tid; j < m; j += nt) {
    const double v = lam[order[j]];
    theta_all[(size_t)t * m + j] = v;
    if (v > 1e299) atomicAdd(dropped, 1);
  }
}

// placement bits and dynamic shared memory of k_small_rr for m columns: the packed A
// first, then S beside it, within what the device grants one CTA beyond the kernel's
// static shared memory
template <class T> inline int small_rr_place(int m, size_t* sm_bytes) {
  static size_t budget = 0;
  if (!budget) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncGetAttributes(&fa, k_small_rr<T>);
    budget = optin > (int)fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 1;
  }
  const size_t a_bytes = ((size_t)m * (m + 1) / 2 + 1) / 2 * 2 * sizeof(Cx<T>);
  const size_t s_bytes = (size_t)m * (m + 1) * sizeof(Cx<T>);
  int place = 0;
  *sm_bytes = 0;
  if (a_bytes <= budget) { place |= kRrShA; *sm_bytes = a_bytes; }
  if (a_bytes + s_bytes <= budget) { place |= kRrShS; *sm_bytes += s_bytes; }
  return place;
}
