// Spatial covariant Laplacian of Eq. 1 and its low modes, batched over
// timeslices.
//
//   (lap v)(m, t) = -6 v(m) + sum_{j=1..3} [U_j(m,t) v(m+j) + U_j(m-j,t)^dag v(m-j)]
//
// The modes are the N lowest eigenpairs of A = -lap(t) (spectrum in [0, 12]),
// for every timeslice at once: a Chebyshev-filtered subspace iteration.  Each
// iteration filters an m-column block (m = N + buffer) with a degree-d
// Chebyshev polynomial of A that damps [cut, 12], then orthonormalises and
// diagonalises the filtered block (Rayleigh-Ritz) per timeslice:
//   G = Y^dag Y, H = Y^dag (A Y)  ->  G = Q diag(g) Q^dag, S = Q g^-1/2,
//   S^dag H S = Z diag(theta) Z^dag,  X <- Y S Z,  A X <- (A Y) S Z,
// all in FP64 (the small m x m eigenproblems by parallel cyclic Jacobi, one
// CTA per timeslice).  Stops when every wanted pair has
// ||A x - theta x|| <= tol * max(theta, 1).
// Block layout: column j of timeslice t (of a batch of Tn timeslices starting
// at t0) is the colour field [Vs][3] at offset (j * Tn + t) * 3 Vs.
#include "common.cuh"
#include <algorithm>
#include <math.h>

namespace {

// --------------------------------------------------------------------------
// fused stencil: out = alpha_t (A in) + beta_t in + gamma_t prev, A = -lap
__global__ void __launch_bounds__(128) k_lap_fused(Geom g, int t0, int Tn, const double2* __restrict__ U3,
                                                   const double2* __restrict__ in, const double2* __restrict__ prev,
                                                   double2* __restrict__ out, int nvec, const double* __restrict__ coef) {
  const int sl = blockIdx.x * blockDim.x + threadIdx.x;     // site within the batch
  const int j = blockIdx.y;
  if (sl >= Tn * g.Vs || j >= nvec) return;
  const int tl = sl / g.Vs;
  const int m = sl - tl * g.Vs;
  const int x = m % g.L, y = (m / g.L) % g.L, z = m / (g.L * g.L);
  const size_t s = (size_t)(t0 + tl) * g.Vs + m;            // global site for links
  const size_t col = ((size_t)j * Tn + tl) * g.Vs * 3;
  const double2* v = in + col;
  const double alpha = coef[3 * tl], beta = coef[3 * tl + 1], gamma = coef[3 * tl + 2];
  Cx<double> own[3], acc[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    double2 e = v[(size_t)m * 3 + a];
    own[a] = cx<double>(e.x, e.y);
    acc[a] = cx<double>(6.0 * e.x, 6.0 * e.y);       // A = 6 - hopping
  }
#pragma unroll
  for (int k = 0; k < 3; k++) {
    int xf = x, yf = y, zf = z, xb = x, yb = y, zb = z;
    if (k == 0) { xf = x + 1 == g.L ? 0 : x + 1; xb = x == 0 ? g.L - 1 : x - 1; }
    else if (k == 1) { yf = y + 1 == g.L ? 0 : y + 1; yb = y == 0 ? g.L - 1 : y - 1; }
    else { zf = z + 1 == g.L ? 0 : z + 1; zb = z == 0 ? g.L - 1 : z - 1; }
    const int mf = xf + g.L * (yf + g.L * zf), mb = xb + g.L * (yb + g.L * zb);
    const size_t sb = (size_t)(t0 + tl) * g.Vs + mb;
    Cx<double> vf[3], vb[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      double2 e = v[(size_t)mf * 3 + a];
      vf[a] = cx<double>(e.x, e.y);
      e = v[(size_t)mb * 3 + a];
      vb[a] = cx<double>(e.x, e.y);
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
      Cx<double> h = cx<double>(0, 0);
#pragma unroll
      for (int b = 0; b < 3; b++) {
        double2 uf = __ldg(U3 + ((size_t)k * 9 + a * 3 + b) * g.V + s);
        double2 ub = __ldg(U3 + ((size_t)k * 9 + b * 3 + a) * g.V + sb);
        fma_acc(h, cx<double>(uf.x, uf.y), vf[b]);
        fma_conj_acc(h, cx<double>(ub.x, ub.y), vb[b]);
      }
      acc[a] = acc[a] - h;
    }
  }
  double2* o = out + col;
  const double2* pv = prev ? prev + col : nullptr;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    Cx<double> r = alpha * acc[a] + beta * own[a];
    if (pv) {
      double2 e = pv[(size_t)m * 3 + a];
      r = r + gamma * cx<double>(e.x, e.y);
    }
    o[(size_t)m * 3 + a] = make_double2(r.re, r.im);
  }
}

// --------------------------------------------------------------------------
// Gram partials: part[t][split][i][j] = sum_{k in chunk} conj(X_t[k][i]) Y_t[k][j]
constexpr int GT = 32, GKS = 32;
__global__ void __launch_bounds__(256) k_gram(const double2* __restrict__ X, const double2* __restrict__ Y, int n,
                                              int Tn, int m1, int m2, int nsplit, double2* part) {
  __shared__ double2 xs[GKS][GT + 1];
  __shared__ double2 ys[GKS][GT + 1];
  const int tiles_j = (m2 + GT - 1) / GT;
  const int i0 = (blockIdx.x / tiles_j) * GT, j0 = (blockIdx.x % tiles_j) * GT;
  const int split = blockIdx.y, t = blockIdx.z;
  const int chunk = (n + nsplit - 1) / nsplit;
  const int k0 = split * chunk, k1 = min(n, k0 + chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4, tid = threadIdx.x;
  Cx<double> acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) acc[a][b] = cx<double>(0, 0);
  for (int kb = k0; kb < k1; kb += GKS) {
#pragma unroll
    for (int q = 0; q < (GKS * GT) / 256; q++) {
      int e = tid + 256 * q;
      int c = e / GKS, r = e % GKS;
      int k = kb + r;
      double2 vx = make_double2(0, 0), vy = make_double2(0, 0);
      if (k < k1) {
        if (i0 + c < m1) vx = X[((size_t)(i0 + c) * Tn + t) * n + k];
        if (j0 + c < m2) vy = Y[((size_t)(j0 + c) * Tn + t) * n + k];
      }
      xs[r][c] = vx;
      ys[r][c] = vy;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < GKS; r++) {
      double2 x0 = xs[r][ty], x1 = xs[r][ty + 16], y0 = ys[r][tx], y1 = ys[r][tx + 16];
      fma_conj_acc(acc[0][0], cx<double>(x0.x, x0.y), cx<double>(y0.x, y0.y));
      fma_conj_acc(acc[0][1], cx<double>(x0.x, x0.y), cx<double>(y1.x, y1.y));
      fma_conj_acc(acc[1][0], cx<double>(x1.x, x1.y), cx<double>(y0.x, y0.y));
      fma_conj_acc(acc[1][1], cx<double>(x1.x, x1.y), cx<double>(y1.x, y1.y));
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < m1 && j < m2) part[(((size_t)t * nsplit + split) * m1 + i) * m2 + j] = make_double2(acc[a][b].re, acc[a][b].im);
    }
}

__global__ void k_gram_reduce(const double2* part, int nsplit, int m1, int m2, int Tn, double2* G) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t per = (size_t)m1 * m2;
  if (e >= per * Tn) return;
  size_t t = e / per, ij = e % per;
  double2 s = make_double2(0, 0);
  for (int q = 0; q < nsplit; q++) {
    double2 v = part[(t * nsplit + q) * per + ij];
    s.x += v.x;
    s.y += v.y;
  }
  G[e] = s;
}

// --------------------------------------------------------------------------
// rotation: Z_t[k][j] = sum_l X_t[k][l] C_t[l][j], C_t [m1][m2] row-major
constexpr int RJ = 16;
__global__ void __launch_bounds__(128) k_rotate(const double2* __restrict__ X, const double2* __restrict__ Cm, int n,
                                                int Tn, int m1, int m2, double2* __restrict__ Z) {
  extern __shared__ double2 cs[];          // [m1][RJ]
  const int t = blockIdx.z, j0 = blockIdx.y * RJ;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const double2* C = Cm + (size_t)t * m1 * m2;
  for (int e = threadIdx.x; e < m1 * RJ; e += blockDim.x) {
    int l = e / RJ, jj = e % RJ;
    cs[e] = (j0 + jj < m2) ? C[(size_t)l * m2 + j0 + jj] : make_double2(0, 0);
  }
  __syncthreads();
  if (k >= n) return;
  Cx<double> acc[RJ];
#pragma unroll
  for (int jj = 0; jj < RJ; jj++) acc[jj] = cx<double>(0, 0);
  for (int l = 0; l < m1; l++) {
    double2 xv = __ldg(X + ((size_t)l * Tn + t) * n + k);
    Cx<double> x = cx<double>(xv.x, xv.y);
#pragma unroll
    for (int jj = 0; jj < RJ; jj++) {
      double2 c = cs[l * RJ + jj];
      fma_acc(acc[jj], x, cx<double>(c.x, c.y));
    }
  }
#pragma unroll
  for (int jj = 0; jj < RJ; jj++)
    if (j0 + jj < m2) Z[((size_t)(j0 + jj) * Tn + t) * n + k] = make_double2(acc[jj].re, acc[jj].im);
}

// --------------------------------------------------------------------------
// small dense hermitian eigenproblems (parallel cyclic Jacobi), one CTA per timeslice
__device__ __forceinline__ int rr_pos(int idx, int r, int m) { return idx == 0 ? 0 : ((idx - 1 + r) % (m - 1)) + 1; }

// Diagonalise the hermitian A [m][m] (row-major, in place) and accumulate the
// eigenvectors into V (columns); V must hold the initial basis.
__device__ void jacobi(double2* A, double2* V, int m, double* rc, double* rs, double2* re, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int np = m / 2;
  for (int sweep = 0; sweep < 40; sweep++) {
    // convergence: off-diagonal vs diagonal
    double off = 0, dia = 0;
    for (int e = tid; e < m * m; e += nt) {
      int i = e / m, j = e % m;
      double2 v = A[e];
      if (i == j) dia += v.x * v.x;
      else off += v.x * v.x + v.y * v.y;
    }
    red[tid] = off;
    red[nt + tid] = dia;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s) { red[tid] += red[tid + s]; red[nt + tid] += red[nt + tid + s]; }
      __syncthreads();
    }
    bool done = red[0] <= 1e-30 * red[nt] || red[0] == 0.0;
    __syncthreads();
    if (done) break;
    for (int r = 0; r < m - 1; r++) {
      for (int k = tid; k < np; k += nt) {
        int p = rr_pos(k, r, m), q = rr_pos(m - 1 - k, r, m);
        double a = A[p * m + p].x, d = A[q * m + q].x;
        double2 b = A[p * m + q];
        double ab = sqrt(b.x * b.x + b.y * b.y);
        if (ab < 1e-300) { rc[k] = 1; rs[k] = 0; re[k] = make_double2(1, 0); continue; }
        double tau = (d - a) / (2 * ab);
        double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1 + tau * tau));
        double c = 1 / sqrt(1 + tt * tt);
        rc[k] = c;
        rs[k] = tt * c;
        re[k] = make_double2(b.x / ab, -b.y / ab);   // e^{-i phi}
      }
      __syncthreads();
      // A <- A J and V <- V J (columns p, q)
      for (int e = tid; e < np * m; e += nt) {
        int k = e / m, i = e % m;
        int p = rr_pos(k, r, m), q = rr_pos(m - 1 - k, r, m);
        Cx<double> c = cx<double>(rc[k], 0), s = cx<double>(rs[k], 0), ph = cx<double>(re[k].x, re[k].y);
        Cx<double> ap = cx<double>(A[i * m + p].x, A[i * m + p].y), aq = cx<double>(A[i * m + q].x, A[i * m + q].y);
        Cx<double> np_ = c * ap - s * (ph * aq), nq = s * ap + c * (ph * aq);
        A[i * m + p] = make_double2(np_.re, np_.im);
        A[i * m + q] = make_double2(nq.re, nq.im);
        Cx<double> vp = cx<double>(V[i * m + p].x, V[i * m + p].y), vq = cx<double>(V[i * m + q].x, V[i * m + q].y);
        np_ = c * vp - s * (ph * vq);
        nq = s * vp + c * (ph * vq);
        V[i * m + p] = make_double2(np_.re, np_.im);
        V[i * m + q] = make_double2(nq.re, nq.im);
      }
      __syncthreads();
      // A <- J^dag A (rows p, q)
      for (int e = tid; e < np * m; e += nt) {
        int k = e / m, j = e % m;
        int p = rr_pos(k, r, m), q = rr_pos(m - 1 - k, r, m);
        Cx<double> c = cx<double>(rc[k], 0), s = cx<double>(rs[k], 0), ph = conj(cx<double>(re[k].x, re[k].y));
        Cx<double> ap = cx<double>(A[p * m + j].x, A[p * m + j].y), aq = cx<double>(A[q * m + j].x, A[q * m + j].y);
        Cx<double> np_ = c * ap - s * (ph * aq), nq = s * ap + c * (ph * aq);
        A[p * m + j] = make_double2(np_.re, np_.im);
        A[q * m + j] = make_double2(nq.re, nq.im);
      }
      __syncthreads();
    }
  }
}

// Rayleigh-Ritz on one timeslice: from G = Y^dag Y and H = Y^dag A Y produce C
// (Y C orthonormal Ritz vectors, ascending Ritz values theta).  Work: 3 m x m buffers.
__global__ void __launch_bounds__(256) k_small_rr(const double2* Gall, const double2* Hall, int m, double2* Call,
                                                  double* theta_all, double2* gwork, int use_smem, int* dropped) {
  extern __shared__ double2 sm[];
  const int t = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const size_t mm = (size_t)m * m;
  double2 *S, *A, *Z;
  if (use_smem) { S = sm; A = sm + mm; Z = sm + 2 * mm; }
  else { S = gwork + 3 * mm * t; A = S + mm; Z = A + mm; }
  __shared__ double rc[128], rs[128], red[512], lam[256];
  __shared__ double2 re[128];
  __shared__ int order[256];
  const double2* G = Gall + mm * t;
  const double2* H = Hall + mm * t;
  // 1) eigen-decomposition of the Gram matrix
  for (size_t e = tid; e < mm; e += nt) {
    A[e] = G[e];
    S[e] = make_double2((e / m) == (e % m) ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  jacobi(A, S, m, rc, rs, re, red);
  // 2) S <- Q diag(g)^-1/2, dropping directions with g <= 1e-24 gmax (round-off level)
  if (tid == 0) {
    double gmax = 0;
    for (int i = 0; i < m; i++) gmax = fmax(gmax, A[i * m + i].x);
    red[0] = gmax;
  }
  __syncthreads();
  const double gmax = red[0];
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    double gi = A[i * m + i].x;
    lam[i] = gi > 1e-24 * gmax ? 1.0 / sqrt(gi) : 0.0;
  }
  __syncthreads();
  for (size_t e = tid; e < mm; e += nt) {
    int j = e % m;
    S[e] = make_double2(S[e].x * lam[j], S[e].y * lam[j]);
  }
  __syncthreads();
  // 3) Z <- H S ; A <- S^dag Z  (= S^dag H S)
  for (size_t e = tid; e < mm; e += nt) {
    int i = e / m, j = e % m;
    Cx<double> s = cx<double>(0, 0);
    for (int l = 0; l < m; l++) fma_acc(s, cx<double>(H[i * m + l].x, H[i * m + l].y), cx<double>(S[l * m + j].x, S[l * m + j].y));
    Z[e] = make_double2(s.re, s.im);
  }
  __syncthreads();
  for (size_t e = tid; e < mm; e += nt) {
    int i = e / m, j = e % m;
    Cx<double> s = cx<double>(0, 0);
    for (int l = 0; l < m; l++) fma_conj_acc(s, cx<double>(S[l * m + i].x, S[l * m + i].y), cx<double>(Z[l * m + j].x, Z[l * m + j].y));
    A[e] = make_double2(s.re, s.im);
  }
  __syncthreads();
  // symmetrise (round-off) and reset Z to the identity
  for (size_t e = tid; e < mm; e += nt) {
    int i = e / m, j = e % m;
    if (i < j) {
      double2 a = A[i * m + j], b = A[j * m + i];
      double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      A[i * m + j] = h;
      A[j * m + i] = make_double2(h.x, -h.y);
    } else if (i == j) {
      A[e].y = 0;
    }
  }
  for (size_t e = tid; e < mm; e += nt) Z[e] = make_double2((e / m) == (e % m) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  jacobi(A, Z, m, rc, rs, re, red);
  // 4) sort ascending; dropped directions (zero S column) sort last
  for (int i = tid; i < m; i += nt) lam[i] = lam[i] > 0 ? A[i * m + i].x : 1e300;
  __syncthreads();
  // (a dropped direction i has an exactly zero row and column in S^dag H S, so
  //  Jacobi never rotates it and it keeps diagonal position i: sorted last above)
  for (int i = tid; i < m; i += nt) {
    int rank = 0;
    for (int l = 0; l < m; l++) rank += (lam[l] < lam[i]) || (lam[l] == lam[i] && l < i);
    order[rank] = i;
  }
  __syncthreads();
  // 5) C = S Z[:, order]
  double2* Cout = Call + mm * t;
  for (size_t e = tid; e < mm; e += nt) {
    int i = e / m, j = e % m;
    int zj = order[j];
    Cx<double> s = cx<double>(0, 0);
    for (int l = 0; l < m; l++) fma_acc(s, cx<double>(S[i * m + l].x, S[i * m + l].y), cx<double>(Z[l * m + zj].x, Z[l * m + zj].y));
    Cout[e] = make_double2(s.re, s.im);
  }
  for (int j = tid; j < m; j += nt) {
    double v = lam[order[j]];
    theta_all[(size_t)t * m + j] = v;
    if (v > 1e299) atomicAdd(dropped, 1);
  }
}

// residual norms res[t][j] = ||W_j - theta_j X_j|| for the batch
__global__ void k_resid(const double2* __restrict__ X, const double2* __restrict__ W, const double* theta, int n,
                        int Tn, int m, double* res) {
  const int j = blockIdx.x, t = blockIdx.y;
  const double th = theta[(size_t)t * m + j];
  const double2* x = X + ((size_t)j * Tn + t) * n;
  const double2* w = W + ((size_t)j * Tn + t) * n;
  double s = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double2 a = w[k], b = x[k];
    double dx = a.x - th * b.x, dy = a.y - th * b.y;
    s += dx * dx + dy * dy;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) res[(size_t)t * m + j] = sqrt(red[0]);
}

// counter-based start vectors: splitmix64 of (seed, index) -> two uniforms in (-1, 1)
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__global__ void k_random(double2* X, size_t count, uint64_t seed) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  uint64_t h = splitmix64(seed ^ splitmix64(e));
  double a = (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  uint64_t h2 = splitmix64(h);
  double b = (double)(h2 >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  X[e] = make_double2(a, b);
}

// copy the first N columns of the block into evecs [Tn][N][Vs][3] (or the cache layout [N][T][Vs][3])
__global__ void k_extract(const double2* X, int n, int Tn, int N, double2* out, int cache_layout, int T, int t0) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = (size_t)N * Tn * n;
  if (e >= total) return;
  size_t k = e % n;
  size_t rest = e / n;
  int t = rest % Tn;
  int j = rest / Tn;
  double2 v = X[((size_t)j * Tn + t) * n + k];
  if (cache_layout) out[((size_t)j * T + t0 + t) * n + k] = v;
  else out[((size_t)t * N + j) * n + k] = v;
}

}  // namespace

// ---------------------------------------------------------------------------
struct EigBufs {
  double2 *X, *Y, *Yn, *W, *G, *H, *part, *C, *gwork;
  double *theta, *res, *coef;
  int* dropped;
};

static dlma_status lap_apply_batch(dlma_ctx* ctx, int t0, int Tn, int m, const double2* in, const double2* prev,
                                   double2* out, const double* coef) {
  dim3 grid((Tn * ctx->g.Vs + 127) / 128, m);
  k_lap_fused<<<grid, 128, 0, ctx->stream>>>(ctx->g, t0, Tn, ctx->U3, in, prev, out, m, coef);
  CHECK_LAUNCH();
  return DLMA_OK;
}

static dlma_status gram(dlma_ctx* ctx, const double2* X, const double2* Y, int n, int Tn, int m, EigBufs& B,
                        double2* out, int nsplit) {
  int tiles = ((m + GT - 1) / GT) * ((m + GT - 1) / GT);
  dim3 grid(tiles, nsplit, Tn);
  k_gram<<<grid, 256, 0, ctx->stream>>>(X, Y, n, Tn, m, m, nsplit, B.part);
  CHECK_LAUNCH();
  size_t tot = (size_t)m * m * Tn;
  k_gram_reduce<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(B.part, nsplit, m, m, Tn, out);
  CHECK_LAUNCH();
  return DLMA_OK;
}

static dlma_status rotate(dlma_ctx* ctx, const double2* X, const double2* C, int n, int Tn, int m, double2* Z) {
  dim3 grid((n + 127) / 128, (m + RJ - 1) / RJ, Tn);
  size_t sm = (size_t)m * RJ * sizeof(double2);
  if (sm > 48 * 1024) CU(cudaFuncSetAttribute(k_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_rotate<<<grid, 128, sm, ctx->stream>>>(X, C, n, Tn, m, m, Z);
  CHECK_LAUNCH();
  return DLMA_OK;
}

static dlma_status small_rr(dlma_ctx* ctx, EigBufs& B, int Tn, int m) {
  size_t sm = (size_t)3 * m * m * sizeof(double2);
  // the kernel also holds ~11 KB of static shared memory: always raise the dynamic limit
  int use_smem = sm <= 200 * 1024;
  if (use_smem) CU(cudaFuncSetAttribute(k_small_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_small_rr<<<Tn, 256, use_smem ? sm : 0, ctx->stream>>>(B.G, B.H, m, B.C, B.theta, B.gwork, use_smem, B.dropped);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// One Rayleigh-Ritz step on the block Y (with W = A Y computed here):
// X <- Y C, Wx <- W C, theta, residual norms.  Y, W are clobbered only via outputs.
static dlma_status rayleigh_ritz(dlma_ctx* ctx, EigBufs& B, int t0, int Tn, int m, int n, double2* Yblk,
                                 double2* Wblk, double2* Xout, double2* Wout, int nsplit) {
  // W = A Y (alpha 1, beta 0)
  TRY(lap_apply_batch(ctx, t0, Tn, m, Yblk, nullptr, Wblk, B.coef));
  TRY(gram(ctx, Yblk, Yblk, n, Tn, m, B, B.G, nsplit));
  TRY(gram(ctx, Yblk, Wblk, n, Tn, m, B, B.H, nsplit));
  CU(cudaMemsetAsync(B.dropped, 0, sizeof(int), ctx->stream));
  TRY(small_rr(ctx, B, Tn, m));
  TRY(rotate(ctx, Yblk, B.C, n, Tn, m, Xout));
  TRY(rotate(ctx, Wblk, B.C, n, Tn, m, Wout));
  k_resid<<<dim3(m, Tn), 256, 0, ctx->stream>>>(Xout, Wout, B.theta, n, Tn, m, B.res);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// Modes of timeslices [t0, t0 + Tn): eigenvalues into lam_out [Tn][N] (host), vectors into the block X
static dlma_status eig_batch(dlma_ctx* ctx, int t0, int Tn, int N, double tol, double* lam_out, double2** Xres,
                             int* m_out) {
  const int n = 3 * ctx->g.Vs;
  int buf = std::max(8, (N + 3) / 4);
  int m = N + buf;
  m += m & 1;
  if (m > n) m = n - (n & 1);
  if (m < N) return set_err(ctx, DLMA_ERR_INVALID_ARG, "N too large for the timeslice");
  if (m > 254) return set_err(ctx, DLMA_ERR_INVALID_ARG, "N above the eigensolver's limit of 240");
  const size_t blk = (size_t)m * Tn * n;
  EigBufs B;
  TRY(workT(ctx, WS_EIG_X, blk, &B.X));
  TRY(workT(ctx, WS_EIG_Y, blk, &B.Y));
  TRY(workT(ctx, WS_EIG_Y2, blk, &B.Yn));
  TRY(workT(ctx, WS_EIG_W, blk, &B.W));
  int nsplit = std::max(1, std::min(64, (4 * 152) / std::max(1, Tn * ((m + GT - 1) / GT) * ((m + GT - 1) / GT))));
  nsplit = std::min(nsplit, std::max(1, n / 256));
  const size_t mm = (size_t)m * m;
  TRY(workT(ctx, WS_EIG_G, 3 * mm * Tn, &B.G));
  B.H = B.G + mm * Tn;
  B.C = B.H + mm * Tn;
  TRY(workT(ctx, WS_EIG_PART, (size_t)nsplit * mm * Tn, &B.part));
  TRY(workT(ctx, WS_EIG_S, 3 * mm * Tn, &B.gwork));
  double* aux;
  TRY(workT(ctx, WS_EIG_AUX, (size_t)2 * m * Tn + 64 * (size_t)Tn * 3 + 16, &aux));
  B.theta = aux;
  B.res = aux + (size_t)m * Tn;
  B.coef = aux + (size_t)2 * m * Tn;
  B.dropped = (int*)(B.coef + 64 * (size_t)Tn * 3);

  std::vector<double> hcoef(64 * 3 * (size_t)Tn);
  // W = A Y uses alpha 1, beta 0, gamma 0 from the first coefficient slot
  for (int t = 0; t < Tn; t++) { hcoef[3 * t] = 1; hcoef[3 * t + 1] = 0; hcoef[3 * t + 2] = 0; }
  CU(cudaMemcpyAsync(B.coef, hcoef.data(), sizeof(double) * 3 * Tn, cudaMemcpyHostToDevice, ctx->stream));
  k_random<<<(blk + 255) / 256, 256, 0, ctx->stream>>>(B.Y, blk, 0x5eed2022ULL + (uint64_t)t0 * 7919ULL);
  CHECK_LAUNCH();
  // initial Rayleigh-Ritz on the random block
  TRY(rayleigh_ritz(ctx, B, t0, Tn, m, n, B.Y, B.W, B.X, B.Yn, nsplit));
  std::vector<double> th((size_t)m * Tn), rs((size_t)m * Tn);
  const int degree = 20;
  const int max_iter = 400;
  int it = 0;
  bool conv = false;
  for (; it < max_iter; it++) {
    CU(cudaMemcpyAsync(th.data(), B.theta, sizeof(double) * m * Tn, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(rs.data(), B.res, sizeof(double) * m * Tn, cudaMemcpyDeviceToHost, ctx->stream));
    int hdrop = 0;
    CU(cudaMemcpyAsync(&hdrop, B.dropped, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (hdrop) return set_err(ctx, DLMA_ERR_NOT_CONVERGED, "eigensolver lost rank (%d directions)", hdrop);
    double worst = 0;
    for (int t = 0; t < Tn; t++)
      for (int k = 0; k < N; k++) {
        double r = rs[(size_t)t * m + k] / std::max(1.0, fabs(th[(size_t)t * m + k]));
        if (!(r == r)) return set_err(ctx, DLMA_ERR_NONFINITE, "NaN in the eigensolver");
        worst = std::max(worst, r);
      }
    if (worst <= tol) { conv = true; break; }
    // Chebyshev filter of degree d damping [cut_t, 12], scaled at lam0_t
    for (int t = 0; t < Tn; t++) {
      double a = th[(size_t)t * m + m - 1], a0 = th[(size_t)t * m];
      double b = 12.0;
      if (a >= b) a = 0.5 * (a0 + b);
      double e = 0.5 * (b - a), c = 0.5 * (b + a);
      double sigma = e / (a0 - c), tau = 2.0 / sigma;
      hcoef[3 * t + 0] = sigma / e;
      hcoef[3 * t + 1] = -c * sigma / e;
      hcoef[3 * t + 2] = 0.0;
      for (int k = 2; k <= degree; k++) {
        double sn = 1.0 / (tau - sigma);
        size_t o = (size_t)(k - 1) * 3 * Tn + 3 * t;
        hcoef[o + 0] = 2.0 * sn / e;
        hcoef[o + 1] = -2.0 * c * sn / e;
        hcoef[o + 2] = -sigma * sn;
        sigma = sn;
      }
      size_t o = (size_t)degree * 3 * Tn + 3 * t;   // slot for the plain A application
      hcoef[o] = 1; hcoef[o + 1] = 0; hcoef[o + 2] = 0;
    }
    CU(cudaMemcpyAsync(B.coef, hcoef.data(), sizeof(double) * 3 * Tn * (degree + 1), cudaMemcpyHostToDevice,
                       ctx->stream));
    // three-term recurrence: prev = X, cur = Y
    double2 *prev = B.X, *cur = B.Y, *nxt = B.Yn;
    TRY(lap_apply_batch(ctx, t0, Tn, m, prev, nullptr, cur, B.coef));
    for (int k = 2; k <= degree; k++) {
      TRY(lap_apply_batch(ctx, t0, Tn, m, cur, prev, nxt, B.coef + (size_t)(k - 1) * 3 * Tn));
      double2* tmp = prev;
      prev = cur;
      cur = nxt;
      nxt = tmp;
    }
    // Rayleigh-Ritz on the filtered block cur: needs W (use nxt), outputs X (prev is free) and AX (W buffer)
    double* coef_save = B.coef;
    B.coef = B.coef + (size_t)degree * 3 * Tn;
    dlma_status s = rayleigh_ritz(ctx, B, t0, Tn, m, n, cur, nxt, prev, B.W, nsplit);
    // near convergence, a second Rayleigh-Ritz pass on the (now well-conditioned)
    // block restores orthonormality lost in the one-pass Gram orthogonalisation
    if (s == DLMA_OK && worst < 1e-6) s = rayleigh_ritz(ctx, B, t0, Tn, m, n, prev, nxt, cur, B.W, nsplit);
    B.coef = coef_save;
    TRY(s);
    if (worst < 1e-6) { B.X = cur; B.Y = prev; B.Yn = nxt; }
    else { B.X = prev; B.Y = cur; B.Yn = nxt; }
  }
  if (!conv) return set_err(ctx, DLMA_ERR_NOT_CONVERGED, "eigensolver did not reach tol %.3g in %d iterations", tol, it);
  for (int t = 0; t < Tn; t++)
    for (int k = 0; k < N; k++) lam_out[(size_t)t * N + k] = th[(size_t)t * m + k];
  *Xres = B.X;
  *m_out = m;
  return DLMA_OK;
}

extern "C" dlma_status dlma_apply_laplacian(dlma_ctx* ctx, const double* in, double* out, int nvec, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge) return set_err(ctx, DLMA_ERR_STATE, "no gauge field");
  if (!in || !out || nvec < 1) return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument");
  CU(cudaSetDevice(ctx->device));
  size_t bytes = (size_t)nvec * ctx->g.V * 3 * 16;
  const double* din;
  TRY(copy_in(ctx, WS_IN, in, bytes, mem, &din));
  double* dout = out;
  if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_OUT, bytes / 8, &dout));
  // lap = -A: alpha = -1
  double* coef;
  TRY(workT(ctx, WS_T0, (size_t)3 * ctx->g.T, &coef));
  std::vector<double> h(3 * ctx->g.T);
  for (int t = 0; t < ctx->g.T; t++) { h[3 * t] = -1; h[3 * t + 1] = 0; h[3 * t + 2] = 0; }
  CU(cudaMemcpyAsync(coef, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, ctx->stream));
  // canonical [nvec][V][3] equals the block layout with Tn = 1 per column when t0 = 0 and Tn = T
  // (column j of timeslice t at (j T + t) 3 Vs)
  TRY(lap_apply_batch(ctx, 0, ctx->g.T, nvec, (const double2*)din, nullptr, (double2*)dout, coef));
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
  double2* X = nullptr;
  int m = 0;
  TRY(eig_batch(ctx, t0, Tn, N, tol, evals, &X, &m));
  // cache (all timeslices, [N][T][Vs][3])
  if (ctx->eig_N != N || !ctx->eig_V) {
    if (ctx->eig_V) cudaFree(ctx->eig_V);
    ctx->eig_V = nullptr;
    ctx->eig_N = 0;
    CU(cudaMalloc(&ctx->eig_V, (size_t)N * ctx->g.T * n * sizeof(double2)));
    ctx->eig_lam.assign((size_t)N * ctx->g.T, 0.0);
    ctx->eig_have.assign(ctx->g.T, 0);
    ctx->eig_N = N;
  }
  size_t tot = (size_t)N * Tn * n;
  k_extract<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(X, n, Tn, N, ctx->eig_V, 1, ctx->g.T, t0);
  CHECK_LAUNCH();
  for (int tt = 0; tt < Tn; tt++) {
    ctx->eig_have[t0 + tt] = 1;
    for (int k = 0; k < N; k++) ctx->eig_lam[(size_t)(t0 + tt) * N + k] = evals[(size_t)tt * N + k];
  }
  if (evecs) {
    size_t bytes = tot * sizeof(double2);
    double2* dst = (double2*)evecs;
    if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_OUT, tot, &dst));
    k_extract<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(X, n, Tn, N, dst, 0, ctx->g.T, t0);
    CHECK_LAUNCH();
    if (mem == DLMA_MEM_HOST) TRY(copy_out(ctx, evecs, (const double*)dst, bytes, mem));
  }
  CU(cudaEventRecord(e1, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  ctx->timing[0] = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return DLMA_OK;
}
