// Conventional low-mode averaging with Dirac low modes: the control of Sec. 1
// and of the remark after Eq. 2 (with Box built from eigenmodes of the Dirac
// operator, Box and the propagator commute and C_mixed vanishes).
//
// The modes are eigenpairs of the hermitian even-odd operator Qhat = g5 Dhat on
// the even sites with the smallest |lambda|.  They are found by Chebyshev-
// filtered subspace iteration on Qhat^2 = Dhat^dag Dhat (FP64 Schur operator):
// Rayleigh-Ritz of Qhat^2 on a block of m = N + max(8, N) vectors, a degree-d
// filter damping [theta_max, lambda_max(Qhat^2)], until the N lowest Ritz pairs
// of Qhat^2 converge; a last Rayleigh-Ritz of Qhat itself in their span gives
// the signed eigenvalues (the span of the N lowest Qhat^2 modes is
// Qhat-invariant when no pair +-lambda is split by the cut).  The small dense
// problems reuse the Jacobi Rayleigh-Ritz kernel of the Laplacian eigensolver.
//
// With P = sum_i u_i u_i^dag: Dhat^-1 = Qhat^-1 g5, so P Dhat^-1 (1 - g5 P g5) =
// Qhat^-1 P (1 - P) g5 = 0 -- the mixed block of Eq. 2 vanishes; the
// Laplacian Box (spin-diagonal, g5 Box g5 = Box) gives Box Dhat^-1 (1 - Box) != 0.
#include "common.cuh"

#include <algorithm>
#include <math.h>

namespace lma_small {
#include "smalleig.cuh"
}

namespace {

// G[a][b] = sum_e conj(X_a[e]) Y_b[e] (X_a = X + a n): one block per (a, b)
__global__ void __launch_bounds__(256) k_fgram(const double2* __restrict__ X, const double2* __restrict__ Y, int ma,
                                               int mb, size_t n, double2* G) {
  const int a = blockIdx.x, b = blockIdx.y;
  const double2* x = X + (size_t)a * n;
  const double2* y = Y + (size_t)b * n;
  double sr = 0, si = 0;
  for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
    const double2 u = x[e], v = y[e];
    sr += u.x * v.x + u.y * v.y;
    si += u.x * v.y - u.y * v.x;
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = sr;
  red[1][threadIdx.x] = si;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) G[(size_t)a * mb + b] = make_double2(red[0][0], red[1][0]);
}

// Y_b[e] = sum_a X_a[e] C[a][b]  (C [ma][mb] row-major)
__global__ void k_frot(const double2* __restrict__ X, const double2* __restrict__ C, int ma, int mb, size_t n,
                       double2* Y) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (e >= n) return;
  Cx<double> s = cx<double>(0, 0);
  for (int a = 0; a < ma; a++) {
    const double2 x = X[(size_t)a * n + e], c = C[(size_t)a * mb + b];
    fma_acc(s, cx<double>(x.x, x.y), cx<double>(c.x, c.y));
  }
  Y[(size_t)b * n + e] = make_double2(s.re, s.im);
}

// Yn = c0 AY + c1 Y + c2 Yp
__global__ void k_cheb(size_t total, const double2* AY, const double2* Y, const double2* Yp, double c0, double c1,
                       double c2, double2* Yn) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const double2 a = AY[e], y = Y[e], p = Yp ? Yp[e] : make_double2(0, 0);
  Yn[e] = make_double2(c0 * a.x + c1 * y.x + c2 * p.x, c0 * a.y + c1 * y.y + c2 * p.y);
}

// gamma_5 on FP64 fields [m][12][Vh] (components 6..11 are spins 2, 3)
__global__ void k_g5(size_t total, int Vh, double2* X) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int comp = (int)((e / Vh) % 12);
  if (comp >= 6) X[e] = make_double2(-X[e].x, -X[e].y);
}

// counter-based Gaussian-free start vectors: uniform in [-1, 1) from a 64-bit hash
__global__ void k_hash_fill(size_t total, uint64_t seed, double2* X) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  uint64_t z = seed + 0x9e3779b97f4a7c15ull * (e + 1);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  const double v = (double)((z * 0x2545f4914f6cdd1dull) >> 11) * (1.0 / 9007199254740992.0);
  X[e] = make_double2(2 * u - 1, 2 * v - 1);
}

// res[b] = |AX_b - theta_b X_b|^2
__global__ void __launch_bounds__(256) k_fresid(const double2* __restrict__ X, const double2* __restrict__ AX,
                                                const double* theta, size_t n, double* res) {
  const int b = blockIdx.x;
  const double th = theta[b];
  double s = 0;
  for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
    const double2 x = X[(size_t)b * n + e], y = AX[(size_t)b * n + e];
    const double dr = y.x - th * x.x, di = y.y - th * x.y;
    s += dr * dr + di * di;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) res[b] = red[0];
}

}  // namespace

// fields as flat FP64 blocks: column a of a block is Field data + a * n, n = 12 Vh
static Field block_field(double2* base, int m, int Vh) {
  Field f;
  f.data = base;
  f.prec = DLMA_FP64;
  f.nrhs = m;
  f.Vh = Vh;
  return f;
}

struct DiracEig {
  dlma_ctx* ctx;
  int m, Vh;
  size_t n;
  double2 *X, *AX, *Y, *Yp, *Yn, *T1, *T2, *G, *H, *C, *gwork;
  double *theta, *res;
  int* dropped;
};

// AX = Dhat^dag Dhat X on m columns
static dlma_status apply_A(DiracEig& E, double2* X, double2* AX, int m) {
  Field in = block_field(X, m, E.Vh), t1 = block_field(E.T1, m, E.Vh), t2 = block_field(E.T2, m, E.Vh),
        out = block_field(AX, m, E.Vh);
  Field odd = block_field(E.Yn, m, E.Vh);   // odd-site work field of the Schur applications
  TRY(schur_apply(E.ctx, in, odd, t2, 0, nullptr, nullptr));
  TRY(schur_apply(E.ctx, t2, odd, out, 1, nullptr, nullptr));
  (void)t1;
  return DLMA_OK;
}

static dlma_status gram(DiracEig& E, const double2* X, const double2* Y, int ma, int mb, double2* G) {
  k_fgram<<<dim3(ma, mb), 256, 0, E.ctx->stream>>>(X, Y, ma, mb, E.n, G);
  dlma_ctx* ctx = E.ctx;
  CHECK_LAUNCH();
  return DLMA_OK;
}

static dlma_status rotate(DiracEig& E, const double2* X, const double2* C, int ma, int mb, double2* Y) {
  dlma_ctx* ctx = E.ctx;
  k_frot<<<dim3((unsigned)((E.n + 255) / 256), mb), 256, 0, ctx->stream>>>(X, C, ma, mb, E.n, Y);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// Rayleigh-Ritz of the hermitian operator whose images of X are in AX: X <- X C,
// AX <- AX C, theta ascending
static dlma_status rayleigh_ritz(DiracEig& E, double2* X, double2* AX, int m) {
  dlma_ctx* ctx = E.ctx;
  TRY(gram(E, X, X, m, m, E.G));
  TRY(gram(E, X, AX, m, m, E.H));
  size_t sm = 0;
  const int place = lma_small::small_rr_place<double>(m, &sm);
  if (sm)
    CU(cudaFuncSetAttribute(lma_small::k_small_rr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  CU(cudaMemsetAsync(E.dropped, 0, sizeof(int), ctx->stream));
  lma_small::k_small_rr<double><<<1, 256, sm, ctx->stream>>>(E.G, E.H, m, E.C, E.theta, (Cx<double>*)E.gwork, place,
                                                             E.dropped, 1e-24);
  CHECK_LAUNCH();
  TRY(rotate(E, X, E.C, m, m, E.Y));
  CU(cudaMemcpyAsync(X, E.Y, sizeof(double2) * E.n * m, cudaMemcpyDeviceToDevice, ctx->stream));
  TRY(rotate(E, AX, E.C, m, m, E.Y));
  CU(cudaMemcpyAsync(AX, E.Y, sizeof(double2) * E.n * m, cudaMemcpyDeviceToDevice, ctx->stream));
  return DLMA_OK;
}

extern "C" dlma_status dlma_dirac_eigs(dlma_ctx* ctx, int N, double tol, double* evals, double* evecs,
                                       dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge || !ctx->have_params) return set_err(ctx, DLMA_ERR_STATE, "gauge / params not set");
  const int Vh = ctx->g.Vh;
  const size_t n = (size_t)12 * Vh;
  int m = N + std::max(8, N);
  m += m & 1;
  if (!evals || N < 1 || !(tol > 0) || (size_t)m > n / 2 || m > lma_small::kSmallMaxM - 2)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_dirac_eigs (N %d, block %d)", N, m);
  CU(cudaSetDevice(ctx->device));
  DiracEig E;
  E.ctx = ctx;
  E.m = m;
  E.Vh = Vh;
  E.n = n;
  double2* blk;
  TRY(workT(ctx, WS_EIG_X, n * m * 7, &blk));
  E.X = blk;
  E.AX = blk + n * m;
  E.Y = blk + 2 * n * m;
  E.Yp = blk + 3 * n * m;
  E.Yn = blk + 4 * n * m;
  E.T1 = blk + 5 * n * m;
  E.T2 = blk + 6 * n * m;
  TRY(workT(ctx, WS_EIG_G, (size_t)3 * m * m, &E.G));
  E.H = E.G + (size_t)m * m;
  E.C = E.H + (size_t)m * m;
  TRY(workT(ctx, WS_EIG_S, (size_t)3 * m * (m + 1), &E.gwork));
  double* aux;
  TRY(workT(ctx, WS_EIG_AUX, (size_t)2 * m + 16, &aux));
  E.theta = aux;
  E.res = aux + m;
  E.dropped = (int*)(aux + 2 * m);
  const size_t tot = n * m;
  const unsigned nbk = (unsigned)((tot + 255) / 256);
  // spectral bound of Dhat^dag Dhat: power iteration on one column, with a margin
  double lmax = 0;
  {
    k_hash_fill<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, 0x1a3c5e7ull, E.X);
    CHECK_LAUNCH();
    std::vector<double2> hv(1);
    double nrm_prev = 0;
    for (int it = 0; it < 40; it++) {
      TRY(apply_A(E, E.X, E.AX, 1));
      TRY(gram(E, E.AX, E.AX, 1, 1, E.G));
      TRY(gram(E, E.X, E.X, 1, 1, E.H));
      double2 ga, gx;
      CU(cudaMemcpyAsync(&ga, E.G, sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaMemcpyAsync(&gx, E.H, sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaStreamSynchronize(ctx->stream));
      const double r = sqrt(ga.x / gx.x);
      lmax = std::max(lmax, r);
      const double s = 1.0 / sqrt(ga.x);
      k_cheb<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, E.AX, E.X, nullptr, s, 0.0, 0.0, E.X);
      CHECK_LAUNCH();
      if (it > 5 && fabs(r - nrm_prev) < 1e-3 * r) break;
      nrm_prev = r;
    }
    lmax *= 1.1;
  }
  // start block, first Rayleigh-Ritz
  k_hash_fill<<<nbk, 256, 0, ctx->stream>>>(tot, 0x5eed2201ull + (uint64_t)N, E.X);
  CHECK_LAUNCH();
  TRY(apply_A(E, E.X, E.AX, m));
  TRY(rayleigh_ritz(E, E.X, E.AX, m));
  std::vector<double> th(m), rs(m);
  bool conv = false;
  int it = 0;
  const int degree = 16, max_it = 400;
  double worst = 0;
  for (; it < max_it; it++) {
    k_fresid<<<m, 256, 0, ctx->stream>>>(E.X, E.AX, E.theta, n, E.res);
    CHECK_LAUNCH();
    CU(cudaMemcpyAsync(th.data(), E.theta, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(rs.data(), E.res, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    worst = 0;
    for (int k = 0; k < N; k++) worst = std::max(worst, sqrt(rs[k]) / lmax);
    if (!(worst == worst)) return set_err(ctx, DLMA_ERR_NONFINITE, "NaN in the Dirac eigensolver");
    if (worst <= 0.01 * tol) { conv = true; break; }
    // Chebyshev filter damping [theta_max, lmax]
    double a = th[m - 1];
    if (!(a < lmax)) a = 0.5 * (th[0] + lmax);
    const double e = 0.5 * (lmax - a), c = 0.5 * (lmax + a);
    // Y1 = (A X - c X) / e ; Yk = 2 (A Y_{k-1} - c Y_{k-1}) / e - Y_{k-2}
    k_cheb<<<nbk, 256, 0, ctx->stream>>>(tot, E.AX, E.X, nullptr, 1.0 / e, -c / e, 0.0, E.Y);
    CHECK_LAUNCH();
    CU(cudaMemcpyAsync(E.Yp, E.X, sizeof(double2) * tot, cudaMemcpyDeviceToDevice, ctx->stream));
    for (int k = 2; k <= degree; k++) {
      TRY(apply_A(E, E.Y, E.AX, m));
      k_cheb<<<nbk, 256, 0, ctx->stream>>>(tot, E.AX, E.Y, E.Yp, 2.0 / e, -2.0 * c / e, -1.0, E.X);
      CHECK_LAUNCH();
      std::swap(E.Yp, E.Y);   // Yp <- Y_{k-1}
      std::swap(E.Y, E.X);    // Y <- Y_k ; X is free
    }
    CU(cudaMemcpyAsync(E.X, E.Y, sizeof(double2) * tot, cudaMemcpyDeviceToDevice, ctx->stream));
    TRY(apply_A(E, E.X, E.AX, m));
    TRY(rayleigh_ritz(E, E.X, E.AX, m));
  }
  if (!conv)
    return set_err(ctx, DLMA_ERR_NOT_CONVERGED, "Dirac eigensolver at %.3g, not %.3g, after %d iterations", worst,
                   0.01 * tol, it);
  // Rayleigh-Ritz of Qhat = g5 Dhat in the span of the N lowest Qhat^2 pairs
  {
    Field in = block_field(E.X, N, Vh), odd = block_field(E.Yn, N, Vh), out = block_field(E.AX, N, Vh);
    TRY(schur_apply(ctx, in, odd, out, 0, nullptr, nullptr));
    k_g5<<<(unsigned)((n * N + 255) / 256), 256, 0, ctx->stream>>>(n * N, Vh, E.AX);
    CHECK_LAUNCH();
    TRY(rayleigh_ritz(E, E.X, E.AX, N));
    k_fresid<<<N, 256, 0, ctx->stream>>>(E.X, E.AX, E.theta, n, E.res);
    CHECK_LAUNCH();
  }
  CU(cudaMemcpyAsync(th.data(), E.theta, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(rs.data(), E.res, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  // order by |lambda| (ties: ascending lambda)
  std::vector<int> ord(N);
  for (int k = 0; k < N; k++) ord[k] = k;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return fabs(th[a]) < fabs(th[b]); });
  double qworst = 0;
  for (int k = 0; k < N; k++) qworst = std::max(qworst, sqrt(rs[k]) / std::max(1.0, fabs(th[k])));
  // cache the modes in |lambda| order: a permutation rotation
  std::vector<double2> perm((size_t)N * N, make_double2(0, 0));
  for (int k = 0; k < N; k++) perm[(size_t)ord[k] * N + k] = make_double2(1, 0);
  CU(cudaMemcpyAsync(E.C, perm.data(), sizeof(double2) * N * N, cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->dirac_N != N || !ctx->dirac_V) {
    if (ctx->dirac_V) cudaFree(ctx->dirac_V);
    ctx->dirac_V = nullptr;
    ctx->dirac_N = 0;
    CU(cudaMalloc(&ctx->dirac_V, sizeof(double2) * n * N));
  }
  TRY(rotate(E, E.X, E.C, N, N, ctx->dirac_V));
  ctx->dirac_N = N;
  for (int k = 0; k < N; k++) evals[k] = th[ord[k]];
  if (evecs) {
    Field f = block_field(ctx->dirac_V, N, Vh);
    double* dst = evecs;
    const size_t bytes = sizeof(double2) * n * N;
    if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_OUT, bytes / 8, &dst));
    TRY(unpack_parity(ctx, f, 0, 0, dst));
    if (mem == DLMA_MEM_HOST) TRY(copy_out(ctx, evecs, dst, bytes, mem));
  }
  CU(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < kTimingSlots; i++) ctx->timing[i] = 0;
  ctx->timing[1] = it;
  if (qworst > tol)
    return set_err(ctx, DLMA_ERR_NOT_CONVERGED, "Dirac eigenpairs at residual %.3g, not %.3g", qworst, tol);
  return DLMA_OK;
}

extern "C" dlma_status dlma_dirac_project(dlma_ctx* ctx, const double* in, double* out, int nrhs, int conj_g5,
                                          dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!in || !out || nrhs < 1) return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_dirac_project");
  if (!ctx->dirac_V || ctx->dirac_N < 1) return set_err(ctx, DLMA_ERR_STATE, "no Dirac low modes: dlma_dirac_eigs first");
  CU(cudaSetDevice(ctx->device));
  const int Vh = ctx->g.Vh, N = ctx->dirac_N;
  const size_t n = (size_t)12 * Vh, bytes = sizeof(double2) * n * nrhs;
  const double* din;
  TRY(copy_in(ctx, WS_IN, in, bytes, mem, &din));
  double* dout = out;
  if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_OUT, bytes / 8, &dout));
  double2* blk;
  TRY(workT(ctx, WS_T0, n * nrhs * 2 + (size_t)N * nrhs, &blk));
  double2* F = blk;
  double2* Pf = blk + n * nrhs;
  double2* c = blk + 2 * n * nrhs;
  Field f = block_field(F, nrhs, Vh), pf = block_field(Pf, nrhs, Vh);
  TRY(pack_parity(ctx, din, 0, 0, f));
  if (conj_g5) {
    k_g5<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, ctx->stream>>>(n * nrhs, Vh, F);
    CHECK_LAUNCH();
  }
  // c[i][r] = <u_i, f_r>, Pf_r = sum_i u_i c[i][r]
  k_fgram<<<dim3(N, nrhs), 256, 0, ctx->stream>>>(ctx->dirac_V, F, N, nrhs, n, c);
  CHECK_LAUNCH();
  k_frot<<<dim3((unsigned)((n + 255) / 256), nrhs), 256, 0, ctx->stream>>>(ctx->dirac_V, c, N, nrhs, n, Pf);
  CHECK_LAUNCH();
  if (conj_g5) {
    k_g5<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, ctx->stream>>>(n * nrhs, Vh, Pf);
    CHECK_LAUNCH();
  }
  TRY(unpack_parity(ctx, pf, 0, 0, dout));
  TRY(copy_out(ctx, out, dout, bytes, mem));
  CU(cudaStreamSynchronize(ctx->stream));
  return DLMA_OK;
}
