// Distillation sources, V^dag psi projections and the correlator parts of
// Eqs. 2-4.
//
//   sources (text after Eq. 3, Eq. 4): v_k(t') (x) e_alpha; eta_r;
//     (1 - Box(t')) eta_r; gamma_5 gamma_k (1 - Box(t')) eta_r, k = 1..3
//   projection (Eq. 1): c_j(t)[alpha][k] = sum_{m,c} conj(v_k(m,c;t)) psi_j(m,t,alpha,c)
//   perambulator tau(t)[(k,alpha),(l,beta)] = c_{4l+beta}(t)[alpha][k]
//   C_dist(t)  = tr[g5 G tau G g5 tau^dag]                                  (Eq. 3)
//   C_mixed(t) = 1/N_r sum_r sum_{alpha,beta} (g5 G)_{alpha beta} sum_k conj(a_r[k,alpha]) c_r[k,beta]
//   C_rest(t)  = 1/N_r sum_r sum_{alpha,beta} (g5 G)_{alpha beta} M_r[alpha][beta] - C_mixed(t)
// with c_r the coefficients of phi_r, a_r those of the left vector chi_r and
// M_r[alpha][beta] = sum_{x in t} conj(chi_r(x,alpha)) . phi_r(x,beta): the
// Box(t) insertion at the sink only needs the projection coefficients, since
// Box is diagonal in spin.
//
// The source-side mixed term (the second mixed contribution of Eq. 2, Box at the
// source and 1 - Box at the sink) is exact, noise-free, from the distillation
// solutions phi^{(k,beta)} = D^-1 (v_k (x) e_beta): with Box(t') = sum_{k,beta}
// (v_k e_beta)(v_k e_beta)^dag,
//   C^{1,Box'}(t) = sum_{k,beta,beta'} (G g5)_{beta' beta} <phi^{(k,beta)}, g5 G phi^{(k,beta')}>_t
//   C_mixed_src(t) = C^{1,Box'}(t) - C_dist(t),
// and the total of Eq. 2 is C = C_rest + 2 C_mixed + C_dist.
#include "common.cuh"
#include <algorithm>

namespace {

struct SpinMats {
  // [0..3] g5 G for G = g5, g1, g2, g3; [4..7] G g5; [8..10] g5 g_k (k = 1..3)
  double re[11][4][4], im[11][4][4];
};

SpinMats spin_mats() {
  double G[4][4][4][2];
  gamma_matrices(G);
  // gamma_5 = g0 g1 g2 g3
  auto mul = [](const double a[4][4][2], const double b[4][4][2], double o[4][4][2]) {
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) {
        double r = 0, im = 0;
        for (int k = 0; k < 4; k++) {
          r += a[i][k][0] * b[k][j][0] - a[i][k][1] * b[k][j][1];
          im += a[i][k][0] * b[k][j][1] + a[i][k][1] * b[k][j][0];
        }
        o[i][j][0] = r;
        o[i][j][1] = im;
      }
  };
  double t1[4][4][2], t2[4][4][2], g5[4][4][2];
  mul(G[0], G[1], t1);
  mul(t1, G[2], t2);
  mul(t2, G[3], g5);
  const double(*ch[4])[4][2] = {g5, G[1], G[2], G[3]};
  SpinMats S;
  double o[4][4][2];
  for (int c = 0; c < 4; c++) {
    mul(g5, ch[c], o);
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) { S.re[c][i][j] = o[i][j][0]; S.im[c][i][j] = o[i][j][1]; }
    mul(ch[c], g5, o);
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) { S.re[4 + c][i][j] = o[i][j][0]; S.im[4 + c][i][j] = o[i][j][1]; }
  }
  for (int k = 0; k < 3; k++) {
    mul(g5, G[k + 1], o);
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) { S.re[8 + k][i][j] = o[i][j][0]; S.im[8 + k][i][j] = o[i][j][1]; }
  }
  return S;
}

// VT[t][(m*3 + c) * N + k] = V(t, k, m, c); V(t, k) at vector index t * st_t + k * st_k
__global__ void k_transpose_V(const double2* __restrict__ V, int st_t, int st_k, int Tsel, int t0, int N, int n,
                              double2* VT) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)Tsel * N * n;
  if (e >= tot) return;
  int k = e % N;
  size_t r = e / N;
  int mc = r % n;
  int t = r / n;
  VT[e] = V[((size_t)(t0 + t) * st_t + (size_t)k * st_k) * n + mc];
}

// coeff[j][t][alpha][k] = sum_{m,c} conj(V_t[k][m][c]) psi_j(site0(t) + m, alpha, c)
// Block (ntk, KW): threadIdx.x = mode k, threadIdx.y = a slice m = y, y + KW, ... of the
// timeslice's sites (the sum is split over KW warps so that enough warps keep the
// FP64 pipes busy), JB right-hand sides per block; the KW partial sums meet in
// shared memory.
constexpr int JB = 4;
__global__ void k_project(const double2* __restrict__ VT, int N, int Vs, int Tsel, const double2* __restrict__ psi,
                          size_t psi_stride_sites, int site_t0, int nrhs, double2* coeff) {
  extern __shared__ double2 pred[];   // [KW - 1][JB * 4][ntk]
  const int t = blockIdx.x, j0 = blockIdx.y * JB, k = threadIdx.x, w = threadIdx.y;
  const int KW = blockDim.y, ntk = blockDim.x;
  const bool on = k < N;
  Cx<double> acc[JB][4];
#pragma unroll
  for (int jj = 0; jj < JB; jj++)
#pragma unroll
    for (int a = 0; a < 4; a++) acc[jj][a] = cx<double>(0, 0);
  const double2* vt = VT + (size_t)t * 3 * Vs * N;
  const size_t site0 = (size_t)(site_t0 + t) * Vs;
  for (int m = w; m < Vs; m += KW) {
    Cx<double> v[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      double2 e = on ? vt[(size_t)(m * 3 + c) * N + k] : make_double2(0, 0);
      v[c] = cx<double>(e.x, e.y);
    }
#pragma unroll
    for (int jj = 0; jj < JB; jj++) {
      if (j0 + jj >= nrhs) break;
      const double2* p = psi + ((size_t)(j0 + jj) * psi_stride_sites + site0 + m) * 12;
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          double2 e = __ldg(p + a * 3 + c);
          fma_conj_acc(acc[jj][a], v[c], cx<double>(e.x, e.y));
        }
    }
  }
  if (w > 0) {
#pragma unroll
    for (int jj = 0; jj < JB; jj++)
#pragma unroll
      for (int a = 0; a < 4; a++)
        pred[((size_t)(w - 1) * JB * 4 + jj * 4 + a) * ntk + k] = make_double2(acc[jj][a].re, acc[jj][a].im);
  }
  __syncthreads();
  if (w != 0 || !on) return;
#pragma unroll
  for (int jj = 0; jj < JB; jj++) {
    if (j0 + jj >= nrhs) break;
#pragma unroll
    for (int a = 0; a < 4; a++) {
      Cx<double> s = acc[jj][a];
      for (int q = 1; q < KW; q++) {
        const double2 e = pred[((size_t)(q - 1) * JB * 4 + jj * 4 + a) * ntk + k];
        s.re += e.x;
        s.im += e.y;
      }
      coeff[(((size_t)(j0 + jj) * Tsel + t) * 4 + a) * N + k] = make_double2(s.re, s.im);
    }
  }
}

// pe[r][m][alpha][c] = eta - sum_k V[k][m][c] coeff[r][alpha][k]   ((1 - Box) eta on one timeslice)
__global__ void k_deproject(const double2* __restrict__ VT, int N, int Vs, const double2* __restrict__ eta,
                            const double2* __restrict__ coeff, int nn, double2* pe) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nn * Vs * 12) return;
  int c = e % 3, a = (e / 3) % 4;
  size_t m = (e / 12) % Vs, r = e / ((size_t)12 * Vs);
  Cx<double> s = cx<double>(eta[e].x, eta[e].y);
  for (int k = 0; k < N; k++) {
    double2 v = VT[(m * 3 + c) * N + k], q = coeff[(r * 4 + a) * N + k];
    s = s - cx<double>(v.x, v.y) * cx<double>(q.x, q.y);
  }
  pe[e] = make_double2(s.re, s.im);
}

// sources j in [j0, j0 + nb): b must be zeroed; writes the timeslice t_src part
__global__ void k_sources(int j0, int nb, int N, int Vs, int t_src, const double2* __restrict__ VT,
                          const double2* __restrict__ eta, const double2* __restrict__ pe, SpinMats S, double2* b,
                          size_t stride_sites) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nb * Vs) return;
  int m = e % Vs;
  int jl = e / Vs;
  int j = j0 + jl;
  double2* out = b + ((size_t)jl * stride_sites + (size_t)t_src * Vs + m) * 12;
  if (j < 4 * N) {
    int k = j / 4, a = j % 4;
    for (int c = 0; c < 3; c++) out[a * 3 + c] = VT[((size_t)m * 3 + c) * N + k];
    return;
  }
  int r = (j - 4 * N) / 5, kind = (j - 4 * N) % 5;
  const double2* src = (kind == 0 ? eta : pe) + ((size_t)r * Vs + m) * 12;
  if (kind <= 1) {
    for (int q = 0; q < 12; q++) out[q] = src[q];
    return;
  }
  const int mi = 8 + (kind - 2);   // g5 g_k
  for (int a = 0; a < 4; a++)
    for (int c = 0; c < 3; c++) {
      Cx<double> s = cx<double>(0, 0);
      for (int bb = 0; bb < 4; bb++)
        fma_acc(s, cx<double>(S.re[mi][a][bb], S.im[mi][a][bb]), cx<double>(src[bb * 3 + c].x, src[bb * 3 + c].y));
      out[a * 3 + c] = make_double2(s.re, s.im);
    }
}

// M[p][t][alpha][beta] = sum_{m in t, c} conj(chi(m, alpha, c)) phi(m, beta, c) for pairs p = (chi_idx, phi_idx)
__global__ void __launch_bounds__(256) k_spin_inner(const double2* __restrict__ psi, size_t stride_sites, int Vs,
                                                    const int* __restrict__ pairs, double2* M, int T) {
  const int t = blockIdx.x, p = blockIdx.y;
  const int ci = pairs[2 * p], fi = pairs[2 * p + 1];
  Cx<double> acc[16];
#pragma unroll
  for (int q = 0; q < 16; q++) acc[q] = cx<double>(0, 0);
  for (int m = threadIdx.x; m < Vs; m += blockDim.x) {
    const double2* x = psi + ((size_t)ci * stride_sites + (size_t)t * Vs + m) * 12;
    const double2* f = psi + ((size_t)fi * stride_sites + (size_t)t * Vs + m) * 12;
    Cx<double> xv[12], fv[12];
#pragma unroll
    for (int q = 0; q < 12; q++) {
      xv[q] = cx<double>(x[q].x, x[q].y);
      fv[q] = cx<double>(f[q].x, f[q].y);
    }
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++)
#pragma unroll
        for (int c = 0; c < 3; c++) fma_conj_acc(acc[a * 4 + b], xv[a * 3 + c], fv[b * 3 + c]);
  }
  __shared__ double red[2][256];
  for (int q = 0; q < 16; q++) {
    red[0][threadIdx.x] = acc[q].re;
    red[1][threadIdx.x] = acc[q].im;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        red[0][threadIdx.x] += red[0][threadIdx.x + o];
        red[1][threadIdx.x] += red[1][threadIdx.x + o];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) M[((size_t)p * T + t) * 16 + q] = make_double2(red[0][0], red[1][0]);
    __syncthreads();
  }
}

// C_dist[ch][t] from the distillation coefficient rows coeff[4l+beta][t][alpha][k]
__global__ void __launch_bounds__(256) k_cdist(const double2* __restrict__ coeff, int N, int T, SpinMats S,
                                               double2* out) {
  const int t = blockIdx.x, ch = blockIdx.y;
  Cx<double> acc = cx<double>(0, 0);
  for (int kl = threadIdx.x; kl < N * N; kl += blockDim.x) {
    const int k = kl / N, l = kl % N;
    Cx<double> tau[4][4];          // tau[alpha][beta] = coeff[4l+beta][t][alpha][k]
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++) {
        double2 e = coeff[(((size_t)(4 * l + b) * T + t) * 4 + a) * N + k];
        tau[a][b] = cx<double>(e.x, e.y);
      }
    // sum_{a,a',b,b'} A[a][a'] tau[a'][b] B[b][b'] conj(tau[a][b'])
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int bp = 0; bp < 4; bp++) {
        Cx<double> p = cx<double>(0, 0);
#pragma unroll
        for (int ap = 0; ap < 4; ap++)
#pragma unroll
          for (int b = 0; b < 4; b++) {
            Cx<double> ab = cx<double>(S.re[ch][a][ap], S.im[ch][a][ap]) * cx<double>(S.re[4 + ch][b][bp], S.im[4 + ch][b][bp]);
            fma_acc(p, ab, tau[ap][b]);
          }
        fma_acc(acc, p, conj(tau[a][bp]));
      }
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = acc.re;
  red[1][threadIdx.x] = acc.im;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(size_t)ch * T + t] = make_double2(red[0][0], red[1][0]);
}

// noise parts: rest/mixed[ch][t] from M[r][ch][t][16] and coefficient rows of chi / phi
__global__ void __launch_bounds__(128) k_noise_parts(const double2* __restrict__ M, const double2* __restrict__ coeff,
                                                     int N, int T, int nn, int row0, SpinMats S, double2* rest,
                                                     double2* mixed) {
  const int t = blockIdx.x, ch = blockIdx.y;
  Cx<double> mix = cx<double>(0, 0), full = cx<double>(0, 0);
  for (int e = threadIdx.x; e < nn * N; e += blockDim.x) {
    const int r = e / N, k = e % N;
    const int rphi = row0 + 5 * r, rchi = row0 + 5 * r + 1 + ch;
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) {
        Cx<double> A = cx<double>(S.re[ch][a][b], S.im[ch][a][b]);
        double2 ca = coeff[(((size_t)rchi * T + t) * 4 + a) * N + k];
        double2 cb = coeff[(((size_t)rphi * T + t) * 4 + b) * N + k];
        Cx<double> pr = conj(cx<double>(ca.x, ca.y)) * cx<double>(cb.x, cb.y);
        fma_acc(mix, A, pr);
        if (k == 0) {
          double2 mv = M[(((size_t)r * 4 + ch) * T + t) * 16 + a * 4 + b];
          fma_acc(full, A, cx<double>(mv.x, mv.y));
        }
      }
  }
  __shared__ double red[4][128];
  red[0][threadIdx.x] = mix.re;
  red[1][threadIdx.x] = mix.im;
  red[2][threadIdx.x] = full.re;
  red[3][threadIdx.x] = full.im;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 4; q++) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double inv = 1.0 / nn;
    mixed[(size_t)ch * T + t] = make_double2(red[0][0] * inv, red[1][0] * inv);
    rest[(size_t)ch * T + t] = make_double2((red[2][0] - red[0][0]) * inv, (red[3][0] - red[1][0]) * inv);
  }
}

// ---- colour x even-odd diluted wall sources, spin-explicit (Sec. 3) --------
// Piece d = 2 c + p of noise r keeps colour c and the sites of t' with
// (x + y + z + t') mod 2 = p.  Rows of the solution set after the 4N
// distillation rows: 4N + 48 r + 8 d + 4 kind + beta, kind 0: phi_{d,beta} =
// D^-1 (eta_d (x) e_beta), kind 1: phibar_{d,beta} = D^-1 ((1 - Box(t')) eta_d (x) e_beta).

// H[r * 6 + d][m][spin 0][c] = eta_d(m, c) (other spins zero): the pieces as
// spinor fields, so that the (1 - Box(t')) of the undiluted path applies unchanged
__global__ void k_dilute(const double2* __restrict__ eta, int nn, int L, int t_src, double2* H) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int Vs = L * L * L;
  if (e >= (size_t)nn * 6 * Vs) return;
  const int m = (int)(e % Vs);
  const int rd = (int)(e / Vs), r = rd / 6, d = rd % 6, c = d / 2, p = d % 2;
  const int x = m % L, y = (m / L) % L, z = m / (L * L);
  double2* out = H + e * 12;
#pragma unroll
  for (int q = 0; q < 12; q++) out[q] = make_double2(0, 0);
  if ((x + y + z + t_src) % 2 == p) out[c] = eta[((size_t)r * Vs + m) * 3 + c];
}

// noise rows j in [j0, j0 + nb) (all >= 4N): b zeroed beforehand, timeslice t_src written
__global__ void k_sources_dil(int j0, int nb, int N, int Vs, int t_src, const double2* __restrict__ H,
                              const double2* __restrict__ pe, double2* b, size_t stride_sites) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nb * Vs) return;
  const int m = (int)(e % Vs), jl = (int)(e / Vs);
  const int q = j0 + jl - 4 * N, r = q / 48, w = q % 48, d = w / 8, kind = (w % 8) / 4, beta = w % 4;
  const double2* src = (kind == 0 ? H : pe) + ((size_t)(r * 6 + d) * Vs + m) * 12;   // spin 0 of the piece
  double2* out = b + ((size_t)jl * stride_sites + (size_t)t_src * Vs + m) * 12;
#pragma unroll
  for (int c = 0; c < 3; c++) out[beta * 3 + c] = src[c];
}

// rest / mixed [ch][t] of the diluted estimator:
//   1/N_r sum_{r,d,beta,beta'} B[beta][beta'] sum_{a,b} A[a][b] (W - Wbox)[beta' a][beta b]
// W from the spin inner products M[(r, d, beta', beta)][t][a b], Wbox from the coefficients
__global__ void __launch_bounds__(128) k_noise_parts_dil(const double2* __restrict__ M,
                                                         const double2* __restrict__ coeff, int N, int T, int nn,
                                                         int row0, SpinMats S, double2* rest, double2* mixed) {
  const int t = blockIdx.x, ch = blockIdx.y;
  Cx<double> mix = cx<double>(0, 0), full = cx<double>(0, 0);
  const int per = 6 * 16 * N;                    // (d, beta', beta, k) per noise vector
  for (int e = threadIdx.x; e < nn * per; e += blockDim.x) {
    const int r = e / per, w = e % per;
    const int d = w / (16 * N), bq = (w / N) % 16, k = w % N;
    const int bp = bq / 4, bt = bq % 4;          // beta' (phibar), beta (phi)
    const Cx<double> Bv = cx<double>(S.re[4 + ch][bt][bp], S.im[4 + ch][bt][bp]);
    if (Bv.re == 0.0 && Bv.im == 0.0) continue;
    const int rphi = row0 + 48 * r + 8 * d + bt, rbar = row0 + 48 * r + 8 * d + 4 + bp;
    Cx<double> sm = cx<double>(0, 0), sf = cx<double>(0, 0);
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) {
        const Cx<double> A = cx<double>(S.re[ch][a][b], S.im[ch][a][b]);
        if (A.re == 0.0 && A.im == 0.0) continue;
        const double2 ca = coeff[(((size_t)rbar * T + t) * 4 + a) * N + k];
        const double2 cb = coeff[(((size_t)rphi * T + t) * 4 + b) * N + k];
        fma_acc(sm, A, conj(cx<double>(ca.x, ca.y)) * cx<double>(cb.x, cb.y));
        if (k == 0) {
          const double2 mv = M[((((size_t)r * 6 + d) * 16 + bq) * T + t) * 16 + a * 4 + b];
          fma_acc(sf, A, cx<double>(mv.x, mv.y));
        }
      }
    fma_acc(mix, Bv, sm);
    fma_acc(full, Bv, sf);
  }
  __shared__ double red[4][128];
  red[0][threadIdx.x] = mix.re;
  red[1][threadIdx.x] = mix.im;
  red[2][threadIdx.x] = full.re;
  red[3][threadIdx.x] = full.im;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 4; q++) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double inv = 1.0 / nn;
    mixed[(size_t)ch * T + t] = make_double2(red[0][0] * inv, red[1][0] * inv);
    rest[(size_t)ch * T + t] = make_double2((red[2][0] - red[0][0]) * inv, (red[3][0] - red[1][0]) * inv);
  }
}

// The spin matrices A = g5 G and B = G g5 of the four channels are permutations
// with phases (one nonzero per row and column): for channel ch, row a of A has its
// entry in column bOf[ch][a], and column beta of B its entry in row bpOf[ch][beta].
struct SrcPerm {
  int bOf[4][4], bpOf[4][4];
  double2 av[4][4], bv[4][4];
};
static bool src_perm(const SpinMats& S, SrcPerm* P) {
  for (int ch = 0; ch < 4; ch++)
    for (int i = 0; i < 4; i++) {
      int na = 0, nb = 0;
      for (int j = 0; j < 4; j++) {
        if (S.re[ch][i][j] != 0.0 || S.im[ch][i][j] != 0.0) {
          P->bOf[ch][i] = j;
          P->av[ch][i] = make_double2(S.re[ch][i][j], S.im[ch][i][j]);
          na++;
        }
        if (S.re[4 + ch][j][i] != 0.0 || S.im[4 + ch][j][i] != 0.0) {
          P->bpOf[ch][i] = j;
          P->bv[ch][i] = make_double2(S.re[4 + ch][j][i], S.im[4 + ch][j][i]);
          nb++;
        }
      }
      if (na != 1 || nb != 1) return false;
    }
  return true;
}

// Per mode k and timeslice t: sum_{beta,beta'} B[beta'][beta] sum_{x in t} sum_{a,b}
// A[a][b] conj(phi^{(k,beta)}(x,a,.)) . phi^{(k,beta')}(x,b,.) for the four channels.
// The four solutions of mode k are rows 4 k .. 4 k + 3 of psi (batch-relative).  One
// thread per (site, beta): it holds phi^{(k,beta)} and reads, per channel, the one
// phi^{(k,beta')} that B pairs with it (no branches on the spin structure).
__global__ void __launch_bounds__(128) k_src_box(const double2* __restrict__ psi, size_t stride_sites, int Vs,
                                                 SrcPerm P, int k0, double2* part, int T) {
  const int t = blockIdx.x, kl = blockIdx.y;
  const int bt = threadIdx.x & 3;
  Cx<double> acc[4];
#pragma unroll
  for (int ch = 0; ch < 4; ch++) acc[ch] = cx<double>(0, 0);
  for (int m = threadIdx.x >> 2; m < Vs; m += blockDim.x >> 2) {
    const size_t site = (size_t)t * Vs + m;
    Cx<double> ft[12];
    {
      const double2* p = psi + ((size_t)(4 * kl + bt) * stride_sites + site) * 12;
#pragma unroll
      for (int q = 0; q < 12; q++) {
        const double2 e = __ldg(p + q);
        ft[q] = cx<double>(e.x, e.y);
      }
    }
#pragma unroll
    for (int ch = 0; ch < 4; ch++) {
      const int bp = P.bpOf[ch][bt];
      const double2* pp = psi + ((size_t)(4 * kl + bp) * stride_sites + site) * 12;
      Cx<double> inner = cx<double>(0, 0);
#pragma unroll
      for (int a = 0; a < 4; a++) {
        const int b = P.bOf[ch][a];
        Cx<double> d = cx<double>(0, 0);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const double2 e = __ldg(pp + b * 3 + c);
          fma_conj_acc(d, ft[a * 3 + c], cx<double>(e.x, e.y));
        }
        fma_acc(inner, cx<double>(P.av[ch][a].x, P.av[ch][a].y), d);
      }
      fma_acc(acc[ch], cx<double>(P.bv[ch][bt].x, P.bv[ch][bt].y), inner);
    }
  }
  __shared__ double red[8][128];
#pragma unroll
  for (int ch = 0; ch < 4; ch++) {
    red[2 * ch][threadIdx.x] = acc[ch].re;
    red[2 * ch + 1][threadIdx.x] = acc[ch].im;
  }
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 8; q++) red[q][threadIdx.x] += red[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 4)
    part[((size_t)(k0 + kl) * 4 + threadIdx.x) * T + t] =
        make_double2(red[2 * threadIdx.x][0], red[2 * threadIdx.x + 1][0]);
}

// out [5][4][T]: dist, rest, mixed (in), then mixed_src = sum_k part[k] - dist and
// the total of Eq. 2, C = rest + 2 mixed + dist
__global__ void k_totals(const double2* __restrict__ part, int N, int T, double2* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4 * T) return;
  const double2 d = out[e], r = out[4 * T + e], mx = out[8 * T + e];
  double sr = 0, si = 0;
  for (int k = 0; k < N; k++) {
    const double2 v = part[(size_t)k * 4 * T + e];
    sr += v.x;
    si += v.y;
  }
  out[12 * T + e] = make_double2(sr - d.x, si - d.y);
  out[16 * T + e] = make_double2(r.x + 2.0 * mx.x + d.x, r.y + 2.0 * mx.y + d.y);
}

// plain stochastic estimator, undiluted noise: rows 4 r + q of the solutions are
// phi_r = D^-1 eta_r (q = 0) and chi_{r,k} = D^-1 g5 g_k eta_r (q = k);
//   C[ch][t] = 1/N_r sum_r sum_{a,b} (g5 G)_{ab} M_r[ch][t][a][b],
// M_r[ch] the spin inner products <chi, phi>_t (chi = phi_r for the pseudoscalar)
__global__ void k_plain_parts(const double2* __restrict__ M, int T, int nn, SpinMats S, double2* out) {
  const int t = blockIdx.x, ch = threadIdx.x;
  if (ch >= 4) return;
  Cx<double> s = cx<double>(0, 0);
  for (int r = 0; r < nn; r++)
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) {
        const double2 mv = M[(((size_t)r * 4 + ch) * T + t) * 16 + a * 4 + b];
        fma_acc(s, cx<double>(S.re[ch][a][b], S.im[ch][a][b]), cx<double>(mv.x, mv.y));
      }
  out[(size_t)ch * T + t] = make_double2(s.re / nn, s.im / nn);
}

// plain stochastic estimator, diluted wall sources: rows 24 r + 4 d + beta are
// phi_{d,beta} = D^-1 (eta_d (x) e_beta);
//   C[ch][t] = 1/N_r sum_{r,d} sum_{beta,beta'} B[beta][beta'] sum_{a,b} A[a][b] W[beta' a][beta b],
// W from the spin inner products <phi_{d,beta'}, phi_{d,beta}>_t
__global__ void k_plain_parts_dil(const double2* __restrict__ M, int T, int nn, SpinMats S, double2* out) {
  const int t = blockIdx.x, ch = threadIdx.x;
  if (ch >= 4) return;
  Cx<double> s = cx<double>(0, 0);
  for (int r = 0; r < nn; r++)
    for (int d = 0; d < 6; d++)
      for (int bq = 0; bq < 16; bq++) {
        const int bp = bq / 4, bt = bq % 4;
        const Cx<double> Bv = cx<double>(S.re[4 + ch][bt][bp], S.im[4 + ch][bt][bp]);
        if (Bv.re == 0.0 && Bv.im == 0.0) continue;
        Cx<double> sf = cx<double>(0, 0);
        for (int a = 0; a < 4; a++)
          for (int b = 0; b < 4; b++) {
            const double2 mv = M[((((size_t)r * 6 + d) * 16 + bq) * T + t) * 16 + a * 4 + b];
            fma_acc(sf, cx<double>(S.re[ch][a][b], S.im[ch][a][b]), cx<double>(mv.x, mv.y));
          }
        fma_acc(s, Bv, sf);
      }
  out[(size_t)ch * T + t] = make_double2(s.re / nn, s.im / nn);
}

// plain estimator sources, undiluted: row 4 r + q = eta_r (q = 0) or g5 g_q eta_r
__global__ void k_sources_plain(int j0, int nb, int Vs, int t_src, const double2* __restrict__ eta, SpinMats S,
                                double2* b, size_t stride_sites) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nb * Vs) return;
  const int m = (int)(e % Vs), jl = (int)(e / Vs), j = j0 + jl, r = j / 4, q = j % 4;
  const double2* src = eta + ((size_t)r * Vs + m) * 12;
  double2* out = b + ((size_t)jl * stride_sites + (size_t)t_src * Vs + m) * 12;
  if (q == 0) {
    for (int i = 0; i < 12; i++) out[i] = src[i];
    return;
  }
  const int mi = 8 + (q - 1);   // g5 g_q
  for (int a = 0; a < 4; a++)
    for (int c = 0; c < 3; c++) {
      Cx<double> s = cx<double>(0, 0);
      for (int bb = 0; bb < 4; bb++)
        fma_acc(s, cx<double>(S.re[mi][a][bb], S.im[mi][a][bb]), cx<double>(src[bb * 3 + c].x, src[bb * 3 + c].y));
      out[a * 3 + c] = make_double2(s.re, s.im);
    }
}

// plain estimator sources, diluted: row 24 r + 4 d + beta = eta_d (x) e_beta (pieces H of k_dilute)
__global__ void k_sources_plain_dil(int j0, int nb, int Vs, int t_src, const double2* __restrict__ H, double2* b,
                                    size_t stride_sites) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nb * Vs) return;
  const int m = (int)(e % Vs), jl = (int)(e / Vs), j = j0 + jl, rd = j / 4, beta = j % 4;
  const double2* src = H + ((size_t)rd * Vs + m) * 12;   // spin 0 of the piece
  double2* out = b + ((size_t)jl * stride_sites + (size_t)t_src * Vs + m) * 12;
#pragma unroll
  for (int c = 0; c < 3; c++) out[beta * 3 + c] = src[c];
}

}  // namespace

// ---------------------------------------------------------------------------
// internal drivers
static dlma_status transpose_V(dlma_ctx* ctx, const double* V, int st_t, int st_k, int Tsel, int t0, int N,
                               double2** VT, int slot) {
  const int n = 3 * ctx->g.Vs;
  size_t tot = (size_t)Tsel * N * n;
  TRY(workT(ctx, slot, tot, VT));
  k_transpose_V<<<(tot + 255) / 256, 256, 0, ctx->stream>>>((const double2*)V, st_t, st_k, Tsel, t0, N, n, *VT);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// The projection runs on the tensor cores (tcproj.cu); DLMA_PROJECT_FP64=1 selects the
// FP64 CUDA-core kernel k_project instead (the comparison path of the tests).
static dlma_status project(dlma_ctx* ctx, const double2* VT, int N, int Tsel, const double* psi, size_t stride_sites,
                           int site_t0, int nrhs, double2* coeff) {
  const char* sel = getenv("DLMA_PROJECT_FP64");
  if (!(sel && atoi(sel) == 1)) return project_tc(ctx, VT, N, Tsel, psi, stride_sites, site_t0, nrhs, coeff);
  if (N > 256) return set_err(ctx, DLMA_ERR_INVALID_ARG, "N above 256 in the projection");
  const int nt = ((N + 31) / 32) * 32;
  // warps splitting the site sum: at most 4, partial sums within 40 KB of shared memory
  int kw = 4;
  while (kw > 1 && ((size_t)(kw - 1) * JB * 4 * nt * 16 > 40 * 1024 || nt * kw > 256)) kw--;
  const size_t smem = (size_t)(kw - 1) * JB * 4 * nt * 16;
  dim3 grid(Tsel, (nrhs + JB - 1) / JB);
  k_project<<<grid, dim3(nt, kw), smem, ctx->stream>>>(VT, N, ctx->g.Vs, Tsel, (const double2*)psi, stride_sites,
                                                      site_t0, nrhs, coeff);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// the same helpers for the backward pass (grad.cu)
dlma_status contract_transpose_V(dlma_ctx* ctx, const double* V, int st_t, int st_k, int Tsel, int t0, int N,
                                 double2** VT, int slot) {
  return transpose_V(ctx, V, st_t, st_k, Tsel, t0, N, VT, slot);
}
dlma_status contract_project(dlma_ctx* ctx, const double2* VT, int N, int Tsel, const double* psi,
                             size_t stride_sites, int site_t0, int nrhs, double2* coeff) {
  return project(ctx, VT, N, Tsel, psi, stride_sites, site_t0, nrhs, coeff);
}

// (1 - Box(t')) eta for all noise vectors: pe [nn][Vs][4][3]
static dlma_status project_noise(dlma_ctx* ctx, const double2* VTs, int N, const double* eta, int nn, double2** pe) {
  const int Vs = ctx->g.Vs;
  double2* co;
  TRY(workT(ctx, WS_CON2, (size_t)nn * 4 * N, &co));
  TRY(project(ctx, VTs, N, 1, eta, (size_t)Vs, 0, nn, co));
  TRY(workT(ctx, WS_ETA, (size_t)nn * Vs * 12, pe));
  size_t tot = (size_t)nn * Vs * 12;
  k_deproject<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(VTs, N, Vs, (const double2*)eta, co, nn, *pe);
  CHECK_LAUNCH();
  return DLMA_OK;
}

static dlma_status sources_range(dlma_ctx* ctx, int j0, int nb, int N, int t_src, const double2* VTs,
                                 const double* eta, const double2* pe, double* b) {
  const int Vs = ctx->g.Vs;
  CU(cudaMemsetAsync(b, 0, (size_t)nb * ctx->g.V * 12 * 16, ctx->stream));
  size_t tot = (size_t)nb * Vs;
  k_sources<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(j0, nb, N, Vs, t_src, VTs, (const double2*)eta, pe,
                                                        spin_mats(), (double2*)b, (size_t)ctx->g.V);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// noise-pair spin inner products for noise groups r in [r0, r0 + nr) whose 5 solutions start at row `base` of psi
static dlma_status spin_inner(dlma_ctx* ctx, const double* psi, int nr, int base, double2* M) {
  std::vector<int> hp(8 * nr);
  for (int r = 0; r < nr; r++)
    for (int ch = 0; ch < 4; ch++) {
      hp[2 * (4 * r + ch)] = base + 5 * r + 1 + ch;   // chi
      hp[2 * (4 * r + ch) + 1] = base + 5 * r;        // phi
    }
  int* dp;
  TRY(workT(ctx, WS_T2, hp.size(), &dp));
  CU(cudaMemcpyAsync(dp, hp.data(), sizeof(int) * hp.size(), cudaMemcpyHostToDevice, ctx->stream));
  dim3 grid(ctx->g.T, 4 * nr);
  k_spin_inner<<<grid, 256, 0, ctx->stream>>>((const double2*)psi, (size_t)ctx->g.V, ctx->g.Vs, dp, M, ctx->g.T);
  CHECK_LAUNCH();
  // stream-ordered use of the pinned-free host vector: wait before it goes out of scope
  CU(cudaStreamSynchronize(ctx->stream));
  return DLMA_OK;
}

// copy the five [4][T] parts (dist, rest, mixed, mixed_src, total) to the host outputs
static dlma_status fetch_parts(dlma_ctx* ctx, const double2* out, double* C_dist, double* C_rest, double* C_mixed,
                               double* C_mixed_src, double* C_full) {
  const int T = ctx->g.T;
  std::vector<double2> h(20 * T);
  CU(cudaMemcpyAsync(h.data(), out, sizeof(double2) * 20 * T, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  double* dst[5] = {C_dist, C_rest, C_mixed, C_mixed_src, C_full};
  for (int q = 0; q < 5; q++)
    if (dst[q]) memcpy(dst[q], h.data() + (size_t)q * 4 * T, sizeof(double2) * 4 * T);
  return DLMA_OK;
}

// exact source-side Box terms of the distillation rows 4 k0 .. 4 (k0 + nk) - 1, which
// are rows 0 .. 4 nk - 1 of psi: part[k][ch][t]
static dlma_status src_box(dlma_ctx* ctx, const double* psi, int k0, int nk, double2* part) {
  if (nk < 1) return DLMA_OK;
  SrcPerm P;
  if (!src_perm(spin_mats(), &P)) return set_err(ctx, DLMA_ERR_CUDA, "spin matrices are not permutations");
  k_src_box<<<dim3(ctx->g.T, nk), 128, 0, ctx->stream>>>((const double2*)psi, (size_t)ctx->g.V, ctx->g.Vs, P, k0,
                                                         part, ctx->g.T);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// C_dist, C_rest, C_mixed, C_mixed_src and the total C of Eq. 2 ([4][T] complex each,
// HOST; the last two may be NULL) from the projection coefficients, the noise-pair
// spin inner products and the source-side Box partials
static dlma_status finish_contract(dlma_ctx* ctx, int N, int nn, const double2* coeff, const double2* M,
                                   const double2* srcpart, double* C_dist, double* C_rest, double* C_mixed,
                                   double* C_mixed_src, double* C_full) {
  const int T = ctx->g.T;
  double2* out;
  TRY(workT(ctx, WS_CON, (size_t)20 * T, &out));
  SpinMats S = spin_mats();
  k_cdist<<<dim3(T, 4), 256, 0, ctx->stream>>>(coeff, N, T, S, out);
  CHECK_LAUNCH();
  if (nn > 0) {
    k_noise_parts<<<dim3(T, 4), 128, 0, ctx->stream>>>(M, coeff, N, T, nn, 4 * N, S, out + 4 * T, out + 8 * T);
    CHECK_LAUNCH();
  } else {
    CU(cudaMemsetAsync(out + 4 * T, 0, sizeof(double2) * 8 * T, ctx->stream));
  }
  k_totals<<<(4 * T + 127) / 128, 128, 0, ctx->stream>>>(srcpart, N, T, out);
  CHECK_LAUNCH();
  return fetch_parts(ctx, out, C_dist, C_rest, C_mixed, C_mixed_src, C_full);
}

// ---------------------------------------------------------------------------
// C ABI
extern "C" dlma_status dlma_make_sources(dlma_ctx* ctx, int t_src, int N, const double* V, int n_noise,
                                         const double* eta, double* b, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!V || !b || N < 1 || n_noise < 0 || (n_noise > 0 && !eta) || t_src < 0 || t_src >= ctx->g.T)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_make_sources");
  CU(cudaSetDevice(ctx->device));
  const int Vs = ctx->g.Vs, n = 3 * Vs;
  const double* dV;
  TRY(copy_in(ctx, WS_PROJ_V, V, (size_t)N * n * 16, mem, &dV));
  const double* deta = nullptr;
  if (n_noise) TRY(copy_in(ctx, WS_SRC, eta, (size_t)n_noise * Vs * 12 * 16, mem, &deta));
  double2* VT;
  TRY(transpose_V(ctx, dV, 0, 1, 1, 0, N, &VT, WS_PROJ_PART));
  double2* pe = nullptr;
  if (n_noise) TRY(project_noise(ctx, VT, N, deta, n_noise, &pe));
  const int J = 4 * N + 5 * n_noise;
  size_t bytes = (size_t)J * ctx->g.V * 12 * 16;
  double* db = b;
  if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_SOL, bytes / 8, &db));
  TRY(sources_range(ctx, 0, J, N, t_src, VT, deta, pe, db));
  TRY(copy_out(ctx, b, db, bytes, mem));
  CU(cudaStreamSynchronize(ctx->stream));
  return DLMA_OK;
}

extern "C" dlma_status dlma_project(dlma_ctx* ctx, int t, const double* V, int N, const double* psi, int nrhs,
                                    double* coeff, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!V || !psi || !coeff || N < 1 || nrhs < 1 || t < -1 || t >= ctx->g.T)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_project");
  CU(cudaSetDevice(ctx->device));
  const int n = 3 * ctx->g.Vs;
  const int Tsel = t < 0 ? ctx->g.T : 1;
  const double* dV;
  TRY(copy_in(ctx, WS_PROJ_V, V, (size_t)Tsel * N * n * 16, mem, &dV));
  const double* dpsi;
  TRY(copy_in(ctx, WS_SRC, psi, (size_t)nrhs * ctx->g.V * 12 * 16, mem, &dpsi));
  double2* VT;
  // V: [T][N] (t = -1) or [N] vectors
  TRY(transpose_V(ctx, dV, N, 1, Tsel, 0, N, &VT, WS_PROJ_PART));
  size_t cbytes = (size_t)nrhs * Tsel * 4 * N * 16;
  double* dc = coeff;
  if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_OUT, cbytes / 8, &dc));
  TRY(project(ctx, VT, N, Tsel, dpsi, (size_t)ctx->g.V, t < 0 ? 0 : t, nrhs, (double2*)dc));
  TRY(copy_out(ctx, coeff, dc, cbytes, mem));
  CU(cudaStreamSynchronize(ctx->stream));
  return DLMA_OK;
}

extern "C" dlma_status dlma_contract(dlma_ctx* ctx, int t_src, int N, const double* V, int n_noise,
                                     const double* phi, double* C_dist, double* C_rest, double* C_mixed,
                                     double* C_mixed_src, double* C_full, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!V || !phi || !C_dist || !C_rest || !C_mixed || N < 1 || n_noise < 0 || t_src < 0 || t_src >= ctx->g.T)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_contract");
  CU(cudaSetDevice(ctx->device));
  const int T = ctx->g.T, n = 3 * ctx->g.Vs;
  const int J = 4 * N + 5 * n_noise;
  const double* dV;
  TRY(copy_in(ctx, WS_PROJ_V, V, (size_t)T * N * n * 16, mem, &dV));
  const double* dphi;
  TRY(copy_in(ctx, WS_SRC, phi, (size_t)J * ctx->g.V * 12 * 16, mem, &dphi));
  double2* VT;
  TRY(transpose_V(ctx, dV, N, 1, T, 0, N, &VT, WS_PROJ_PART));
  double2* coeff;
  TRY(workT(ctx, WS_PROJ_C, (size_t)J * T * 4 * N, &coeff));
  TRY(project(ctx, VT, N, T, dphi, (size_t)ctx->g.V, 0, J, coeff));
  double2* M = nullptr;
  if (n_noise) {
    TRY(workT(ctx, WS_T1, (size_t)n_noise * 4 * T * 16, &M));
    TRY(spin_inner(ctx, dphi + (size_t)4 * N * ctx->g.V * 24, n_noise, 0, M));
  }
  double2* sp;
  TRY(workT(ctx, WS_CON2, (size_t)N * 4 * T, &sp));
  TRY(src_box(ctx, dphi, 0, N, sp));
  (void)t_src;
  return finish_contract(ctx, N, n_noise, coeff, M, sp, C_dist, C_rest, C_mixed, C_mixed_src, C_full);
}

// memory-bounded batch size of the correlator pipelines: two full complex128
// fields per right-hand side plus the solver's work space
static int pipeline_batch(dlma_ctx* ctx, int J, int granule) {
  const size_t V = ctx->g.V;
  const size_t per_rhs = V * 12 * 16 * 2 + field_bytes_per_rhs(DLMA_FP64, ctx->g.Vh) * 7 +
                         field_bytes_per_rhs(DLMA_FP32, ctx->g.Vh) * 8;
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  // the work buffers this pipeline reuses (sources, solutions, the solver's fields)
  // count as available: a repeated call must not size its batches by the memory its
  // own previous call still holds
  size_t held = 0;
  for (int s : {WS_SRC, WS_SOL, WS_SOLVE_B, WS_SOLVE_X64, WS_SOLVE_R64, WS_SOLVE_BH, WS_SOLVE_TMP64, WS_CG_X, WS_CG_R,
                WS_CG_P, WS_CG_PLO, WS_CG_Q, WS_CG_Z, WS_CG_TMP, WS_CG_RHS, WS_BI_S, WS_BI_R0, WS_RETRY_B, WS_RETRY_X})
    held += ctx->wb[s].bytes;
  const size_t budget = ctx->memcap ? ctx->memcap : (size_t)(0.8 * (double)(freeb + held));
  int nb = (int)std::max<size_t>((size_t)granule, std::min<size_t>((size_t)J, budget / per_rhs));
  return std::min(nb, J);
}

static dlma_status check_modes(dlma_ctx* ctx, int N) {
  if (ctx->eig_N != N) return set_err(ctx, DLMA_ERR_STATE, "no cached Laplacian modes for N = %d", N);
  for (int t = 0; t < ctx->g.T; t++)
    if (!ctx->eig_have[t]) return set_err(ctx, DLMA_ERR_STATE, "Laplacian modes of timeslice %d not computed", t);
  return DLMA_OK;
}

// timing slots of the correlator pipelines
constexpr int kPhSources = 1, kPhSolves = 2, kPhProject = 3, kPhContract = 4;

static void store_phases(dlma_ctx* ctx, PhaseTimer& pt, float total_ms) {
  for (int i = 0; i < kTimingSlots; i++) ctx->timing[i] = 0;
  ctx->timing[0] = total_ms;
  for (int q : {kPhSources, kPhSolves, kPhProject, kPhContract}) ctx->timing[q] = pt.acc[q];
}

extern "C" dlma_status dlma_correlators(dlma_ctx* ctx, int t_src, int N, int n_noise, const double* eta, double tol,
                                        dlma_prec inner, double* C_dist, double* C_rest, double* C_mixed,
                                        double* C_mixed_src, double* C_full, dlma_solve_info* info, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge || !ctx->have_params) return set_err(ctx, DLMA_ERR_STATE, "gauge / params not set");
  if (N < 1 || n_noise < 0 || (n_noise && !eta) || t_src < 0 || t_src >= ctx->g.T || !(tol > 0) || !C_dist ||
      !C_rest || !C_mixed)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_correlators");
  TRY(check_modes(ctx, N));
  CU(cudaSetDevice(ctx->device));
  const int T = ctx->g.T, Vs = ctx->g.Vs;
  const size_t V = ctx->g.V;
  const int J = 4 * N + 5 * n_noise;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, ctx->stream));
  PhaseTimer pt(ctx->stream);
  pt.enter(kPhSources);
  const double* deta = nullptr;
  if (n_noise) TRY(copy_in(ctx, WS_ETA + 0, eta, (size_t)n_noise * Vs * 12 * 16, mem, &deta));
  // modes: all timeslices from the cache ([N][T] vectors) and the source timeslice
  double2 *VT, *VTs;
  TRY(transpose_V(ctx, (const double*)ctx->eig_V, 1, T, T, 0, N, &VT, WS_PROJ_PART));
  TRY(transpose_V(ctx, (const double*)ctx->eig_V, 1, T, 1, t_src, N, &VTs, WS_PROJ_V));
  double2* pe = nullptr;
  if (n_noise) {
    // copy eta out of the slot project_noise reuses
    double2* etac;
    TRY(workT(ctx, WS_CON + 0, (size_t)n_noise * Vs * 12 + 20 * T, &etac));
    CU(cudaMemcpyAsync(etac, deta, (size_t)n_noise * Vs * 12 * 16, cudaMemcpyDeviceToDevice, ctx->stream));
    deta = (const double*)etac;
    TRY(project_noise(ctx, VTs, N, deta, n_noise, &pe));
  }
  double2* coeff;
  TRY(workT(ctx, WS_PROJ_C, (size_t)J * T * 4 * N, &coeff));
  double2* M = nullptr;
  if (n_noise) TRY(workT(ctx, WS_T1, (size_t)n_noise * 4 * T * 16, &M));
  double2* sp;
  TRY(workT(ctx, WS_CON2, (size_t)N * 4 * T + (size_t)n_noise * 4 * N, &sp));
  // project_noise keeps its coefficients at the start of WS_CON2: the partials follow them
  sp += (size_t)n_noise * 4 * N;
  const int nb = pipeline_batch(ctx, J, 5);
  const int nb4 = std::max(4, (nb / 4) * 4);
  double *b, *x;
  TRY(workT(ctx, WS_SRC, (size_t)std::max(nb, nb4) * V * 24, &b));
  TRY(workT(ctx, WS_SOL, (size_t)std::max(nb, nb4) * V * 24, &x));
  // checkpoint (for dlma_correlators_backward): distillation solutions and phi_r, phibar_r
  const int J2 = 4 * N + 2 * n_noise;
  const size_t fbytes = V * 12 * 16;
  if (ctx->checkpoint) {
    if (ctx->ckpt_J < J2) {
      if (ctx->ckpt) cudaFree(ctx->ckpt);
      ctx->ckpt = nullptr;
      ctx->ckpt_J = 0;
      if (cudaMalloc(&ctx->ckpt, (size_t)J2 * fbytes) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, DLMA_ERR_OOM, "checkpoint of %d solutions does not fit", J2);
      }
      ctx->ckpt_J = J2;
    }
    ctx->ckpt_N = N;
    ctx->ckpt_nn = n_noise;
    ctx->ckpt_tsrc = t_src;
    ctx->ckpt_m0 = ctx->m0;
    ctx->ckpt_csw = ctx->csw;
    ctx->ckpt_gauge_gen = ctx->gauge_gen;
    ctx->ckpt_eig_gen = ctx->eig_gen;
    ctx->ckpt_serial = ++ctx->ckpt_count;
  }
  dlma_status worst = DLMA_OK;
  // distillation rows in chunks of whole modes (4 spins), then noise rows in whole groups of 5
  int j0 = 0;
  while (j0 < J) {
    int cnt;
    if (j0 < 4 * N) cnt = std::min(nb4, 4 * N - j0);
    else cnt = std::max(5, (nb / 5) * 5), cnt = std::min(cnt, J - j0);
    pt.enter(kPhSources);
    TRY(sources_range(ctx, j0, cnt, N, t_src, VTs, deta, pe, b));
    pt.enter(kPhSolves);
    dlma_status s = solve_fields(ctx, b, x, cnt, tol, inner, info ? info + j0 : nullptr);
    if (s != DLMA_OK && s != DLMA_ERR_NOT_CONVERGED) return s;
    if (s != DLMA_OK) worst = s;
    pt.enter(kPhProject);
    TRY(project(ctx, VT, N, T, x, V, 0, cnt, coeff + (size_t)j0 * T * 4 * N));
    pt.enter(kPhContract);
    if (j0 >= 4 * N) {
      int r0 = (j0 - 4 * N) / 5;
      TRY(spin_inner(ctx, x, cnt / 5, 0, M + (size_t)r0 * 4 * T * 16));
    } else {
      TRY(src_box(ctx, x, j0 / 4, cnt / 4, sp));
    }
    if (ctx->checkpoint) {
      if (j0 < 4 * N) {
        CU(cudaMemcpyAsync(ctx->ckpt + (size_t)j0 * V * 24, x, (size_t)cnt * fbytes, cudaMemcpyDeviceToDevice,
                           ctx->stream));
      } else {
        const int r0 = (j0 - 4 * N) / 5;
        for (int r = 0; r < cnt / 5; r++)
          CU(cudaMemcpyAsync(ctx->ckpt + ((size_t)4 * N + 2 * (r0 + r)) * V * 24, x + (size_t)5 * r * V * 24,
                             2 * fbytes, cudaMemcpyDeviceToDevice, ctx->stream));
      }
    }
    j0 += cnt;
  }
  pt.enter(kPhContract);
  TRY(finish_contract(ctx, N, n_noise, coeff, M, sp, C_dist, C_rest, C_mixed, C_mixed_src, C_full));
  CU(cudaEventRecord(e1, ctx->stream));
  pt.mark(-1);
  CU(cudaStreamSynchronize(ctx->stream));
  pt.collect();
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  store_phases(ctx, pt, ms);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return worst;
}

// ---------------------------------------------------------------------------
// diluted wall sources (Sec. 3): 4N distillation solves + 48 per noise vector
extern "C" dlma_status dlma_correlators_diluted(dlma_ctx* ctx, int t_src, int N, int n_noise, const double* eta,
                                                double tol, dlma_prec inner, double* C_dist, double* C_rest,
                                                double* C_mixed, double* C_mixed_src, double* C_full,
                                                dlma_solve_info* info, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge || !ctx->have_params) return set_err(ctx, DLMA_ERR_STATE, "gauge / params not set");
  if (N < 1 || n_noise < 1 || !eta || t_src < 0 || t_src >= ctx->g.T || !(tol > 0) || !C_dist || !C_rest ||
      !C_mixed)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_correlators_diluted");
  TRY(check_modes(ctx, N));
  CU(cudaSetDevice(ctx->device));
  const int T = ctx->g.T, Vs = ctx->g.Vs, L = ctx->g.L;
  const size_t V = ctx->g.V;
  const int nn = n_noise, J = 4 * N + 48 * nn;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, ctx->stream));
  PhaseTimer pt(ctx->stream);
  pt.enter(kPhSources);
  const double* deta;
  TRY(copy_in(ctx, WS_T0, eta, (size_t)nn * Vs * 3 * 16, mem, &deta));
  double2* H;
  TRY(workT(ctx, WS_CON, (size_t)nn * 6 * Vs * 12, &H));
  {
    const size_t tot = (size_t)nn * 6 * Vs;
    k_dilute<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>((const double2*)deta, nn, L, t_src, H);
    CHECK_LAUNCH();
  }
  double2 *VT, *VTs;
  TRY(transpose_V(ctx, (const double*)ctx->eig_V, 1, T, T, 0, N, &VT, WS_PROJ_PART));
  TRY(transpose_V(ctx, (const double*)ctx->eig_V, 1, T, 1, t_src, N, &VTs, WS_PROJ_V));
  double2* pe;
  TRY(project_noise(ctx, VTs, N, (const double*)H, 6 * nn, &pe));
  double2* coeff;
  TRY(workT(ctx, WS_PROJ_C, (size_t)J * T * 4 * N, &coeff));
  double2* M;
  TRY(workT(ctx, WS_T1, (size_t)nn * 6 * 16 * T * 16, &M));
  double2* sp;
  TRY(workT(ctx, WS_CON2, (size_t)N * 4 * T + (size_t)6 * nn * 4 * N, &sp));
  sp += (size_t)6 * nn * 4 * N;
  const int nb = pipeline_batch(ctx, J, 48);
  const int nb4 = std::max(4, (nb / 4) * 4);
  double *b, *x;
  TRY(workT(ctx, WS_SRC, (size_t)std::max(nb, nb4) * V * 24, &b));
  TRY(workT(ctx, WS_SOL, (size_t)std::max(nb, nb4) * V * 24, &x));
  std::vector<int> hp;
  dlma_status worst = DLMA_OK;
  int j0 = 0;
  while (j0 < J) {
    int cnt;
    pt.enter(kPhSources);
    if (j0 < 4 * N) {
      cnt = std::min(nb4, 4 * N - j0);
      TRY(sources_range(ctx, j0, cnt, N, t_src, VTs, nullptr, nullptr, b));
    } else {
      cnt = std::min(std::max(48, (nb / 48) * 48), J - j0);
      CU(cudaMemsetAsync(b, 0, (size_t)cnt * V * 12 * 16, ctx->stream));
      const size_t tot = (size_t)cnt * Vs;
      k_sources_dil<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(j0, cnt, N, Vs, t_src, H, pe,
                                                                          (double2*)b, V);
      CHECK_LAUNCH();
    }
    pt.enter(kPhSolves);
    dlma_status st = solve_fields(ctx, b, x, cnt, tol, inner, info ? info + j0 : nullptr);
    if (st != DLMA_OK && st != DLMA_ERR_NOT_CONVERGED) return st;
    if (st != DLMA_OK) worst = st;
    pt.enter(kPhProject);
    TRY(project(ctx, VT, N, T, x, V, 0, cnt, coeff + (size_t)j0 * T * 4 * N));
    pt.enter(kPhContract);
    if (j0 >= 4 * N) {
      // spin inner products <phibar_{d,beta'}, phi_{d,beta}>_t of every piece in the batch
      const int r0 = (j0 - 4 * N) / 48, nr = cnt / 48;
      hp.assign((size_t)nr * 6 * 16 * 2, 0);
      for (int r = 0; r < nr; r++)
        for (int d = 0; d < 6; d++)
          for (int bq = 0; bq < 16; bq++) {
            const size_t pi = ((size_t)r * 6 + d) * 16 + bq;
            hp[2 * pi] = 48 * r + 8 * d + 4 + bq / 4;   // phibar_{d, beta'}
            hp[2 * pi + 1] = 48 * r + 8 * d + bq % 4;   // phi_{d, beta}
          }
      int* dp;
      TRY(workT(ctx, WS_T2, hp.size(), &dp));
      CU(cudaMemcpyAsync(dp, hp.data(), sizeof(int) * hp.size(), cudaMemcpyHostToDevice, ctx->stream));
      dim3 grid(T, nr * 6 * 16);
      k_spin_inner<<<grid, 256, 0, ctx->stream>>>((const double2*)x, V, Vs, dp, M + (size_t)r0 * 6 * 16 * T * 16, T);
      CHECK_LAUNCH();
      CU(cudaStreamSynchronize(ctx->stream));     // hp is reused by the next batch
    } else {
      TRY(src_box(ctx, x, j0 / 4, cnt / 4, sp));
    }
    j0 += cnt;
  }
  pt.enter(kPhContract);
  {
    double2* out;
    TRY(workT(ctx, WS_OUT, (size_t)20 * T, &out));
    SpinMats S = spin_mats();
    k_cdist<<<dim3(T, 4), 256, 0, ctx->stream>>>(coeff, N, T, S, out);
    CHECK_LAUNCH();
    k_noise_parts_dil<<<dim3(T, 4), 128, 0, ctx->stream>>>(M, coeff, N, T, nn, 4 * N, S, out + 4 * T, out + 8 * T);
    CHECK_LAUNCH();
    k_totals<<<(4 * T + 127) / 128, 128, 0, ctx->stream>>>(sp, N, T, out);
    CHECK_LAUNCH();
    CU(cudaEventRecord(e1, ctx->stream));
    TRY(fetch_parts(ctx, out, C_dist, C_rest, C_mixed, C_mixed_src, C_full));
  }
  pt.mark(-1);
  CU(cudaStreamSynchronize(ctx->stream));
  pt.collect();
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  store_phases(ctx, pt, ms);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return worst;
}

// ---------------------------------------------------------------------------
// plain stochastic estimator of C (no distillation; the comparison of Fig. 1)
extern "C" dlma_status dlma_correlators_plain(dlma_ctx* ctx, int t_src, int n_noise, const double* eta, int diluted,
                                              double tol, dlma_prec inner, double* C, dlma_solve_info* info,
                                              dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge || !ctx->have_params) return set_err(ctx, DLMA_ERR_STATE, "gauge / params not set");
  if (n_noise < 1 || !eta || !C || t_src < 0 || t_src >= ctx->g.T || !(tol > 0))
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_correlators_plain");
  CU(cudaSetDevice(ctx->device));
  const int T = ctx->g.T, Vs = ctx->g.Vs, L = ctx->g.L;
  const size_t V = ctx->g.V;
  const int nn = n_noise;
  const int per = diluted ? 24 : 4;          // solves per noise vector
  const int J = per * nn;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, ctx->stream));
  PhaseTimer pt(ctx->stream);
  pt.enter(kPhSources);
  const double* deta;
  TRY(copy_in(ctx, WS_T0, eta, (size_t)nn * Vs * (diluted ? 3 : 12) * 16, mem, &deta));
  double2* H = nullptr;
  if (diluted) {
    TRY(workT(ctx, WS_ETA, (size_t)nn * 6 * Vs * 12, &H));
    const size_t tot = (size_t)nn * 6 * Vs;
    k_dilute<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>((const double2*)deta, nn, L, t_src, H);
    CHECK_LAUNCH();
  } else {
    double2* ec;
    TRY(workT(ctx, WS_ETA, (size_t)nn * Vs * 12, &ec));
    CU(cudaMemcpyAsync(ec, deta, (size_t)nn * Vs * 12 * 16, cudaMemcpyDeviceToDevice, ctx->stream));
    deta = (const double*)ec;
  }
  const size_t npairs = diluted ? (size_t)nn * 6 * 16 : (size_t)nn * 4;
  double2* M;
  TRY(workT(ctx, WS_T1, npairs * T * 16, &M));
  const int nb = pipeline_batch(ctx, J, per);
  double *b, *x;
  TRY(workT(ctx, WS_SRC, (size_t)nb * V * 24, &b));
  TRY(workT(ctx, WS_SOL, (size_t)nb * V * 24, &x));
  SpinMats S = spin_mats();
  std::vector<int> hp;
  dlma_status worst = DLMA_OK;
  for (int j0 = 0; j0 < J;) {
    const int cnt = std::min(std::max(per, (nb / per) * per), J - j0);
    pt.enter(kPhSources);
    CU(cudaMemsetAsync(b, 0, (size_t)cnt * V * 12 * 16, ctx->stream));
    const size_t tot = (size_t)cnt * Vs;
    if (diluted)
      k_sources_plain_dil<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(j0, cnt, Vs, t_src, H,
                                                                                (double2*)b, V);
    else
      k_sources_plain<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(j0, cnt, Vs, t_src,
                                                                            (const double2*)deta, S, (double2*)b, V);
    CHECK_LAUNCH();
    pt.enter(kPhSolves);
    dlma_status st = solve_fields(ctx, b, x, cnt, tol, inner, info ? info + j0 : nullptr);
    if (st != DLMA_OK && st != DLMA_ERR_NOT_CONVERGED) return st;
    if (st != DLMA_OK) worst = st;
    pt.enter(kPhContract);
    // spin inner products: undiluted <chi_{r,ch}, phi_r>, chi = phi_r (ch 0) or row 4 r + ch;
    // diluted <phi_{d,beta'}, phi_{d,beta}> for every piece
    const int ng = cnt / per, g0 = j0 / per;
    hp.clear();
    for (int r = 0; r < ng; r++) {
      if (diluted) {
        for (int d = 0; d < 6; d++)
          for (int bq = 0; bq < 16; bq++) {
            hp.push_back(24 * r + 4 * d + bq / 4);
            hp.push_back(24 * r + 4 * d + bq % 4);
          }
      } else {
        for (int ch = 0; ch < 4; ch++) {
          hp.push_back(4 * r + ch);
          hp.push_back(4 * r);
        }
      }
    }
    int* dp;
    TRY(workT(ctx, WS_T2, hp.size(), &dp));
    CU(cudaMemcpyAsync(dp, hp.data(), sizeof(int) * hp.size(), cudaMemcpyHostToDevice, ctx->stream));
    const size_t moff = diluted ? (size_t)g0 * 6 * 16 : (size_t)g0 * 4;
    k_spin_inner<<<dim3(T, (unsigned)(hp.size() / 2)), 256, 0, ctx->stream>>>((const double2*)x, V, Vs, dp,
                                                                              M + moff * T * 16, T);
    CHECK_LAUNCH();
    CU(cudaStreamSynchronize(ctx->stream));     // hp is reused by the next batch
    j0 += cnt;
  }
  pt.enter(kPhContract);
  double2* out;
  TRY(workT(ctx, WS_OUT, (size_t)4 * T, &out));
  if (diluted) k_plain_parts_dil<<<T, 32, 0, ctx->stream>>>(M, T, nn, S, out);
  else k_plain_parts<<<T, 32, 0, ctx->stream>>>(M, T, nn, S, out);
  CHECK_LAUNCH();
  CU(cudaEventRecord(e1, ctx->stream));
  CU(cudaMemcpyAsync(C, out, sizeof(double2) * 4 * T, cudaMemcpyDeviceToHost, ctx->stream));
  pt.mark(-1);
  CU(cudaStreamSynchronize(ctx->stream));
  pt.collect();
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  store_phases(ctx, pt, ms);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return worst;
}
