// Context, gauge field set-up and the Sheikholeslami-Wohlert clover field.
//
// set_params builds T(x) = (4 + m0) + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} Fhat_{mu nu}(x)
// with Fhat = (Q_{mu nu} - Q_{nu mu}) / 8 from the four plaquette leaves (the
// O(a)-improved Wilson operator of the abstract and Sec. 2, m0-normalised),
// stores its two 6x6 chirality blocks per site and inverts them.
#include "common.cuh"
#include <math.h>

dlma_status set_err(dlma_ctx* ctx, dlma_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

dlma_status work(dlma_ctx* ctx, int slot, size_t bytes, void** out) {
  DevBuf& b = ctx->wb[slot];
  if (bytes == 0) bytes = 16;
  if (b.bytes < bytes) {
    if (b.p) {
      CU(cudaStreamSynchronize(ctx->stream));
      CU(cudaFree(b.p));
      ctx->work_bytes -= b.bytes;
      b.p = nullptr;
      b.bytes = 0;
    }
    if (ctx->memcap && bytes > ctx->memcap)
      return set_err(ctx, DLMA_ERR_OOM, "a work buffer of %zu bytes exceeds the memory cap", bytes);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return set_err(ctx, DLMA_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.bytes = bytes;
    ctx->work_bytes += bytes;
  }
  *out = b.p;
  return DLMA_OK;
}

dlma_status field_alloc(dlma_ctx* ctx, int slot, int prec, int nrhs, Field* f) {
  size_t per = field_bytes_per_rhs(prec, ctx->g.Vh);
  void* p;
  TRY(work(ctx, slot, per * nrhs + 256, &p));
  f->data = p;
  f->prec = prec;
  f->nrhs = nrhs;
  f->Vh = ctx->g.Vh;
  f->scale = prec == DLMA_FP16S ? (float*)((char*)p + (size_t)3 * ctx->g.Vh * 16 * nrhs) : nullptr;
  return DLMA_OK;
}

dlma_status copy_in(dlma_ctx* ctx, int slot, const double* p, size_t bytes, dlma_mem mem, const double** dev) {
  if (mem == DLMA_MEM_DEVICE) {
    *dev = p;
    return DLMA_OK;
  }
  void* d;
  TRY(work(ctx, slot, bytes, &d));
  CU(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *dev = (const double*)d;
  return DLMA_OK;
}

dlma_status copy_out(dlma_ctx* ctx, double* dst, const double* dev, size_t bytes, dlma_mem mem) {
  if (mem == DLMA_MEM_DEVICE) {
    if (dst != dev) CU(cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    return DLMA_OK;
  }
  CU(cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return DLMA_OK;
}

// ---------------------------------------------------------------------------
// 3x3 complex matrices
template <class R> struct M3 { Cx<R> a[3][3]; };

template <class R> __device__ __forceinline__ M3<R> mmul(const M3<R>& A, const M3<R>& B) {
  M3<R> C;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      Cx<R> s = cx<R>(0, 0);
#pragma unroll
      for (int k = 0; k < 3; k++) fma_acc(s, A.a[i][k], B.a[k][j]);
      C.a[i][j] = s;
    }
  return C;
}
template <class R> __device__ __forceinline__ M3<R> mdag(const M3<R>& A) {
  M3<R> C;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) C.a[i][j] = conj(A.a[j][i]);
  return C;
}
__device__ __forceinline__ M3<double> load_can(const double2* U, int s, int mu) {
  M3<double> m;
  const double2* p = U + ((size_t)s * 4 + mu) * 9;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    double2 v = p[i];
    m.a[i / 3][i % 3] = cx<double>(v.x, v.y);
  }
  return m;
}

// ---------------------------------------------------------------------------
// gauge conversion: canonical [V][4][3][3] -> even-odd SoA copies
__global__ void k_gauge_convert(Geom g, const double2* __restrict__ Ucan, double2* U64, float4* U32, float4* U32f,
                                uint4* U16a, uint2* U16b, double2* U3, float4* U3f, int* flag) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x = s % g.L, y = (s / g.L) % g.L, z = (s / (g.L * g.L)) % g.L, t = s / (g.L * g.L * g.L);
  int p = (x + y + z + t) & 1;
  int i = s >> 1;
  for (int mu = 0; mu < 4; mu++) {
    const double2* src = Ucan + ((size_t)s * 4 + mu) * 9;
    double2 e[9];
    bool bad = false;
    for (int k = 0; k < 9; k++) {
      e[k] = src[k];
      if (!isfinite(e[k].x) || !isfinite(e[k].y)) bad = true;
    }
    if (bad) atomicOr(flag, 1);
    size_t base = ((size_t)(p * 4 + mu));
    for (int k = 0; k < 9; k++) U64[(base * 9 + k) * g.Vh + i] = e[k];
    for (int q = 0; q < 3; q++)
      U32[(base * 3 + q) * g.Vh + i] = make_float4((float)e[2 * q].x, (float)e[2 * q].y,
                                                   (float)e[2 * q + 1].x, (float)e[2 * q + 1].y);
    for (int q = 0; q < 5; q++) {
      const double2 a = e[2 * q], b = 2 * q + 1 < 9 ? e[2 * q + 1] : make_double2(0, 0);
      U32f[(base * 5 + q) * g.Vh + i] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
    __half2 h[6];
    for (int k = 0; k < 6; k++) h[k] = __floats2half2_rn((float)e[k].x, (float)e[k].y);
    uint4 a;
    uint2 b;
    a.x = *(unsigned*)&h[0]; a.y = *(unsigned*)&h[1]; a.z = *(unsigned*)&h[2]; a.w = *(unsigned*)&h[3];
    b.x = *(unsigned*)&h[4]; b.y = *(unsigned*)&h[5];
    U16a[base * g.Vh + i] = a;
    U16b[base * g.Vh + i] = b;
    if (mu >= 1) {
      for (int k = 0; k < 9; k++) U3[((size_t)(mu - 1) * 9 + k) * g.V + s] = e[k];
      for (int q = 0; q < 3; q++)
        U3f[((size_t)(mu - 1) * 3 + q) * g.V + s] = make_float4((float)e[2 * q].x, (float)e[2 * q].y,
                                                               (float)e[2 * q + 1].x, (float)e[2 * q + 1].y);
    }
  }
}

// ---------------------------------------------------------------------------
// clover field
struct SigmaBlocks {
  // sig[plane][chirality][2][2] complex, planes (mu, nu) with mu < nu in the order
  // (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
  double re[6][2][2][2], im[6][2][2][2];
};

// Q_{mu nu}(x): sum of the four plaquette leaves at x, each traversed mu then nu
__device__ M3<double> leaves(const Geom& g, const double2* U, int s, int mu, int nu) {
  int x = s % g.L, y = (s / g.L) % g.L, z = (s / (g.L * g.L)) % g.L, t = s / (g.L * g.L * g.L);
  Coord c{x, y, z, t};
  int xpm = nbr_lex(g, c, mu, +1), xpn = nbr_lex(g, c, nu, +1);
  int xmm = nbr_lex(g, c, mu, -1), xmn = nbr_lex(g, c, nu, -1);
  Coord cm{xmm % g.L, (xmm / g.L) % g.L, (xmm / (g.L * g.L)) % g.L, xmm / (g.L * g.L * g.L)};
  Coord cp{xpm % g.L, (xpm / g.L) % g.L, (xpm / (g.L * g.L)) % g.L, xpm / (g.L * g.L * g.L)};
  int xmm_pn = nbr_lex(g, cm, nu, +1);
  int xmm_mn = nbr_lex(g, cm, nu, -1);
  int xpm_mn = nbr_lex(g, cp, nu, -1);
  M3<double> Um = load_can(U, s, mu), Un = load_can(U, s, nu);
  M3<double> q = mmul(mmul(Um, load_can(U, xpm, nu)), mmul(mdag(load_can(U, xpn, mu)), mdag(Un)));
  M3<double> l2 = mmul(mmul(Un, mdag(load_can(U, xmm_pn, mu))), mmul(mdag(load_can(U, xmm, nu)), load_can(U, xmm, mu)));
  M3<double> l3 = mmul(mmul(mdag(load_can(U, xmm, mu)), mdag(load_can(U, xmm_mn, nu))),
                       mmul(load_can(U, xmm_mn, mu), load_can(U, xmn, nu)));
  M3<double> l4 = mmul(mmul(mdag(load_can(U, xmn, nu)), load_can(U, xmn, mu)), mmul(load_can(U, xpm_mn, nu), mdag(Um)));
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) q.a[i][j] = q.a[i][j] + l2.a[i][j] + l3.a[i][j] + l4.a[i][j];
  return q;
}

// Gauss-Jordan inverse of a 6x6 complex matrix with partial pivoting; returns false if singular
__device__ bool inv6(Cx<double> A[6][6], Cx<double> B[6][6]) {
  double scale = 0;
  for (int i = 0; i < 6; i++)
    for (int j = 0; j < 6; j++) {
      B[i][j] = cx<double>(i == j ? 1.0 : 0.0, 0.0);
      scale = fmax(scale, sqrt(norm2(A[i][j])));
    }
  for (int c = 0; c < 6; c++) {
    int piv = c;
    double best = norm2(A[c][c]);
    for (int r = c + 1; r < 6; r++)
      if (norm2(A[r][c]) > best) { best = norm2(A[r][c]); piv = r; }
    if (!(sqrt(best) > 1e-13 * scale)) return false;
    if (piv != c)
      for (int j = 0; j < 6; j++) {
        Cx<double> tmp = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = tmp;
        tmp = B[c][j]; B[c][j] = B[piv][j]; B[piv][j] = tmp;
      }
    Cx<double> d = A[c][c];
    double dn = norm2(d);
    Cx<double> di = cx<double>(d.re / dn, -d.im / dn);
    for (int j = 0; j < 6; j++) { A[c][j] = A[c][j] * di; B[c][j] = B[c][j] * di; }
    for (int r = 0; r < 6; r++) {
      if (r == c) continue;
      Cx<double> f = A[r][c];
      for (int j = 0; j < 6; j++) {
        A[r][j] = A[r][j] - f * A[c][j];
        B[r][j] = B[r][j] - f * B[c][j];
      }
    }
  }
  return true;
}

// pack a hermitian 6x6 block into 36 reals: diag re (6), then lower triangle row-major (15 complex)
__device__ __forceinline__ void pack_block(Cx<double> A[6][6], double* out) {
  for (int i = 0; i < 6; i++) out[i] = A[i][i].re;
  int k = 6;
  for (int i = 1; i < 6; i++)
    for (int j = 0; j < i; j++) {
      out[k++] = 0.5 * (A[i][j].re + A[j][i].re);
      out[k++] = 0.5 * (A[i][j].im - A[j][i].im);
    }
}

__global__ void k_clover(Geom g, const double2* __restrict__ Ucan, SigmaBlocks sb, double m0, double csw,
                         double2* C64, double2* Ci64, float4* C32, float4* Ci32, uint4* C16, uint4* Ci16,
                         int* flag) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x = s % g.L, y = (s / g.L) % g.L, z = (s / (g.L * g.L)) % g.L, t = s / (g.L * g.L * g.L);
  int p = (x + y + z + t) & 1;
  int i = s >> 1;
  // Fhat for the six planes mu < nu
  Cx<double> F[6][3][3];
  int plane = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++) {
      M3<double> q = leaves(g, Ucan, s, mu, nu);
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) F[plane][a][b] = 0.125 * (q.a[a][b] - conj(q.a[b][a]));
      plane++;
    }
  double packed[72], packedi[72];
  bool ok = true;
  for (int ch = 0; ch < 2; ch++) {
    // A = (4 + m0) + c_sw (i/2) sum_{mu<nu} sigma^ch_{mu nu} (x) Fhat_{mu nu}
    Cx<double> A[6][6], B[6][6];
    for (int r = 0; r < 6; r++)
      for (int c = 0; c < 6; c++) A[r][c] = cx<double>(r == c ? 4.0 + m0 : 0.0, 0.0);
    for (int pl = 0; pl < 6; pl++)
      for (int s1 = 0; s1 < 2; s1++)
        for (int s2 = 0; s2 < 2; s2++) {
          Cx<double> sg = cx<double>(sb.re[pl][ch][s1][s2], sb.im[pl][ch][s1][s2]);
          Cx<double> f = 0.5 * csw * mul_i(sg);
          for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) A[s1 * 3 + a][s2 * 3 + b] = A[s1 * 3 + a][s2 * 3 + b] + f * F[pl][a][b];
        }
    pack_block(A, packed + 36 * ch);
    ok = ok && inv6(A, B);
    pack_block(B, packedi + 36 * ch);
  }
  if (!ok) atomicOr(flag, 2);
  for (int k = 0; k < 36; k++) {
    C64[((size_t)p * 36 + k) * g.Vh + i] = make_double2(packed[2 * k], packed[2 * k + 1]);
    Ci64[((size_t)p * 36 + k) * g.Vh + i] = make_double2(packedi[2 * k], packedi[2 * k + 1]);
  }
  for (int k = 0; k < 18; k++) {
    C32[((size_t)p * 18 + k) * g.Vh + i] = make_float4((float)packed[4 * k], (float)packed[4 * k + 1],
                                                       (float)packed[4 * k + 2], (float)packed[4 * k + 3]);
    Ci32[((size_t)p * 18 + k) * g.Vh + i] = make_float4((float)packedi[4 * k], (float)packedi[4 * k + 1],
                                                        (float)packedi[4 * k + 2], (float)packedi[4 * k + 3]);
  }
  for (int k = 0; k < 9; k++) {
    __half2 h[4], hi[4];
    for (int q = 0; q < 4; q++) {
      h[q] = __floats2half2_rn((float)packed[8 * k + 2 * q], (float)packed[8 * k + 2 * q + 1]);
      hi[q] = __floats2half2_rn((float)packedi[8 * k + 2 * q], (float)packedi[8 * k + 2 * q + 1]);
    }
    C16[((size_t)p * 9 + k) * g.Vh + i] = make_uint4(*(unsigned*)&h[0], *(unsigned*)&h[1], *(unsigned*)&h[2], *(unsigned*)&h[3]);
    Ci16[((size_t)p * 9 + k) * g.Vh + i] = make_uint4(*(unsigned*)&hi[0], *(unsigned*)&hi[1], *(unsigned*)&hi[2], *(unsigned*)&hi[3]);
  }
}

// gamma_mu (mu = 0 time, 1..3 space) in the chiral basis as [mu][row][col][re, im]:
// gamma_0 = -[[0, 1], [1, 0]], gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]
void gamma_matrices(double G[4][4][4][2]) {
  memset(G, 0, sizeof(double) * 4 * 4 * 4 * 2);
  // gamma_0 = -[[0, 1], [1, 0]]
  for (int a = 0; a < 2; a++) { G[0][a][a + 2][0] = -1; G[0][a + 2][a][0] = -1; }
  // sigma_k (Pauli) entries
  const double pr[3][2][2] = {{{0, 1}, {1, 0}}, {{0, 0}, {0, 0}}, {{1, 0}, {0, -1}}};
  const double pi[3][2][2] = {{{0, 0}, {0, 0}}, {{0, -1}, {1, 0}}, {{0, 0}, {0, 0}}};
  for (int k = 0; k < 3; k++)
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) {
        // upper-right block -i sigma_k, lower-left block i sigma_k
        G[k + 1][a][b + 2][0] = pi[k][a][b];
        G[k + 1][a][b + 2][1] = -pr[k][a][b];
        G[k + 1][a + 2][b][0] = -pi[k][a][b];
        G[k + 1][a + 2][b][1] = pr[k][a][b];
      }
}

// sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] in the chiral basis, split into its two 2x2 chirality blocks
static SigmaBlocks sigma_blocks() {
  double G[4][4][4][2];
  gamma_matrices(G);
  SigmaBlocks sb;
  int plane = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++) {
      double S[4][4][2];
      for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) {
          double re = 0, im = 0;
          for (int k = 0; k < 4; k++) {
            // gamma_mu gamma_nu - gamma_nu gamma_mu
            re += G[mu][r][k][0] * G[nu][k][c][0] - G[mu][r][k][1] * G[nu][k][c][1];
            im += G[mu][r][k][0] * G[nu][k][c][1] + G[mu][r][k][1] * G[nu][k][c][0];
            re -= G[nu][r][k][0] * G[mu][k][c][0] - G[nu][r][k][1] * G[mu][k][c][1];
            im -= G[nu][r][k][0] * G[mu][k][c][1] + G[nu][r][k][1] * G[mu][k][c][0];
          }
          // times i/2
          S[r][c][0] = -0.5 * im;
          S[r][c][1] = 0.5 * re;
        }
      for (int ch = 0; ch < 2; ch++)
        for (int a = 0; a < 2; a++)
          for (int b = 0; b < 2; b++) {
            sb.re[plane][ch][a][b] = S[2 * ch + a][2 * ch + b][0];
            sb.im[plane][ch][a][b] = S[2 * ch + a][2 * ch + b][1];
          }
      plane++;
    }
  return sb;
}

// the stencil's neighbour table (see dlma_ctx::nbr_tab)
__global__ void k_build_nbr(Geom g, int bc_t, int4* tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.Vh) return;
  for (int p = 0; p < 2; p++) {
    const Coord c = eo_coords(g, p, i);
    int v[8];
    for (int mu = 0; mu < 4; mu++) {
      v[2 * mu] = nbr_lex(g, c, mu, +1) >> 1;
      v[2 * mu + 1] = nbr_lex(g, c, mu, -1) >> 1;
    }
    if (bc_t) {
      if (c.t == g.T - 1) v[0] |= (int)0x80000000u;
      if (c.t == 0) v[1] |= (int)0x80000000u;
    }
    tab[((size_t)p * 2 + 0) * g.Vh + i] = make_int4(v[0], v[1], v[2], v[3]);
    tab[((size_t)p * 2 + 1) * g.Vh + i] = make_int4(v[4], v[5], v[6], v[7]);
  }
}

// dlma_index_tables: the compressed index of every site and the stencil's own
// neighbour table with the phase bit removed
__global__ void k_index_tables(Geom g, const int4* tab, int* eo_index, int* nbr) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < g.V) eo_index[s] = s >> 1;
  if (s < g.Vh) {
    for (int p = 0; p < 2; p++)
      for (int w = 0; w < 2; w++) {
        const int4 q = tab[((size_t)p * 2 + w) * g.Vh + s];
        const int v[4] = {q.x, q.y, q.z, q.w};
        for (int k = 0; k < 4; k++) nbr[((size_t)p * 8 + 4 * w + k) * g.Vh + s] = v[k] & 0x7fffffff;
      }
  }
}

// ---------------------------------------------------------------------------
// C ABI
static void free_all(dlma_ctx* ctx) {
  void* ptrs[] = {ctx->nbr_tab, ctx->Ucan, ctx->U64, ctx->U32, ctx->U32f, ctx->U16a, ctx->U16b, ctx->U3, ctx->U3f, ctx->C64, ctx->Ci64,
                  ctx->C32, ctx->Ci32, ctx->C16, ctx->Ci16, ctx->flag, ctx->eig_V};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ctx->ckpt) cudaFree(ctx->ckpt);
  if (ctx->dirac_V) cudaFree(ctx->dirac_V);
  for (int i = 0; i < WS_COUNT; i++)
    if (ctx->wb[i].p) cudaFree(ctx->wb[i].p);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
}

extern "C" dlma_status dlma_create(const dlma_lattice* lat, int device, void* cuda_stream, dlma_ctx** out) {
  if (!out || !lat) return DLMA_ERR_INVALID_ARG;
  *out = nullptr;
  if (lat->L < 2 || lat->T < 2 || (lat->L & 1) || (lat->T & 1)) return DLMA_ERR_INVALID_ARG;
  if ((double)lat->L * lat->L * lat->L * lat->T > 2147483647.0 / 16) return DLMA_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return DLMA_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) return DLMA_ERR_CUDA;
  dlma_ctx* ctx = new dlma_ctx();
  ctx->g.L = lat->L;
  ctx->g.T = lat->T;
  ctx->g.Vs = lat->L * lat->L * lat->L;
  ctx->g.V = ctx->g.Vs * lat->T;
  ctx->g.Vh = ctx->g.V / 2;
  ctx->bc_t = lat->bc_t ? 1 : 0;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->err[0] = 0;
  if (const char* e = getenv("DLMA_DF_EIGS")) ctx->df_eigs = atoi(e) != 0;
  if (!ctx->stream) {
    // the legacy default stream cannot be captured into graphs: use a blocking
    // stream of our own (ordered with the legacy default stream)
    if (cudaStreamCreate(&ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return DLMA_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  size_t V = ctx->g.V, Vh = ctx->g.Vh;
  bool ok = cudaMalloc(&ctx->Ucan, 4 * 9 * V * sizeof(double2)) == cudaSuccess &&
            cudaMalloc(&ctx->U64, 2 * 4 * 9 * Vh * sizeof(double2)) == cudaSuccess &&
            cudaMalloc(&ctx->U32, 2 * 4 * 3 * Vh * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&ctx->U32f, 2 * 4 * 5 * Vh * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&ctx->U16a, 2 * 4 * Vh * sizeof(uint4)) == cudaSuccess &&
            cudaMalloc(&ctx->U16b, 2 * 4 * Vh * sizeof(uint2)) == cudaSuccess &&
            cudaMalloc(&ctx->U3, 3 * 9 * V * sizeof(double2)) == cudaSuccess &&
            cudaMalloc(&ctx->U3f, 3 * 3 * V * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&ctx->C64, 2 * 36 * Vh * sizeof(double2)) == cudaSuccess &&
            cudaMalloc(&ctx->Ci64, 2 * 36 * Vh * sizeof(double2)) == cudaSuccess &&
            cudaMalloc(&ctx->C32, 2 * 18 * Vh * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&ctx->Ci32, 2 * 18 * Vh * sizeof(float4)) == cudaSuccess &&
            cudaMalloc(&ctx->C16, 2 * 9 * Vh * sizeof(uint4)) == cudaSuccess &&
            cudaMalloc(&ctx->Ci16, 2 * 9 * Vh * sizeof(uint4)) == cudaSuccess &&
            cudaMalloc(&ctx->flag, 16 * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&ctx->nbr_tab, 4 * Vh * sizeof(int4)) == cudaSuccess &&
            cudaMallocHost(&ctx->pinned, 1 << 20) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_all(ctx);
    delete ctx;
    return DLMA_ERR_OOM;
  }
  k_build_nbr<<<(ctx->g.Vh + 255) / 256, 256, 0, ctx->stream>>>(ctx->g, ctx->bc_t, ctx->nbr_tab);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    free_all(ctx);
    delete ctx;
    return DLMA_ERR_CUDA;
  }
  ctx->launches++;
  *out = ctx;
  return DLMA_OK;
}

extern "C" dlma_status dlma_destroy(dlma_ctx* ctx) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
  return DLMA_OK;
}

extern "C" const char* dlma_last_error(const dlma_ctx* ctx) { return ctx ? ctx->err : "null context"; }

extern "C" dlma_status dlma_release_workspace(dlma_ctx* ctx) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (int i = 0; i < WS_COUNT; i++) {
    if (ctx->wb[i].p) cudaFree(ctx->wb[i].p);
    ctx->wb[i].p = nullptr;
    ctx->wb[i].bytes = 0;
  }
  ctx->work_bytes = 0;
  return DLMA_OK;
}

extern "C" dlma_status dlma_set_memory_cap(dlma_ctx* ctx, uint64_t bytes) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  ctx->memcap = bytes;
  return DLMA_OK;
}

extern "C" uint64_t dlma_kernel_launches(const dlma_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" dlma_status dlma_set_solver(dlma_ctx* ctx, dlma_solver solver) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (solver != DLMA_SOLVER_CGNE && solver != DLMA_SOLVER_BICGSTAB)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "unknown solver %d", (int)solver);
  ctx->solver = solver;
  return DLMA_OK;
}

extern "C" dlma_status dlma_last_timing(const dlma_ctx* ctx, double* out, int n) {
  if (!ctx || !out || n < 0) return DLMA_ERR_INVALID_ARG;
  for (int i = 0; i < n; i++) out[i] = i < kTimingSlots ? ctx->timing[i] : 0.0;
  return DLMA_OK;
}

extern "C" uint64_t dlma_checkpoint_serial(const dlma_ctx* ctx) {
  return ctx && ctx->ckpt ? ctx->ckpt_serial : 0;
}

extern "C" dlma_status dlma_set_gauge(dlma_ctx* ctx, const double* links, dlma_mem mem) {
  if (!ctx || !links) return set_err(ctx, DLMA_ERR_INVALID_ARG, "null argument");
  CU(cudaSetDevice(ctx->device));
  size_t bytes = (size_t)ctx->g.V * 4 * 9 * 16;
  const double* dU;
  TRY(copy_in(ctx, WS_IN, links, bytes, mem, &dU));
  // keep a canonical copy for the clover build
  double2* Ucan = ctx->Ucan;
  CU(cudaMemcpyAsync(Ucan, dU, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CU(cudaMemsetAsync(ctx->flag, 0, 16 * sizeof(int), ctx->stream));
  int nb = (ctx->g.V + 255) / 256;
  k_gauge_convert<<<nb, 256, 0, ctx->stream>>>(ctx->g, Ucan, ctx->U64, ctx->U32, ctx->U32f, ctx->U16a, ctx->U16b,
                                               ctx->U3, ctx->U3f, ctx->flag);
  CHECK_LAUNCH();
  int h = 0;
  CU(cudaMemcpyAsync(&h, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->have_params = false;
  ctx->eig_N = 0;
  ctx->dirac_N = 0;
  ctx->gauge_gen++;
  if (h & 1) {
    ctx->have_gauge = false;
    return set_err(ctx, DLMA_ERR_NONFINITE, "gauge field holds NaN or Inf");
  }
  ctx->have_gauge = true;
  return DLMA_OK;
}

extern "C" dlma_status dlma_set_params(dlma_ctx* ctx, double m0, double c_sw) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge) return set_err(ctx, DLMA_ERR_STATE, "dlma_set_params before dlma_set_gauge");
  if (!isfinite(m0) || !isfinite(c_sw)) return set_err(ctx, DLMA_ERR_INVALID_ARG, "non-finite m0 / c_sw");
  CU(cudaSetDevice(ctx->device));
  double2* Ucan = ctx->Ucan;
  SigmaBlocks sb = sigma_blocks();
  CU(cudaMemsetAsync(ctx->flag, 0, 16 * sizeof(int), ctx->stream));
  int nb = (ctx->g.V + 127) / 128;
  k_clover<<<nb, 128, 0, ctx->stream>>>(ctx->g, Ucan, sb, m0, c_sw, ctx->C64, ctx->Ci64, ctx->C32, ctx->Ci32,
                                        ctx->C16, ctx->Ci16, ctx->flag);
  CHECK_LAUNCH();
  int h = 0;
  CU(cudaMemcpyAsync(&h, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (h & 2) {
    ctx->have_params = false;
    return set_err(ctx, DLMA_ERR_SINGULAR, "a clover block is singular");
  }
  ctx->m0 = m0;
  ctx->csw = c_sw;
  ctx->have_params = true;
  ctx->dirac_N = 0;     // the Dirac low modes belong to the previous operator
  return DLMA_OK;
}

extern "C" dlma_status dlma_index_tables(dlma_ctx* ctx, int32_t* eo_index, int32_t* nbr) {
  if (!ctx || !eo_index || !nbr) return set_err(ctx, DLMA_ERR_INVALID_ARG, "null argument");
  CU(cudaSetDevice(ctx->device));
  int *d_eo, *d_nbr;
  TRY(workT(ctx, WS_T0, (size_t)ctx->g.V, &d_eo));
  TRY(workT(ctx, WS_T1, (size_t)16 * ctx->g.Vh, &d_nbr));
  k_index_tables<<<(ctx->g.V + 255) / 256, 256, 0, ctx->stream>>>(ctx->g, ctx->nbr_tab, d_eo, d_nbr);
  CHECK_LAUNCH();
  CU(cudaMemcpyAsync(eo_index, d_eo, sizeof(int) * ctx->g.V, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(nbr, d_nbr, sizeof(int) * 16 * (size_t)ctx->g.Vh, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return DLMA_OK;
}
