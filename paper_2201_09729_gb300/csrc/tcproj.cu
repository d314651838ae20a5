// V(t)^dag psi projections (Eq. 1, Eq. 3) on the tensor cores, FP64-accurate.
//
// Per timeslice t the projection is the complex contraction
//   coeff[j][t][alpha][k] = sum_{kappa = (m, c)} conj(V_t[k][kappa]) psi_j(m, t, alpha, c),
// rows r = (j, alpha), columns k, contraction over kappa (3 L^3).  Written in real
// arithmetic with the contraction index kappa2 = 2 kappa + (0 re, 1 im):
//   A[r][kappa2]           = (re psi, im psi)
//   B[k][kappa2]           = (re v, im v)        -> re coeff
//   B[N + k][kappa2]       = (-im v, re v)       -> im coeff
//
// Split-precision scheme (in the family of Ozaki's error-free splitting): every
// row of A and of B is cut into chunks of 128 complex kappa; within a chunk each
// real x is written with the chunk's exponent e (|x| < 2^e) as
//   x = 2^(e - 5) sum_{i=1..8} d_i 64^-(i-1)  (+ a remainder below 2^(e - 47)),
// with signed digits |d_i| <= 32, exact in bf16.  The product of two values is
// sum_{i,j} d_i d'_j 2^(ex + ey - 10 - 6 (i + j - 2)); the pairs with
// i + j <= 9 are kept (36 of 64), grouped by class c = i + j - 2 (8 classes).
// A class sum over one chunk is an integer below 8 x 256 x 32^2 = 2^21, so the
// tensor core's FP32 accumulation of the bf16 products is exact; each class is
// scaled by its power of two and added to a double-float (hi, lo) accumulator.
// The result carries about 47 bits: relative to max |x| of a chunk the digits
// lose 2^-47, far below the 1e-12 the correlators need.
//
// Kernels: k_slice_psi / k_slice_modes write the digits as bf16 in the tensor
// core's canonical K-major layout (8-row x 16-byte core matrices), one 8 KB /
// 4 KB tile per digit, per 32 reals of kappa2 and per 128 rows / 64 columns;
// k_proj_mma streams them with cp.async.bulk into a two-stage shared-memory
// ring and issues tcgen05.mma (M 128, N 64, K 16) into eight TMEM class
// accumulators (8 x 64 = 512 columns); eight epilogue warps read the classes
// with tcgen05.ld after every chunk.  Every wait is bounded: a stalled pipeline
// sets an error flag and the kernel drains its copies and MMAs before freeing
// TMEM and returning.
#include "common.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace {

constexpr int S = 8;                   // digits per value
constexpr int NCLS = S;                // classes c = i + j - 2 = 0 .. 7
constexpr int CK = 128;                // complex kappa per chunk
constexpr int KB = 32;                 // reals of kappa2 per pipeline stage (two MMA K-steps)
constexpr int NBK = 2 * CK / KB;       // stages per chunk
constexpr int TM = 128;                // tile rows (j, alpha)
constexpr int TN = 64;                 // tile columns: 32 modes x (re, im)
constexpr int A_TILE = TM * KB * 2;    // bytes of one digit tile of A
constexpr int B_TILE = TN * KB * 2;
constexpr int SBO = (KB / 8) * 128;    // 8-row group stride inside a tile
constexpr int LBO = 128;               // K-adjacent core matrices
constexpr int STAGE_A = S * A_TILE, STAGE_B = S * B_TILE;
constexpr int EXP_BYTES = (TM + TN) * 4;
constexpr int SMEM_BYTES = 2 * (STAGE_A + STAGE_B) + 2 * EXP_BYTES;
constexpr long WAIT_LIMIT = 1l << 22;

// Digits by integer arithmetic on the FP64 bits (FP64 arithmetic is scarce on this
// GPU).  exp_above: e with |x| < 2^e (zero and denormals: kExpZero, below every
// normal exponent).  fixed47: X = round(x 2^(47 - e)), |X| <= 2^47.  Balanced base-64
// digits: X = sum_{i=0..7} d_i 64^(7 - i), |d_i| <= 32, so
// x = 2^(e - 5) sum_i d_i 64^-i up to the rounding of X.
constexpr int kExpZero = -1100;
__device__ __forceinline__ int exp_above(double x) {
  const int E = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return E == 0 ? kExpZero : E - 1023 + 1;
}
__device__ __forceinline__ long long fixed47(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0;
  const long long M = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
  const int k = e + 5 - (E - 1023);            // >= 6 since E - 1023 < e
  const long long X = k >= 62 ? 0 : ((M + (1ll << (k - 1))) >> k);
  return b < 0 ? -X : X;
}
__device__ __forceinline__ void digits(double x, int e, float (&d)[S]) {
  long long X = fixed47(x, e);
#pragma unroll
  for (int i = S - 1; i >= 1; i--) {
    const long long r = ((X + 32) & 63) - 32;   // in [-32, 31]
    d[i] = (float)r;
    X = (X - r) >> 6;                            // exact: X - r is a multiple of 64
  }
  d[0] = (float)X;                               // |d_0| <= 32
}

__device__ __forceinline__ int warp_max_int(int v) { return __reduce_max_sync(0xffffffffu, v); }

// 2^e as a float (exact for -126 <= e <= 127, 0 below)
__device__ __forceinline__ float pow2f(int e) {
  return e < -126 ? 0.f : (e > 127 ? __int_as_float(0x7f800000) : __int_as_float((e + 127) << 23));
}

// one 16-byte core-matrix row of a digit tile: 8 bf16
__device__ __forceinline__ uint4 pack8(const float (&v)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
    w[q] = *(uint32_t*)&h;
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// A digits: one warp per (t, j, chunk q) for the four rows r = 4 j + alpha; lane l
// holds kappa = q CK + 4 l .. + 3 (reals 8 l .. 8 l + 7 of the chunk).  Rows of
// padding (j >= nrhs) and kappa >= K are zero.
__global__ void __launch_bounds__(128) k_slice_psi(const double2* __restrict__ psi, size_t stride_sites, int site_t0,
                                                   int Vs, int Tg, int t0, int nrhs, int K, int q0, int Qg, int RT,
                                                   uint8_t* As, int* eA, int* eAmax) {
  const long wg = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long total = (long)Tg * RT * 32 * Qg;
  if (wg >= total) return;
  const int ql = (int)(wg % Qg);
  const long rest = wg / Qg;
  const int j = (int)(rest % (RT * 32));
  const int tl = (int)(rest / (RT * 32));
  const int q = q0 + ql;
  const int b = lane / 4, kc = lane % 4;
#pragma unroll 1
  for (int alpha = 0; alpha < 4; alpha++) {
    const int row = 4 * j + alpha, rt = row / TM, rr = row % TM;
    double x[8];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int kappa = q * CK + 4 * lane + u;
      double2 v = make_double2(0, 0);
      if (j < nrhs && kappa < K) {
        const int m = kappa / 3, c = kappa % 3;
        v = psi[((size_t)j * stride_sites + (size_t)(site_t0 + t0 + tl) * Vs + m) * 12 + alpha * 3 + c];
      }
      x[2 * u] = v.x;
      x[2 * u + 1] = v.y;
    }
    int ex = kExpZero;
#pragma unroll
    for (int u = 0; u < 8; u++) ex = max(ex, exp_above(x[u]));
    const int e = warp_max_int(ex);
    if (lane == 0) {
      eA[((size_t)(tl * RT + rt) * Qg + ql) * TM + rr] = e;
      atomicMax(eAmax + (size_t)tl * RT * TM + row, e);
    }
    float d[8][S];
#pragma unroll
    for (int u = 0; u < 8; u++) digits(x[u], e, d[u]);
    const size_t tile0 = (((size_t)(tl * RT + rt) * Qg + ql) * NBK + b) * S;
    const size_t off = (size_t)(rr / 8) * SBO + kc * LBO + (rr % 8) * 16;
#pragma unroll
    for (int s = 0; s < S; s++) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; u++) v[u] = d[u][s];
      *(uint4*)(As + (tile0 + s) * A_TILE + off) = pack8(v);
    }
  }
}

// B digits: one warp per (t, mode block mb, chunk q, mode kk of the block): row kk
// (re coefficient: re v, im v) and row 32 + kk (im coefficient: -im v, re v).
// VT is [t][kappa][k] (mode fastest).
__global__ void __launch_bounds__(128) k_slice_modes(const double2* __restrict__ VT, int N, int K, int Tg, int t0,
                                                     int q0, int Qg, int MB, uint8_t* Bs, int* eB, int* eBmax,
                                                     int conj_in = 0) {
  const long wg = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long total = (long)Tg * MB * Qg * 32;
  if (wg >= total) return;
  const int kk = (int)(wg % 32);
  long rest = wg / 32;
  const int ql = (int)(rest % Qg);
  rest /= Qg;
  const int mb = (int)(rest % MB);
  const int tl = (int)(rest / MB);
  const int q = q0 + ql, k = mb * 32 + kk;
  const int b = lane / 4, kc = lane % 4;
  double x[8];
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const int kappa = q * CK + 4 * lane + u;
    double2 v = make_double2(0, 0);
    if (k < N && kappa < K) v = VT[((size_t)(t0 + tl) * K + kappa) * N + k];
    x[2 * u] = v.x;
    x[2 * u + 1] = conj_in ? -v.y : v.y;
  }
  int ex = kExpZero;
#pragma unroll
  for (int u = 0; u < 8; u++) ex = max(ex, exp_above(x[u]));
  const int e = warp_max_int(ex);
  if (lane == 0) {
    eB[((size_t)(tl * MB + mb) * Qg + ql) * TN + kk] = e;
    eB[((size_t)(tl * MB + mb) * Qg + ql) * TN + 32 + kk] = e;
    atomicMax(eBmax + (size_t)(tl * MB + mb) * TN + kk, e);
    atomicMax(eBmax + (size_t)(tl * MB + mb) * TN + 32 + kk, e);
  }
  float d[8][S];
#pragma unroll
  for (int u = 0; u < 8; u++) digits(x[u], e, d[u]);
  const size_t tile0 = (((size_t)(tl * MB + mb) * Qg + ql) * NBK + b) * S;
#pragma unroll
  for (int half = 0; half < 2; half++) {
    const int n = half * 32 + kk;
    const size_t off = (size_t)(n / 8) * SBO + kc * LBO + (n % 8) * 16;
#pragma unroll
    for (int s = 0; s < S; s++) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (half == 0) { v[2 * u] = d[2 * u][s]; v[2 * u + 1] = d[2 * u + 1][s]; }
        else { v[2 * u] = -d[2 * u + 1][s]; v[2 * u + 1] = d[2 * u][s]; }
      }
      *(uint4*)(Bs + (tile0 + s) * B_TILE + off) = pack8(v);
    }
  }
}

// A digits of a generic complex source: row r of timeslice t, element kappa at
// src[t st + r sr + kappa sk] (one warp per (t, row, chunk q); the lanes as in
// k_slice_psi).  Rows r >= R and kappa >= K are zero.
__global__ void __launch_bounds__(128) k_slice_agen(const double2* __restrict__ src, size_t st, size_t sr, size_t sk,
                                                    int Tg, int R, int K, int q0, int Qg, int RT, uint8_t* As, int* eA,
                                                    int* eAmax) {
  const long wg = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long total = (long)Tg * RT * TM * Qg;
  if (wg >= total) return;
  const int ql = (int)(wg % Qg);
  const long rest = wg / Qg;
  const int row = (int)(rest % (RT * TM));
  const int tl = (int)(rest / (RT * TM));
  const int q = q0 + ql;
  const int b = lane / 4, kc = lane % 4;
  const int rt = row / TM, rr = row % TM;
  double x[8];
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const int kappa = q * CK + 4 * lane + u;
    double2 v = make_double2(0, 0);
    if (row < R && kappa < K) v = src[(size_t)tl * st + (size_t)row * sr + (size_t)kappa * sk];
    x[2 * u] = v.x;
    x[2 * u + 1] = v.y;
  }
  int ex = kExpZero;
#pragma unroll
  for (int u = 0; u < 8; u++) ex = max(ex, exp_above(x[u]));
  const int e = warp_max_int(ex);
  if (lane == 0) {
    eA[((size_t)(tl * RT + rt) * Qg + ql) * TM + rr] = e;
    atomicMax(eAmax + (size_t)tl * RT * TM + row, e);
  }
  float d[8][S];
#pragma unroll
  for (int u = 0; u < 8; u++) digits(x[u], e, d[u]);
  const size_t tile0 = (((size_t)(tl * RT + rt) * Qg + ql) * NBK + b) * S;
  const size_t off = (size_t)(rr / 8) * SBO + kc * LBO + (rr % 8) * 16;
#pragma unroll
  for (int s = 0; s < S; s++) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) v[u] = d[u][s];
    *(uint4*)(As + (tile0 + s) * A_TILE + off) = pack8(v);
  }
}

__global__ void k_fill_int(int* p, size_t n, int v) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) p[e] = v;
}

// Tile (row block rt, mode block mb, timeslice tl) over the chunks q0 .. q0 + Qg - 1.
// Warp 0: bulk copies; warp 1: TMEM and MMAs; warps 2..9: epilogue (warp w reads
// TMEM lanes 32 (w % 4) .. + 31 and columns 32 ((w - 2) / 4) .. + 31).
__global__ void __launch_bounds__(320, 1) k_proj_mma(const uint8_t* __restrict__ As, const uint8_t* __restrict__ Bs,
                                                     const int* __restrict__ eA, const int* __restrict__ eB,
                                                     const int* __restrict__ eAmax, const int* __restrict__ eBmax,
                                                     int Qg, int RT, int MB, int R, int N, int Tsel, int t0,
                                                     int accumulate, double* coeff, int* err, int omode = 0) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[2], empty[2], accf, acce, drain;
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  __shared__ int ref_b[TN];     // reference exponents of the tile's columns
  uint8_t* sA[2] = {smem, smem + STAGE_A};
  uint8_t* sB[2] = {smem + 2 * STAGE_A, smem + 2 * STAGE_A + STAGE_B};
  int* sE[2] = {(int*)(smem + 2 * (STAGE_A + STAGE_B)), (int*)(smem + 2 * (STAGE_A + STAGE_B) + EXP_BYTES)};
  const int rt = blockIdx.x, mb = blockIdx.y, tl = blockIdx.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nstages = Qg * NBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; s++) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&accf, 1);
    tc::mbar_init(&acce, 8);
    tc::mbar_init(&drain, 1);
    abort_flag = 0;
    tc::mbar_fence_init();
  }
  if (threadIdx.x < TN) ref_b[threadIdx.x] = eBmax[(size_t)(tl * MB + mb) * TN + threadIdx.x];
  if (warp == 1) tc::tmem_alloc(&tbase, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;

  if (warp == 0) {
    // ---- producer ----
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nstages; it++) {
        if (abort_flag) break;
        const int st = it & 1, use = it >> 1;
        if (it >= 2 && !tc::mbar_wait(&empty[st], (use - 1) & 1, WAIT_LIMIT)) {
          abort_flag = 1;
          atomicExch(err, 1);
          break;
        }
        const int ql = it / NBK, b = it % NBK;
        const size_t ta = (((size_t)(tl * RT + rt) * Qg + ql) * NBK + b) * S;
        const size_t tb = (((size_t)(tl * MB + mb) * Qg + ql) * NBK + b) * S;
        const uint32_t bytes = STAGE_A + STAGE_B + (b == 0 ? EXP_BYTES : 0);
        tc::mbar_arrive_expect_tx(&full[st], bytes);
        tc::bulk_g2s(sA[st], As + ta * A_TILE, STAGE_A, &full[st]);
        tc::bulk_g2s(sB[st], Bs + tb * B_TILE, STAGE_B, &full[st]);
        if (b == 0) {
          tc::bulk_g2s(sE[ql & 1], eA + ((size_t)(tl * RT + rt) * Qg + ql) * TM, TM * 4, &full[st]);
          tc::bulk_g2s(sE[ql & 1] + TM, eB + ((size_t)(tl * MB + mb) * Qg + ql) * TN, TN * 4, &full[st]);
        }
        issued = it + 1;
      }
      // copies still in flight land before the shared memory is given up
      for (int it = issued - 2 < 0 ? 0 : issued - 2; it < issued; it++)
        tc::mbar_wait(&full[it & 1], (it >> 1) & 1, WAIT_LIMIT);
    }
  } else if (warp == 1) {
    // ---- MMA issue ----
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(TM, TN);
      for (int it = 0; it < nstages; it++) {
        const int st = it & 1, use = it >> 1;
        const int ql = it / NBK, b = it % NBK;
        if (abort_flag) break;
        if (b == 0 && ql > 0 && !tc::mbar_wait(&acce, (ql - 1) & 1, WAIT_LIMIT)) {
          abort_flag = 1;
          atomicExch(err, 1);
          break;
        }
        if (!tc::mbar_wait(&full[st], use & 1, WAIT_LIMIT)) {
          abort_flag = 1;
          atomicExch(err, 1);
          break;
        }
        tc::fence_after();
        const uint32_t a0 = tc::smem_addr(sA[st]), b0 = tc::smem_addr(sB[st]);
#pragma unroll
        for (int ks = 0; ks < KB / 16; ks++)
#pragma unroll
          for (int c = 0; c < NCLS; c++)
#pragma unroll
            for (int i = 1; i <= c + 1; i++) {
              const int jd = c + 2 - i;
              const uint64_t ad = tc::smem_desc(a0 + (i - 1) * A_TILE + ks * 256, LBO, SBO);
              const uint64_t bd = tc::smem_desc(b0 + (jd - 1) * B_TILE + ks * 256, LBO, SBO);
              const uint32_t acc = (b == 0 && ks == 0 && i == 1) ? 0u : 1u;
              tc::mma_bf16(tmem + c * TN, ad, bd, idesc, acc);
            }
        tc::mma_commit(&empty[st]);                   // the stage may be refilled
        if (b == NBK - 1) tc::mma_commit(&accf);      // chunk complete: classes ready
      }
      // every MMA issued has completed before TMEM is read for the last time / freed
      tc::mma_commit(&drain);
      tc::mbar_wait(&drain, 0, WAIT_LIMIT);
    }
  } else {
    // ---- epilogue: double-float accumulation of the scaled class sums ----
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    // reference exponents of the row and the columns: the float accumulator holds the
    // sum relative to 2^(ra + rb), restored in FP64 at the end
    const int ra = eAmax[(size_t)tl * RT * TM + rt * TM + row];
    const int* rb = ref_b + half * 32;
    float hi[32], lo[32];
#pragma unroll
    for (int n = 0; n < 32; n++) hi[n] = lo[n] = 0.f;
    for (int ql = 0; ql < Qg; ql++) {
      if (!tc::mbar_wait(&accf, ql & 1, WAIT_LIMIT)) {
        abort_flag = 1;
        atomicExch(err, 1);
        break;
      }
      tc::fence_after();
      const int ea = sE[ql & 1][row];
      const int* eb = sE[ql & 1] + TM + half * 32;
#pragma unroll 1
      for (int c = 0; c < NCLS; c++) {
        uint32_t r[32];
        tc::tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + c * TN + half * 32, r);
        tc::tmem_wait_ld();
#pragma unroll
        for (int n = 0; n < 32; n++) {
          const float v = __uint_as_float(r[n]) * pow2f((ea - ra) + (eb[n] - rb[n]) - 10 - 6 * c);
          const float s = hi[n] + v;
          const float bp = s - hi[n];
          lo[n] += (hi[n] - (s - bp)) + (v - bp);
          hi[n] = s;
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce);
    }
    const int grow = rt * TM + row;
    if (!abort_flag && grow < R) {
      const int j = grow / 4, alpha = grow % 4;
#pragma unroll
      for (int n = 0; n < 32; n++) {
        const int k = mb * 32 + n;
        if (k >= N) break;
        // omode 0: coeff[j][t][alpha][k]; 1: out[t][k][row]; 2: out[t][row][k]
        const size_t idx = omode == 0 ? (((size_t)j * Tsel + t0 + tl) * 4 + alpha) * N + k
                           : omode == 1 ? ((size_t)(t0 + tl) * N + k) * R + grow
                                        : ((size_t)(t0 + tl) * R + grow) * N + k;
        double* o = coeff + 2 * idx + half;
        const double v = ldexp((double)hi[n] + (double)lo[n], ra + rb[n]);
        *o = accumulate ? *o + v : v;
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

}  // namespace

// coeff[j][Tsel][4][N] = V^dag psi on the tensor cores (see the top of the file);
// VT [Tsel][3 Vs][N] (mode fastest), psi canonical with stride_sites per rhs,
// timeslices site_t0 .. site_t0 + Tsel - 1.  The digit buffers are bounded: the
// chunks of kappa run in groups whose results accumulate in FP64 in coeff.
dlma_status project_tc(dlma_ctx* ctx, const double2* VT, int N, int Tsel, const double* psi, size_t stride_sites,
                       int site_t0, int nrhs, double2* coeff) {
  const int Vs = ctx->g.Vs, K = 3 * Vs;
  const int Q = (K + CK - 1) / CK;
  const int R = 4 * nrhs;
  const int RT = (R + TM - 1) / TM, MB = (N + 31) / 32;
  // digit bytes per chunk of every timeslice: A (RT tiles of rows) and B (MB tiles of modes)
  const size_t per_chunk = (size_t)Tsel * NBK * S * ((size_t)RT * A_TILE + (size_t)MB * B_TILE);
  size_t budget = (size_t)4 << 30;
  if (ctx->memcap) budget = std::min(budget, (size_t)ctx->memcap / 4);
  const int Qg = (int)std::max<size_t>(1, std::min<size_t>((size_t)Q, budget / per_chunk));
  uint8_t *As, *Bs;
  int *eA, *eB;
  TRY(workT(ctx, WS_TC_A, (size_t)Tsel * RT * Qg * NBK * S * A_TILE, &As));
  TRY(workT(ctx, WS_TC_B, (size_t)Tsel * MB * Qg * NBK * S * B_TILE, &Bs));
  TRY(workT(ctx, WS_TC_E, (size_t)Tsel * (Qg + 1) * (RT * TM + MB * TN), &eA));
  eB = eA + (size_t)Tsel * Qg * RT * TM;
  int* eAmax = eB + (size_t)Tsel * Qg * MB * TN;
  int* eBmax = eAmax + (size_t)Tsel * RT * TM;
  const size_t nref = (size_t)Tsel * (RT * TM + MB * TN);
  int* err = ctx->flag + 8;
  CU(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  static bool attr_set[64] = {false};
  if (ctx->device >= 0 && ctx->device < 64 && !attr_set[ctx->device]) {
    CU(cudaFuncSetAttribute(k_proj_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr_set[ctx->device] = true;
  }
  for (int q0 = 0; q0 < Q; q0 += Qg) {
    const int qn = std::min(Qg, Q - q0);
    const long wa = (long)Tsel * RT * 32 * qn, wb = (long)Tsel * MB * qn * 32;
    k_fill_int<<<(unsigned)((nref + 255) / 256), 256, 0, ctx->stream>>>(eAmax, nref, kExpZero);
    CHECK_LAUNCH();
    k_slice_psi<<<(unsigned)((wa + 3) / 4), 128, 0, ctx->stream>>>((const double2*)psi, stride_sites, site_t0, Vs, Tsel,
                                                                   0, nrhs, K, q0, qn, RT, As, eA, eAmax);
    CHECK_LAUNCH();
    k_slice_modes<<<(unsigned)((wb + 3) / 4), 128, 0, ctx->stream>>>(VT, N, K, Tsel, 0, q0, qn, MB, Bs, eB, eBmax);
    CHECK_LAUNCH();
    k_proj_mma<<<dim3(RT, MB, Tsel), 320, SMEM_BYTES, ctx->stream>>>(As, Bs, eA, eB, eAmax, eBmax, qn, RT, MB, R, N,
                                                                    Tsel, 0, q0 > 0 ? 1 : 0, (double*)coeff, err);
    CHECK_LAUNCH();
  }
  int h = 0;
  CU(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (h) return set_err(ctx, DLMA_ERR_CUDA, "tensor-core projection: a pipeline wait timed out");
  return DLMA_OK;
}

// Block products of the eigensolver's FP64 phase on the tensor cores, with the same
// FP64-accurate digit scheme.  For every timeslice t:
//   out[t] (omode 1: [N][R], omode 2: [R][N]) holds sum_kappa conj(B_k(kappa)) A_r(kappa)
// with A_r(kappa) = a_src[t a_st + r a_sr + kappa a_sk] (R rows, K long) and
// B_k(kappa) = b_src[(t K + kappa) N + k] (conjugated first when b_conj).
dlma_status tc_block_product(dlma_ctx* ctx, int omode, const double2* a_src, size_t a_st, size_t a_sr, size_t a_sk,
                             int R, const double2* b_src, int b_conj, int N, int K, int T, double2* out) {
  if (omode != 1 && omode != 2) return set_err(ctx, DLMA_ERR_INVALID_ARG, "tc_block_product mode");
  const int Q = (K + CK - 1) / CK;
  const int RT = (R + TM - 1) / TM, MB = (N + 31) / 32;
  const size_t per_chunk = (size_t)T * NBK * S * ((size_t)RT * A_TILE + (size_t)MB * B_TILE);
  size_t budget = (size_t)4 << 30;
  if (ctx->memcap) budget = std::min(budget, (size_t)ctx->memcap / 4);
  const int Qg = (int)std::max<size_t>(1, std::min<size_t>((size_t)Q, budget / per_chunk));
  uint8_t *As, *Bs;
  int *eA, *eB;
  TRY(workT(ctx, WS_TC_A, (size_t)T * RT * Qg * NBK * S * A_TILE, &As));
  TRY(workT(ctx, WS_TC_B, (size_t)T * MB * Qg * NBK * S * B_TILE, &Bs));
  TRY(workT(ctx, WS_TC_E, (size_t)T * (Qg + 1) * (RT * TM + MB * TN), &eA));
  eB = eA + (size_t)T * Qg * RT * TM;
  int* eAmax = eB + (size_t)T * Qg * MB * TN;
  int* eBmax = eAmax + (size_t)T * RT * TM;
  const size_t nref = (size_t)T * (RT * TM + MB * TN);
  int* err = ctx->flag + 8;
  CU(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  static bool attr_set[64] = {false};
  if (ctx->device >= 0 && ctx->device < 64 && !attr_set[ctx->device]) {
    CU(cudaFuncSetAttribute(k_proj_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr_set[ctx->device] = true;
  }
  for (int q0 = 0; q0 < Q; q0 += Qg) {
    const int qn = std::min(Qg, Q - q0);
    const long wa = (long)T * RT * TM * qn, wb = (long)T * MB * qn * 32;
    k_fill_int<<<(unsigned)((nref + 255) / 256), 256, 0, ctx->stream>>>(eAmax, nref, kExpZero);
    CHECK_LAUNCH();
    k_slice_agen<<<(unsigned)((wa + 3) / 4), 128, 0, ctx->stream>>>(a_src, a_st, a_sr, a_sk, T, R, K, q0, qn, RT, As,
                                                                    eA, eAmax);
    CHECK_LAUNCH();
    k_slice_modes<<<(unsigned)((wb + 3) / 4), 128, 0, ctx->stream>>>(b_src, N, K, T, 0, q0, qn, MB, Bs, eB, eBmax,
                                                                     b_conj);
    CHECK_LAUNCH();
    k_proj_mma<<<dim3(RT, MB, T), 320, SMEM_BYTES, ctx->stream>>>(As, Bs, eA, eB, eAmax, eBmax, qn, RT, MB, R, N, T,
                                                                 0, q0 > 0 ? 1 : 0, (double*)out, err, omode);
    CHECK_LAUNCH();
  }
  int h = 0;
  CU(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (h) return set_err(ctx, DLMA_ERR_CUDA, "tensor-core block product: a pipeline wait timed out");
  return DLMA_OK;
}
