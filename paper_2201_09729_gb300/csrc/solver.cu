// Multi-right-hand-side Dirac solves x = D^-1 b (the propagator solves of
// Eq. 4 and of the perambulator after Eq. 3).
//
// Even-odd Schur system Dhat x_e = bhat, bhat = b_e - D_eo T_oo^-1 b_o, solved
// by CG on the normal equations Dhat^dag Dhat x_e = Dhat^dag bhat (CGNE).
// Precision scheme: an FP64 outer defect-correction loop recomputes the true
// residual r = bhat - Dhat x in double precision and restarts an inner CGNE
// run in FP32 (or FP16 with per-site scales, FP32 vector algebra) on the
// normalised residual; the correction is accumulated into x in FP64.  Every
// right-hand side carries its own CG scalars on the device and is retired
// (masked out of every kernel) once converged.  A chunk of inner iterations is
// captured once into a CUDA graph and replayed; the host polls one pinned
// counter per chunk, with an iteration cap and a wall-clock limit, so a solve
// never waits without bound.
#include "fieldio.cuh"
#include <chrono>
#include <math.h>

namespace {

constexpr int BX = 128;   // sites per block for vector kernels

struct CgScal {
  double* rr;      // current |r|^2 of the normal equations
  double* alpha;
  double* beta;
  double* stop2;   // stopping threshold on |r|^2
  double* rnorm;   // FP64 outer residual norm per rhs
  double* bnorm;   // |b| per rhs (full lattice)
  int* active;     // inner-loop mask
  int* outer_active;
  int* iters;      // inner iterations this outer cycle
  int* count;      // [0] number of active rhs, [1] nonfinite flag
};

// reduce per-(rhs, block) partials: out[j] = sum_b part[j * nb + b]; one warp per rhs
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double reduce_row(const double* part, int nb, int j) {
  double s = 0;
  for (int b = threadIdx.x; b < nb; b += 32) s += part[(size_t)j * nb + b];
  return __shfl_sync(0xffffffffu, warp_sum(s), 0);
}

__global__ void k_cg_alpha(const double* part, int nb, int nrhs, CgScal sc) {
  int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs) return;
  if (!sc.active[j]) return;
  // lanes of one warp: recompute with lane index
  double s = 0;
  int lane = threadIdx.x & 31;
  for (int b = lane; b < nb; b += 32) s += part[(size_t)j * nb + b];
  s = warp_sum(s);
  if (lane == 0) {
    double qq = s;
    double a = (qq > 0 && isfinite(qq)) ? sc.rr[j] / qq : 0.0;
    sc.alpha[j] = a;
    if (!(qq > 0) || !isfinite(qq)) {
      sc.active[j] = 0;
      if (!isfinite(qq)) sc.count[1] = 1;
    }
  }
}

__global__ void k_cg_beta(const double* part, int nb, int nrhs, CgScal sc) {
  int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs) return;
  if (!sc.active[j]) return;
  int lane = threadIdx.x & 31;
  double s = 0;
  for (int b = lane; b < nb; b += 32) s += part[(size_t)j * nb + b];
  s = warp_sum(s);
  if (lane == 0) {
    double rrn = s;
    sc.beta[j] = rrn / sc.rr[j];
    sc.rr[j] = rrn;
    sc.iters[j] += 1;
    if (!isfinite(rrn)) { sc.active[j] = 0; sc.count[1] = 1; }
    else if (rrn <= sc.stop2[j]) sc.active[j] = 0;
  }
}

__global__ void k_count(const int* act, int n, int* count) {
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  int c = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) c += act[j] != 0;
  atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) count[0] = s;
}

// block-level partial of a per-thread double, one entry per (rhs, block)
__device__ __forceinline__ void block_partial(double v, double* part, int j, int nrhs) {
  __shared__ double red[BX / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0 && j < nrhs) {
    double t = 0;
    for (int w = 0; w < BX / 32; w++) t += red[w];
    part[(size_t)j * gridDim.x + blockIdx.x] = t;
  }
}

template <class R> __device__ __forceinline__ double snorm(const Spinor<R>& s) {
  double n = 0;
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) n += (double)norm2(s.c[a][c]);
  return n;
}

// x += alpha p; r -= alpha z; partial |r|^2           (PB: vector precision, PS: stencil precision)
template <int PB, int PS>
__global__ void __launch_bounds__(BX) k_update_xr(int Vh, int nrhs, void* x, void* r, const void* p, const void* z,
                                                   const float* zsc, CgScal sc, double* part) {
  typedef typename PT<PB>::R R;
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y;
  double n = 0;
  if (i < Vh && sc.active[j]) {
    size_t sb = field_units_per_rhs(PB, Vh) * 16 * j, ss = field_units_per_rhs(PS, Vh) * 16 * j;
    R a = (R)sc.alpha[j];
    Spinor<R> xv = load_spinor<PB>((char*)x + sb, nullptr, Vh, i);
    Spinor<R> rv = load_spinor<PB>((char*)r + sb, nullptr, Vh, i);
    Spinor<R> pv = load_spinor<PB>((const char*)p + sb, nullptr, Vh, i);
    Spinor<typename PT<PS>::R> zv = load_spinor<PS>((const char*)z + ss, zsc ? zsc + (size_t)j * Vh : nullptr, Vh, i);
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        xv.c[s][c] = xv.c[s][c] + a * pv.c[s][c];
        rv.c[s][c] = rv.c[s][c] - a * cx<R>((R)zv.c[s][c].re, (R)zv.c[s][c].im);
      }
    store_spinor<PB>((char*)x + sb, nullptr, Vh, i, xv);
    store_spinor<PB>((char*)r + sb, nullptr, Vh, i, rv);
    n = snorm(rv);
  }
  block_partial(n, part, sc.active[j] ? j : nrhs, nrhs);
}

// p = r + beta p  (and the stencil-precision copy when PS != PB)
template <int PB, int PS>
__global__ void __launch_bounds__(BX) k_update_p(int Vh, int nrhs, const void* r, void* p, void* ps, float* pssc,
                                                  CgScal sc) {
  typedef typename PT<PB>::R R;
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y;
  if (i >= Vh || !sc.active[j]) return;
  size_t sb = field_units_per_rhs(PB, Vh) * 16 * j;
  R b = (R)sc.beta[j];
  Spinor<R> rv = load_spinor<PB>((const char*)r + sb, nullptr, Vh, i);
  Spinor<R> pv = load_spinor<PB>((char*)p + sb, nullptr, Vh, i);
#pragma unroll
  for (int s = 0; s < 4; s++)
#pragma unroll
    for (int c = 0; c < 3; c++) pv.c[s][c] = rv.c[s][c] + b * pv.c[s][c];
  store_spinor<PB>((char*)p + sb, nullptr, Vh, i, pv);
  if (PS != PB) {
    size_t ss = field_units_per_rhs(PS, Vh) * 16 * j;
    Spinor<typename PT<PS>::R> q;
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) q.c[s][c] = cx<typename PT<PS>::R>(pv.c[s][c].re, pv.c[s][c].im);
    store_spinor<PS>((char*)ps + ss, pssc + (size_t)j * Vh, Vh, i, q);
  }
}

// out = f_j * in   (precision conversion with a per-rhs factor; f = nullptr -> 1); optional |out|^2 partial
template <int PI, int PO>
__global__ void __launch_bounds__(BX) k_convert(int Vh, int nrhs, const void* in, const float* insc, void* out,
                                                 float* outsc, const double* f, int finv, const int* mask,
                                                 double* part) {
  typedef typename PT<PO>::R R;
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y;
  bool on = mask ? mask[j] != 0 : true;
  double n = 0;
  if (i < Vh && on) {
    size_t si = field_units_per_rhs(PI, Vh) * 16 * j, so = field_units_per_rhs(PO, Vh) * 16 * j;
    Spinor<typename PT<PI>::R> v = load_spinor<PI>((const char*)in + si, insc ? insc + (size_t)j * Vh : nullptr, Vh, i);
    double ff = 1.0;
    if (f) ff = finv ? (f[j] > 0 ? 1.0 / f[j] : 0.0) : f[j];
    Spinor<R> o;
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) o.c[s][c] = cx<R>((R)(ff * (double)v.c[s][c].re), (R)(ff * (double)v.c[s][c].im));
    store_spinor<PO>((char*)out + so, outsc ? outsc + (size_t)j * Vh : nullptr, Vh, i, o);
    n = snorm(o);
  }
  if (part) block_partial(n, part, on ? j : nrhs, nrhs);
}

// x64 += f_j * lo    (defect-correction accumulation)
template <int PL>
__global__ void __launch_bounds__(BX) k_accum(int Vh, int nrhs, double2* x, const void* lo, const double* f,
                                               const int* mask) {
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y;
  if (i >= Vh || !mask[j]) return;
  size_t sl = field_units_per_rhs(PL, Vh) * 16 * j;
  Spinor<typename PT<PL>::R> v = load_spinor<PL>((const char*)lo + sl, nullptr, Vh, i);
  double ff = f[j];
  double2* xb = x + (size_t)12 * Vh * j;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    double2 e = xb[(size_t)k * Vh + i];
    e.x += ff * (double)v.c[k / 3][k % 3].re;
    e.y += ff * (double)v.c[k / 3][k % 3].im;
    xb[(size_t)k * Vh + i] = e;
  }
}

// r = a - b (FP64) with |r|^2 partial
__global__ void __launch_bounds__(BX) k_sub64(int Vh, int nrhs, const double2* a, const double2* b, double2* r,
                                               const int* mask, double* part) {
  int i = blockIdx.x * BX + threadIdx.x;
  int j = blockIdx.y;
  bool on = mask ? mask[j] != 0 : true;
  double n = 0;
  if (i < Vh && on) {
    size_t o = (size_t)12 * Vh * j;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 x = a[o + (size_t)k * Vh + i], y = b[o + (size_t)k * Vh + i];
      double2 d = make_double2(x.x - y.x, x.y - y.y);
      r[o + (size_t)k * Vh + i] = d;
      n += d.x * d.x + d.y * d.y;
    }
  }
  block_partial(n, part, on ? j : nrhs, nrhs);
}

// per-rhs totals of a partial buffer: out[j] = sum_b part[j][b]
__global__ void k_rowsum(const double* part, int nb, int nrhs, double* out, int do_sqrt) {
  int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs) return;
  int lane = threadIdx.x & 31;
  double s = 0;
  for (int b = lane; b < nb; b += 32) s += part[(size_t)j * nb + b];
  s = warp_sum(s);
  if (lane == 0) out[j] = do_sqrt ? sqrt(s) : s;
}

// inner-cycle initialisation from the normal-equation residual r0 = |r|^2 per rhs
__global__ void k_inner_init(int nrhs, CgScal sc, const double* rr0, double delta2) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs) return;
  if (!sc.outer_active[j]) { sc.active[j] = 0; sc.iters[j] = 0; return; }
  int on = rr0[j] > 0 && isfinite(rr0[j]);
  sc.active[j] = on;
  sc.rr[j] = rr0[j];
  sc.stop2[j] = delta2 * rr0[j];
  sc.iters[j] = 0;
  if (!isfinite(rr0[j])) sc.count[1] = 1;
}

// outer convergence: rhs j done when |r_j| <= tol * |b_j|
__global__ void k_outer_check(int nrhs, CgScal sc, double tol) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs || !sc.outer_active[j]) return;
  if (!isfinite(sc.rnorm[j])) { sc.count[1] = 1; sc.outer_active[j] = 0; return; }
  if (sc.rnorm[j] <= tol * sc.bnorm[j]) sc.outer_active[j] = 0;
}

}  // namespace

// ---------------------------------------------------------------------------
struct SolveBufs {
  Field b_e, b_o, bh, x64, r64, t64, t64o;     // FP64
  Field xl, rl, pl, ps, q, z, tmp, rhs;        // low precision (pl: vector precision, ps/q/z/tmp/rhs: stencil)
  double *part, *part2;
  CgScal sc;
};

static dlma_status rowsum(dlma_ctx* ctx, const double* part, int nb, int nrhs, double* out, int do_sqrt) {
  k_rowsum<<<(nrhs + 3) / 4, 128, 0, ctx->stream>>>(part, nb, nrhs, out, do_sqrt);
  CHECK_LAUNCH();
  return DLMA_OK;
}

template <int PB, int PS>
static dlma_status inner_iteration(dlma_ctx* ctx, SolveBufs& B, int nrhs) {
  const int Vh = ctx->g.Vh;
  dim3 gv((Vh + BX - 1) / BX, nrhs);
  int nbh = hop_grid_x(ctx, PS);
  // q = Dhat p ; |q|^2 partials
  TRY(schur_apply(ctx, B.ps, B.tmp, B.q, 0, B.sc.active, B.part));
  k_cg_alpha<<<(nrhs + 3) / 4, 128, 0, ctx->stream>>>(B.part, nbh, nrhs, B.sc);
  CHECK_LAUNCH();
  // z = Dhat^dag q
  TRY(schur_apply(ctx, B.q, B.tmp, B.z, 1, B.sc.active, nullptr));
  k_update_xr<PB, PS><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.xl.data, B.rl.data, B.pl.data, B.z.data, B.z.scale,
                                                  B.sc, B.part2);
  CHECK_LAUNCH();
  k_cg_beta<<<(nrhs + 3) / 4, 128, 0, ctx->stream>>>(B.part2, gv.x, nrhs, B.sc);
  CHECK_LAUNCH();
  k_update_p<PB, PS><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.rl.data, B.pl.data, B.ps.data, B.ps.scale, B.sc);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// FP64 residual r64 = bhat - Dhat x64 and its norms; outer check
static dlma_status outer_residual(dlma_ctx* ctx, SolveBufs& B, int nrhs, double tol) {
  const int Vh = ctx->g.Vh;
  dim3 gv((Vh + BX - 1) / BX, nrhs);
  TRY(schur_apply(ctx, B.x64, B.t64o, B.t64, 0, B.sc.outer_active, nullptr));
  k_sub64<<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (const double2*)B.bh.data, (const double2*)B.t64.data,
                                      (double2*)B.r64.data, B.sc.outer_active, B.part2);
  CHECK_LAUNCH();
  TRY(rowsum(ctx, B.part2, gv.x, nrhs, B.sc.rnorm, 1));
  k_outer_check<<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(nrhs, B.sc, tol);
  CHECK_LAUNCH();
  return DLMA_OK;
}

template <int PB, int PS>
static dlma_status solve_batch(dlma_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, double tol,
                               dlma_solve_info* info, double delta, int max_inner, int max_outer) {
  const int Vh = ctx->g.Vh;
  SolveBufs B;
  TRY(field_alloc(ctx, WS_SOLVE_B, DLMA_FP64, 2 * nrhs, &B.b_e));
  B.b_o = B.b_e;
  B.b_e.nrhs = B.b_o.nrhs = nrhs;
  B.b_o.data = (char*)B.b_e.data + field_bytes_per_rhs(DLMA_FP64, Vh) * nrhs;
  TRY(field_alloc(ctx, WS_SOLVE_BH, DLMA_FP64, nrhs, &B.bh));
  TRY(field_alloc(ctx, WS_SOLVE_X64, DLMA_FP64, nrhs, &B.x64));
  TRY(field_alloc(ctx, WS_SOLVE_R64, DLMA_FP64, nrhs, &B.r64));
  TRY(field_alloc(ctx, WS_SOLVE_TMP64, DLMA_FP64, 2 * nrhs, &B.t64));
  B.t64o = B.t64;
  B.t64.nrhs = B.t64o.nrhs = nrhs;
  B.t64o.data = (char*)B.t64.data + field_bytes_per_rhs(DLMA_FP64, Vh) * nrhs;
  TRY(field_alloc(ctx, WS_CG_X, PB, nrhs, &B.xl));
  TRY(field_alloc(ctx, WS_CG_R, PB, nrhs, &B.rl));
  TRY(field_alloc(ctx, WS_CG_P, PB, nrhs, &B.pl));
  if (PS != PB) TRY(field_alloc(ctx, WS_CG_PLO, PS, nrhs, &B.ps));
  else B.ps = B.pl;
  TRY(field_alloc(ctx, WS_CG_Q, PS, nrhs, &B.q));
  TRY(field_alloc(ctx, WS_CG_Z, PS, nrhs, &B.z));
  TRY(field_alloc(ctx, WS_CG_TMP, PS, nrhs, &B.tmp));
  TRY(field_alloc(ctx, WS_CG_RHS, PS, nrhs, &B.rhs));
  int nbmax = (Vh + 31) / 32 + 8;
  TRY(workT(ctx, WS_PART, (size_t)2 * nbmax * nrhs, &B.part));
  B.part2 = B.part + (size_t)nbmax * nrhs;
  double* sd;
  TRY(workT(ctx, WS_SCAL, (size_t)8 * nrhs + 64, &sd));
  B.sc.rr = sd;
  B.sc.alpha = sd + nrhs;
  B.sc.beta = sd + 2 * nrhs;
  B.sc.stop2 = sd + 3 * nrhs;
  B.sc.rnorm = sd + 4 * nrhs;
  B.sc.bnorm = sd + 5 * nrhs;
  double* rr0 = sd + 6 * nrhs;
  int* si;
  TRY(workT(ctx, WS_ACT, (size_t)3 * nrhs + 16, &si));
  B.sc.active = si;
  B.sc.outer_active = si + nrhs;
  B.sc.iters = si + 2 * nrhs;
  B.sc.count = si + 3 * nrhs;
  int* hcount = (int*)ctx->pinned;
  std::vector<int> iters_total(nrhs, 0);

  dim3 gv((Vh + BX - 1) / BX, nrhs);
  // sources
  TRY(pack_parity(ctx, b_dev, 1, 0, B.b_e));
  TRY(pack_parity(ctx, b_dev, 1, 1, B.b_o));
  // |b|^2 over both parities
  k_convert<DLMA_FP64, DLMA_FP64><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.b_e.data, nullptr, B.t64.data, nullptr,
                                                              nullptr, 0, nullptr, B.part);
  CHECK_LAUNCH();
  k_convert<DLMA_FP64, DLMA_FP64><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.b_o.data, nullptr, B.t64o.data, nullptr,
                                                              nullptr, 0, nullptr, B.part + (size_t)gv.x * nrhs);
  CHECK_LAUNCH();
  // sum the two parity halves: treat as 2*nb partial columns per rhs
  {
    // rearrange: rows j have gv.x entries in each half; sum both halves
    TRY(rowsum(ctx, B.part, gv.x, nrhs, rr0, 0));
    TRY(rowsum(ctx, B.part + (size_t)gv.x * nrhs, gv.x, nrhs, B.sc.rnorm, 0));
  }
  std::vector<double> hb(2 * nrhs);
  CU(cudaMemcpyAsync(hb.data(), rr0, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(hb.data() + nrhs, B.sc.rnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  std::vector<double> bn(nrhs);
  std::vector<int> act0(nrhs);
  bool nonfinite_src = false;
  for (int j = 0; j < nrhs; j++) {
    bn[j] = sqrt(hb[j] + hb[nrhs + j]);
    if (!isfinite(bn[j])) nonfinite_src = true;
    act0[j] = bn[j] > 0 && isfinite(bn[j]);
  }
  if (nonfinite_src) return set_err(ctx, DLMA_ERR_NONFINITE, "a source holds NaN or Inf");
  CU(cudaMemcpyAsync(B.sc.bnorm, bn.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemcpyAsync(B.sc.outer_active, act0.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemsetAsync(B.sc.count, 0, 2 * sizeof(int), ctx->stream));
  // bhat = b_e - D_eo T_oo^-1 b_o
  {
    HopOp a;
    a.p_out = 1; a.hop = 0; a.own = 1; a.kout = 3;
    TRY(launch_hop(ctx, a, B.b_o, &B.b_o, B.t64o));
    HopOp b;
    b.p_out = 0; b.own = 1; b.kout = 0; b.s = -1.0;
    TRY(launch_hop(ctx, b, B.t64o, &B.b_e, B.bh));
  }
  CU(cudaMemsetAsync(B.x64.data, 0, field_bytes_per_rhs(DLMA_FP64, Vh) * nrhs, ctx->stream));
  const double tol_target = 0.5 * tol;
  const double delta2 = delta * delta;
  const int chunk = 8;
  auto t_start = std::chrono::steady_clock::now();
  const double wall_limit_s = 600.0;

  // inner CG graph (captured on first use)
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  uint64_t graph_kernels = 0;
  dlma_status st = DLMA_OK;
  int outer = 0;
  for (; outer < max_outer; outer++) {
    TRY(outer_residual(ctx, B, nrhs, tol_target));
    k_count<<<1, 256, 0, ctx->stream>>>(B.sc.outer_active, nrhs, B.sc.count);
    CHECK_LAUNCH();
    CU(cudaMemcpyAsync(hcount, B.sc.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (hcount[1]) { st = set_err(ctx, DLMA_ERR_NONFINITE, "non-finite residual in the solve"); break; }
    if (hcount[0] == 0) break;
    // inner cycle: rhs = r64 / |r64| in stencil precision; r_l = Dhat^dag rhs
    k_convert<DLMA_FP64, PS><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.r64.data, nullptr, B.rhs.data, B.rhs.scale,
                                                         B.sc.rnorm, 1, B.sc.outer_active, nullptr);
    CHECK_LAUNCH();
    if (outer == 0) TRY(autotune_hop(ctx, PS, B.rhs, B.tmp, B.z));   // before the graph capture
    TRY(schur_apply(ctx, B.rhs, B.tmp, B.z, 1, B.sc.outer_active, nullptr));
    k_convert<PS, PB><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.z.data, B.z.scale, B.rl.data, nullptr, nullptr, 0,
                                                  B.sc.outer_active, B.part2);
    CHECK_LAUNCH();
    TRY(rowsum(ctx, B.part2, gv.x, nrhs, rr0, 0));
    k_convert<PB, PB><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.rl.data, nullptr, B.pl.data, nullptr, nullptr, 0,
                                                  B.sc.outer_active, nullptr);
    CHECK_LAUNCH();
    if (PS != PB) {
      k_convert<PB, PS><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.rl.data, nullptr, B.ps.data, B.ps.scale, nullptr, 0,
                                                    B.sc.outer_active, nullptr);
      CHECK_LAUNCH();
    }
    CU(cudaMemsetAsync(B.xl.data, 0, field_bytes_per_rhs(PB, Vh) * nrhs, ctx->stream));
    k_inner_init<<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(nrhs, B.sc, rr0, delta2);
    CHECK_LAUNCH();
    if (!gexec) {
      uint64_t l0 = ctx->launches;
      CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      dlma_status cs = DLMA_OK;
      for (int k = 0; k < chunk && cs == DLMA_OK; k++) cs = inner_iteration<PB, PS>(ctx, B, nrhs);
      if (cs == DLMA_OK) {
        k_count<<<1, 256, 0, ctx->stream>>>(B.sc.active, nrhs, B.sc.count);
        ctx->launches++;
      }
      cudaError_t ce = cudaMemcpyAsync(hcount, B.sc.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
      cudaError_t ee = cudaStreamEndCapture(ctx->stream, &graph);
      if (cs != DLMA_OK) return cs;
      if (ce != cudaSuccess || ee != cudaSuccess)
        return set_err(ctx, DLMA_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ee != cudaSuccess ? ee : ce));
      CU(cudaGraphInstantiate(&gexec, graph, 0));
      graph_kernels = ctx->launches - l0;
      ctx->launches = l0;
    }
    int it = 0;
    while (it < max_inner) {
      CU(cudaGraphLaunch(gexec, ctx->stream));
      ctx->launches += graph_kernels;
      it += chunk;
      CU(cudaStreamSynchronize(ctx->stream));
      if (hcount[1] || hcount[0] == 0) break;
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      if (el > wall_limit_s) { st = set_err(ctx, DLMA_ERR_TIMEOUT, "solve exceeded %.0f s", wall_limit_s); break; }
    }
    if (st != DLMA_OK) break;
    if (hcount[1]) { st = set_err(ctx, DLMA_ERR_NONFINITE, "non-finite value in the inner solve"); break; }
    // x64 += |r| * x_l
    k_accum<PB><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (double2*)B.x64.data, B.xl.data, B.sc.rnorm,
                                            B.sc.outer_active);
    CHECK_LAUNCH();
    std::vector<int> hit(nrhs);
    CU(cudaMemcpyAsync(hit.data(), B.sc.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < nrhs; j++) iters_total[j] += hit[j];
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (st != DLMA_OK && st != DLMA_ERR_NOT_CONVERGED) return st;
  // x_o = T_oo^-1 (b_o - D_oe x_e)
  {
    HopOp r;
    r.p_out = 1; r.own = 1; r.kout = 3; r.s = -1.0;
    TRY(launch_hop(ctx, r, B.x64, &B.b_o, B.t64o));
  }
  TRY(unpack_parity(ctx, B.x64, 1, 0, x_dev));
  TRY(unpack_parity(ctx, B.t64o, 1, 1, x_dev));
  // true residual ||b - D x|| / ||b|| on the full lattice in FP64
  {
    Field xe = B.r64;   // reuse: x_e in r64, x_o in t64o already
    CU(cudaMemcpyAsync(xe.data, B.x64.data, field_bytes_per_rhs(DLMA_FP64, Vh) * nrhs, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    HopOp d;
    d.own = 2; d.kout = 0; d.p_out = 0;
    TRY(launch_hop(ctx, d, B.t64o, &xe, B.t64));            // (Dx)_e
    k_sub64<<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (const double2*)B.b_e.data, (const double2*)B.t64.data,
                                        (double2*)B.bh.data, nullptr, B.part);
    CHECK_LAUNCH();
    TRY(rowsum(ctx, B.part, gv.x, nrhs, rr0, 0));
    d.p_out = 1;
    TRY(launch_hop(ctx, d, xe, &B.t64o, B.t64));            // (Dx)_o
    k_sub64<<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (const double2*)B.b_o.data, (const double2*)B.t64.data,
                                        (double2*)B.bh.data, nullptr, B.part);
    CHECK_LAUNCH();
    TRY(rowsum(ctx, B.part, gv.x, nrhs, B.sc.rnorm, 0));
    std::vector<double> h(2 * nrhs);
    CU(cudaMemcpyAsync(h.data(), rr0, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(h.data() + nrhs, B.sc.rnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    bool all = true;
    for (int j = 0; j < nrhs; j++) {
      double res = bn[j] > 0 ? sqrt(h[j] + h[nrhs + j]) / bn[j] : 0.0;
      int conv = res <= tol;
      all = all && conv;
      if (info) {
        info[j].iters_inner = iters_total[j];
        info[j].iters_outer = outer;
        info[j].true_resid = res;
        info[j].converged = conv;
      }
    }
    if (st == DLMA_OK && !all) st = set_err(ctx, DLMA_ERR_NOT_CONVERGED, "true residual above tolerance");
  }
  return st;
}

dlma_status solve_fields(dlma_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, double tol, dlma_prec inner,
                         dlma_solve_info* info) {
  // batch size bounded by the memory cap (or 85% of free memory)
  const size_t Vh = ctx->g.Vh;
  size_t per_rhs = field_bytes_per_rhs(DLMA_FP64, Vh) * 7;
  int pb = inner == DLMA_FP64 ? DLMA_FP64 : DLMA_FP32;
  per_rhs += field_bytes_per_rhs(pb, Vh) * 3 + field_bytes_per_rhs(inner, Vh) * 5;
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  size_t budget = (size_t)(0.85 * (double)(freeb + ctx->work_bytes));
  if (ctx->memcap) budget = ctx->memcap;
  int nb = (int)std::min<size_t>((size_t)nrhs, budget / per_rhs);
  if (nb < 1) return set_err(ctx, DLMA_ERR_OOM, "one right-hand side needs %zu bytes", per_rhs);
  dlma_status worst = DLMA_OK;
  for (int j0 = 0; j0 < nrhs; j0 += nb) {
    int n = std::min(nb, nrhs - j0);
    const double* b = b_dev + (size_t)j0 * ctx->g.V * 24;
    double* x = x_dev + (size_t)j0 * ctx->g.V * 24;
    dlma_solve_info* inf = info ? info + j0 : nullptr;
    dlma_status s;
    if (inner == DLMA_FP64) s = solve_batch<DLMA_FP64, DLMA_FP64>(ctx, b, x, n, tol, inf, 0.1 * tol, 200000, 20);
    else if (inner == DLMA_FP32) s = solve_batch<DLMA_FP32, DLMA_FP32>(ctx, b, x, n, tol, inf, 1e-5, 20000, 40);
    else s = solve_batch<DLMA_FP32, DLMA_FP16S>(ctx, b, x, n, tol, inf, 3e-3, 20000, 60);
    if (s != DLMA_OK && s != DLMA_ERR_NOT_CONVERGED) return s;
    if (s != DLMA_OK) worst = s;
  }
  return worst;
}

extern "C" dlma_status dlma_solve(dlma_ctx* ctx, const double* b, double* x, int nrhs, double tol, dlma_prec inner,
                                  dlma_solve_info* info, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge || !ctx->have_params) return set_err(ctx, DLMA_ERR_STATE, "gauge / params not set");
  if (!b || !x || nrhs < 1 || !(tol > 0) || inner < DLMA_FP64 || inner > DLMA_FP16S)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_solve");
  CU(cudaSetDevice(ctx->device));
  size_t bytes = (size_t)nrhs * ctx->g.V * 12 * 16;
  const double* db;
  TRY(copy_in(ctx, WS_SRC, b, bytes, mem, &db));
  double* dx = x;
  if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_SOL, bytes / 8, &dx));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, ctx->stream));
  dlma_status s = solve_fields(ctx, db, dx, nrhs, tol, inner, info);
  CU(cudaEventRecord(e1, ctx->stream));
  if (s == DLMA_OK || s == DLMA_ERR_NOT_CONVERGED) {
    dlma_status c = copy_out(ctx, x, dx, bytes, mem);
    if (c != DLMA_OK) return c;
  }
  CU(cudaStreamSynchronize(ctx->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  ctx->timing[0] = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}
