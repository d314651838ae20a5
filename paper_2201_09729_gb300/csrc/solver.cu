// Multi-right-hand-side Dirac solves x = D^-1 b (the propagator solves of
// Eq. 4 and of the perambulator after Eq. 3).
//
// Even-odd Schur system Dhat x_e = bhat, bhat = b_e - D_eo T_oo^-1 b_o, solved
// by CG on the normal equations Dhat^dag Dhat x_e = Dhat^dag bhat (CGNE).
// Precision scheme (reliable updates): the Krylov iteration runs in FP32 (or
// FP16 with per-site scales for the stencil, FP32 vector algebra) on the system
// scaled by s_j = |bhat_j|.  When a right-hand side's iterated residual has
// dropped by a factor delta since its last update, it pauses; at the end of the
// chunk its low-precision solution is folded into the FP64 solution, the true
// Schur residual r = bhat - Dhat x is recomputed in FP64 and, unless it is below
// the tolerance, the iterated normal-equation residual is replaced by
// Dhat^dag r / s_j and the iteration resumes with the same search direction.
// Every right-hand side carries its own CG scalars on the device and is retired
// (masked out of every kernel) once converged.  A chunk of iterations is
// captured once into a CUDA graph and replayed; the host polls one pinned
// counter per chunk, with an iteration cap and a wall-clock limit, so a solve
// never waits without bound.
#include "fieldio.cuh"
#include <chrono>
#include <thread>
#include <math.h>

namespace {

constexpr int BX = 128;   // sites per block for vector kernels

struct CgScal {
  double* rr;      // current |r|^2 of the (scaled) normal equations
  double* alpha;
  double* beta;
  double* stop2;   // |r|^2 that triggers the next reliable update
  double* rnorm;   // FP64 Schur residual norm per rhs (at the last update)
  double* bnorm;   // |b| per rhs (full lattice)
  double* scale;   // s_j = |bhat_j|: the low-precision system solves for x / s_j
  double* rrnew;   // recomputed |r|^2 after an update
  int* active;     // iterating
  int* alive;      // not yet converged
  int* ru;         // paused for a reliable update
  int* upd;        // update and resume (ru and not converged)
  int* iters;      // inner iterations in total
  int* since;      // inner iterations since the last update
  int* nupd;       // reliable updates
  double* rbest;   // smallest FP64 residual seen at an update
  int* stall;      // consecutive updates without halving rbest
  int* rst;        // restart the search direction at this update (p = r)
  int* cf;         // mask of the final full-lattice residual evaluation
  int* exact;      // rnorm comes from an FP64 evaluation of bhat - Dhat x64
  int* count;      // [0] iterating, [1] nonfinite flag, [2] paused for update
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// alpha_j = |r|^2 / |Dhat p|^2 (one warp per rhs over the stencil's partial sums)
__global__ void k_cg_alpha(const double* part, int nb, int nrhs, CgScal sc) {
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs || !sc.active[j]) return;
  const int lane = threadIdx.x & 31;
  double s = 0;
  for (int b = lane; b < nb; b += 32) s += part[(size_t)j * nb + b];
  s = warp_sum(s);
  if (lane == 0) {
    const double qq = s;
    const double a = sc.rr[j] / qq;
    const bool ok = qq > 0 && isfinite(qq) && isfinite(a);
    sc.alpha[j] = ok ? a : 0.0;
    if (!ok) {
      sc.active[j] = 0;
      sc.ru[j] = 1;                       // hand over to the FP64 check
      if (!isfinite(qq)) sc.count[1] = 1;
    }
  }
}

// beta_j; pause for a reliable update when |r|^2 fell below stop2 or after max_since iterations
__global__ void k_cg_beta(const double* part, int nb, int nrhs, CgScal sc, int max_since, double delta2) {
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs || !sc.active[j]) return;
  const int lane = threadIdx.x & 31;
  double s = 0;
  for (int b = lane; b < nb; b += 32) s += part[(size_t)j * nb + b];
  s = warp_sum(s);
  if (lane == 0) {
    const double rrn = s;
    const double bt = rrn / sc.rr[j];
    sc.beta[j] = isfinite(bt) ? bt : 0.0;
    sc.rr[j] = rrn;
    sc.iters[j] += 1;
    sc.since[j] += 1;
    if (!isfinite(rrn)) { sc.active[j] = 0; sc.count[1] = 1; }
    // request a reliable update; the pause takes effect after this iteration's
    // p update (k_pause), so the search direction stays consistent with r.  An
    // exhausted recursion (|r| = 0 or an overflowing beta) also asks for the FP64 check.
    else if (rrn <= sc.stop2[j] || sc.since[j] >= max_since || !(rrn > 0) || !isfinite(bt) ||
             rrn * delta2 > 1e4 * sc.stop2[j])    // |r|^2 grew 1e4 x above its value at the last update
      sc.ru[j] = 1;
  }
}

// apply the pauses requested in k_cg_beta once p has been updated
__global__ void k_pause(int nrhs, CgScal sc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nrhs && sc.ru[j]) sc.active[j] = 0;
}

// End of one pass of the persistent solve loop: count the iterating rhs and decide,
// on the device, whether the WHILE node of the solve graph runs another pass.  It
// stops when no rhs iterates, on a non-finite value, after max_chunks passes
// (count[3] = 1) or when the host has raised the stop flag (count[3] = 2).
__global__ void k_loop(cudaGraphConditionalHandle h, const int* act, const int* ru, int n, int* count, int max_chunks,
                       const volatile int* stop) {
  __shared__ int s0, s2;
  if (threadIdx.x == 0) { s0 = 0; s2 = 0; }
  __syncthreads();
  int c0 = 0, c2 = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) { c0 += act[j] != 0; c2 += ru[j] != 0; }
  atomicAdd(&s0, c0);
  atomicAdd(&s2, c2);
  __syncthreads();
  if (threadIdx.x == 0) {
    count[0] = s0;
    count[2] = s2;
    const int chunks = ++count[4];
    const bool halt = *stop != 0;
    const bool go = (s0 > 0 || s2 > 0) && !count[1] && chunks < max_chunks && !halt;
    if (!go && (s0 > 0 || s2 > 0)) count[3] = halt ? 2 : (count[1] ? 0 : 1);
    cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

// count[0] = iterating rhs, count[2] = rhs paused for an update
__global__ void k_count(const int* act, const int* ru, int n, int* count) {
  __shared__ int s0, s2;
  if (threadIdx.x == 0) { s0 = 0; s2 = 0; }
  __syncthreads();
  int c0 = 0, c2 = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) { c0 += act[j] != 0; c2 += ru[j] != 0; }
  atomicAdd(&s0, c0);
  atomicAdd(&s2, c2);
  __syncthreads();
  if (threadIdx.x == 0) { count[0] = s0; count[2] = s2; }
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

// p = r + beta p  (and the stencil-precision copy when PS != PB)
template <int PB, int PS>
__global__ void __launch_bounds__(BX) k_update_p(int Vh, int nrhs, const void* r, void* p, void* ps, float* pssc,
                                                  CgScal sc) {
  typedef typename PT<PB>::R R;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= Vh || !sc.active[j]) return;
  const size_t sb = field_units_per_rhs(PB, Vh) * 16 * j;
  const R b = (R)sc.beta[j];
  const Spinor<R> rv = load_spinor<PB>((const char*)r + sb, nullptr, Vh, i);
  Spinor<R> pv = load_spinor<PB>((char*)p + sb, nullptr, Vh, i);
#pragma unroll
  for (int s = 0; s < 4; s++)
#pragma unroll
    for (int c = 0; c < 3; c++) pv.c[s][c] = rv.c[s][c] + b * pv.c[s][c];
  store_spinor<PB>((char*)p + sb, nullptr, Vh, i, pv);
  if (PS != PB) {
    const size_t ss = field_units_per_rhs(PS, Vh) * 16 * j;
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
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y;
  const bool on = mask ? mask[j] != 0 : true;
  double n = 0;
  if (i < Vh && on) {
    const size_t si = field_units_per_rhs(PI, Vh) * 16 * j, so = field_units_per_rhs(PO, Vh) * 16 * j;
    const Spinor<typename PT<PI>::R> v =
        load_spinor<PI>((const char*)in + si, insc ? insc + (size_t)j * Vh : nullptr, Vh, i);
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

// x64 += f_j * lo; lo = 0   (reliable update: fold the low-precision solution into FP64)
template <int PL>
__global__ void __launch_bounds__(BX) k_fold(int Vh, int nrhs, double2* x, void* lo, const double* f,
                                              const int* mask) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= Vh || !mask[j]) return;
  const size_t sl = field_units_per_rhs(PL, Vh) * 16 * j;
  const Spinor<typename PT<PL>::R> v = load_spinor<PL>((const char*)lo + sl, nullptr, Vh, i);
  const double ff = f[j];
  double2* xb = x + (size_t)12 * Vh * j;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    double2 e = xb[(size_t)k * Vh + i];
    e.x += ff * (double)v.c[k / 3][k % 3].re;
    e.y += ff * (double)v.c[k / 3][k % 3].im;
    xb[(size_t)k * Vh + i] = e;
  }
  Spinor<typename PT<PL>::R> z;
#pragma unroll
  for (int s = 0; s < 4; s++)
#pragma unroll
    for (int c = 0; c < 3; c++) z.c[s][c] = cx<typename PT<PL>::R>(0, 0);
  store_spinor<PL>((char*)lo + sl, nullptr, Vh, i, z);
}

// r = a - b (FP64) with |r|^2 partial
__global__ void __launch_bounds__(BX) k_sub64(int Vh, int nrhs, const double2* a, const double2* b, double2* r,
                                               const int* mask, double* part) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y;
  const bool on = mask ? mask[j] != 0 : true;
  double n = 0;
  if (i < Vh && on) {
    const size_t o = (size_t)12 * Vh * j;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double2 x = a[o + (size_t)k * Vh + i], y = b[o + (size_t)k * Vh + i];
      const double2 d = make_double2(x.x - y.x, x.y - y.y);
      r[o + (size_t)k * Vh + i] = d;
      n += d.x * d.x + d.y * d.y;
    }
  }
  block_partial(n, part, on ? j : nrhs, nrhs);
}

// per-rhs totals of a partial buffer: out[j] = sum_b part[j][b] (rows with mask[j] == 0 untouched)
__global__ void k_rowsum(const double* part, int nb, int nrhs, double* out, int do_sqrt, const int* mask) {
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs || (mask && !mask[j])) return;
  const int lane = threadIdx.x & 31;
  double s = 0;
  for (int b = lane; b < nb; b += 32) s += part[(size_t)j * nb + b];
  s = warp_sum(s);
  if (lane == 0) out[j] = do_sqrt ? sqrt(s) : s;
}

// the paused rhs get their residual from an FP64 evaluation at this update
// Split the rhs paused for a reliable update: those whose FP64 residual at the last
// update is already below theta |b| (lo) correct it with an FP32 operator applied to
// the FP32 increment; the rest (hi) recompute it with the FP64 operator.
__global__ void k_split_ru(int nrhs, CgScal sc, double theta, int* ru_hi, int* ru_lo) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs) return;
  const bool lo = sc.ru[j] && sc.rnorm[j] <= theta * sc.bnorm[j];
  ru_lo[j] = lo;
  ru_hi[j] = sc.ru[j] && !lo;
}

// r64 -= s_j t (t = Dhat x_l in the low precision P) with the |r64|^2 partial
template <int P>
__global__ void __launch_bounds__(BX) k_corr64(int Vh, int nrhs, double2* r, const void* t, const double* f,
                                               const int* mask, double* part) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y;
  const bool on = mask[j] != 0;
  double n = 0;
  if (i < Vh && on) {
    const size_t sl = field_units_per_rhs(P, Vh) * 16 * j;
    const Spinor<typename PT<P>::R> v = load_spinor<P>((const char*)t + sl, nullptr, Vh, i);
    const double ff = f[j];
    double2* rb = r + (size_t)12 * Vh * j;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 e = rb[(size_t)k * Vh + i];
      e.x -= ff * (double)v.c[k / 3][k % 3].re;
      e.y -= ff * (double)v.c[k / 3][k % 3].im;
      rb[(size_t)k * Vh + i] = e;
      n += e.x * e.x + e.y * e.y;
    }
  }
  block_partial(n, part, on ? j : nrhs, nrhs);
}

// flag[t] = 1 if any right-hand side has a nonzero block partial of |.|^2 on
// timeslice t (bpt blocks of BX sites per timeslice)
__global__ void k_ts_support(const double* part, int nb, int nrhs, int bpt, int* flag) {
  const int t = blockIdx.x;
  int any = 0;
  for (int e = threadIdx.x; e < nrhs * bpt; e += blockDim.x) {
    const int j = e / bpt, b = t * bpt + e % bpt;
    any |= part[(size_t)j * nb + b] != 0.0;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) flag[t] = any;
}

__global__ void k_mark_exact(int nrhs, CgScal sc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nrhs && sc.ru[j]) sc.exact[j] = 1;
}

// rhs whose reported residual still needs an FP64 evaluation on the full lattice:
// stopped before converging, or retired without an FP64 residual
__global__ void k_final_mask(int nrhs, CgScal sc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nrhs) sc.cf[j] = sc.alive[j] || !sc.exact[j];
}

// after the FP64 residual of the paused rhs: retire the converged, mark the rest for resumption
__global__ void k_ru_check(int nrhs, CgScal sc, double tol) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs || !sc.ru[j]) return;
  sc.nupd[j] += 1;
  const double r = sc.rnorm[j];
  if (!isfinite(r)) { sc.count[1] = 1; sc.alive[j] = 0; sc.upd[j] = 0; sc.ru[j] = 0; return; }
  if (r <= tol * sc.bnorm[j]) { sc.alive[j] = 0; sc.upd[j] = 0; sc.ru[j] = 0; return; }
  // stagnation at the rounding level (an unreachable tolerance): restart the search
  // direction, and give up on this rhs after four updates without progress
  sc.rst[j] = 0;
  if (r < 0.5 * sc.rbest[j]) { sc.rbest[j] = r; sc.stall[j] = 0; }
  else if (++sc.stall[j] >= 4) { sc.alive[j] = 0; sc.upd[j] = 0; sc.ru[j] = 0; return; }
  else sc.rst[j] = 1;
  sc.upd[j] = 1;
}

// resume the updated rhs with the recomputed normal-equation residual
__global__ void k_resume(int nrhs, CgScal sc, double delta2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs || !sc.upd[j]) return;
  const double rr = sc.rrnew[j];
  sc.upd[j] = 0;
  sc.ru[j] = 0;
  sc.since[j] = 0;
  if (!(rr > 0) || !isfinite(rr)) {
    if (!isfinite(rr)) sc.count[1] = 1;
    sc.alive[j] = 0;
    return;
  }
  sc.rr[j] = rr;
  sc.stop2[j] = delta2 * rr;
  sc.active[j] = 1;
}

// ---- BiCGStab (complex, per right-hand side) --------------------------------
// Per-rhs complex scalars of the BiCGStab recursion
struct BiScal {
  double2* rho;     // (r0, r)
  double2* alpha;
  double2* omega;
  double2* beta;
  int* brk;         // breakdown seen: restart the shadow residual at the next update
};

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// a breakdown pauses the rhs for an FP64 update that restarts its shadow residual
__device__ __forceinline__ void bi_breakdown(int j, CgScal& sc, BiScal& bs) {
  sc.active[j] = 0;
  sc.ru[j] = 1;
  bs.brk[j] = 1;
}

// alpha = rho / (r0, v)   (one warp per rhs over the stencil's DOT partials)
__global__ void k_bi_alpha(const double2* dpart, int nb, int nrhs, CgScal sc, BiScal bs) {
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs || !sc.active[j]) return;
  const int lane = threadIdx.x & 31;
  double2 s = make_double2(0, 0);
  for (int b = lane; b < nb; b += 32) {
    const double2 v = dpart[(size_t)j * nb + b];
    s.x += v.x;
    s.y += v.y;
  }
  s = warp_sum2(s);
  if (lane == 0) {
    const double2 a = cdiv(bs.rho[j], s);
    const bool ok = (s.x != 0.0 || s.y != 0.0) && cfinite(s) && cfinite(a);
    bs.alpha[j] = ok ? a : make_double2(0, 0);
    if (!ok) {
      bi_breakdown(j, sc, bs);
      if (!cfinite(s)) sc.count[1] = 1;
    }
  }
}

// s = r - alpha v
template <int P>
__global__ void __launch_bounds__(BX) k_bi_s(int Vh, int nrhs, const void* r, const void* v, void* sv, CgScal sc,
                                             BiScal bs) {
  typedef typename PT<P>::R R;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= Vh || !sc.active[j]) return;
  const size_t sb = field_units_per_rhs(P, Vh) * 16 * j;
  const double2 al = bs.alpha[j];
  const R ar = (R)al.x, ai = (R)al.y;
  const Spinor<R> rv = load_spinor<P>((const char*)r + sb, nullptr, Vh, i);
  const Spinor<R> vv = load_spinor<P>((const char*)v + sb, nullptr, Vh, i);
  Spinor<R> o;
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const Cx<R> x = vv.c[a][c];
      o.c[a][c] = cx<R>(rv.c[a][c].re - (ar * x.re - ai * x.im), rv.c[a][c].im - (ar * x.im + ai * x.re));
    }
  store_spinor<P>((char*)sv + sb, nullptr, Vh, i, o);
}

// omega = (t, s) / (t, t) from the partials of sum conj(s) t and |t|^2
__global__ void k_bi_omega(const double2* dpart, const double* npart, int nb, int nrhs, CgScal sc, BiScal bs) {
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs || !sc.active[j]) return;
  const int lane = threadIdx.x & 31;
  double2 d = make_double2(0, 0);
  double n = 0;
  for (int b = lane; b < nb; b += 32) {
    const double2 v = dpart[(size_t)j * nb + b];
    d.x += v.x;
    d.y += v.y;
    n += npart[(size_t)j * nb + b];
  }
  d = warp_sum2(d);
  n = warp_sum(n);
  if (lane == 0) {
    const double2 ts = make_double2(d.x, -d.y);     // (t, s) = conj(sum conj(s) t)
    const double2 om = make_double2(ts.x / n, ts.y / n);
    const bool ok = n > 0 && isfinite(n) && cfinite(om) && (om.x != 0.0 || om.y != 0.0);
    bs.omega[j] = ok ? om : make_double2(0, 0);
    if (!ok) {
      bi_breakdown(j, sc, bs);
      if (!isfinite(n)) sc.count[1] = 1;
    }
  }
}

// x += alpha p + omega s ; r = s - omega t ; partials of (r0, r) and |r|^2
template <int P>
__global__ void __launch_bounds__(BX) k_bi_xr(int Vh, int nrhs, void* x, void* r, const void* p, const void* sv,
                                              const void* t, const void* r0, CgScal sc, BiScal bs, double2* cpart,
                                              double* npart) {
  typedef typename PT<P>::R R;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y;
  const bool on = sc.active[j] != 0;
  R dr = 0, di = 0, nn = 0;
  if (i < Vh && on) {
    const size_t sb = field_units_per_rhs(P, Vh) * 16 * j;
    const double2 al = bs.alpha[j], om = bs.omega[j];
    const R ar = (R)al.x, ai = (R)al.y, wr = (R)om.x, wi = (R)om.y;
    Spinor<R> xv = load_spinor<P>((const char*)x + sb, nullptr, Vh, i);
    const Spinor<R> pv = load_spinor<P>((const char*)p + sb, nullptr, Vh, i);
    const Spinor<R> svv = load_spinor<P>((const char*)sv + sb, nullptr, Vh, i);
    const Spinor<R> tv = load_spinor<P>((const char*)t + sb, nullptr, Vh, i);
    const Spinor<R> zv = load_spinor<P>((const char*)r0 + sb, nullptr, Vh, i);
    Spinor<R> rv;
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const Cx<R> pp = pv.c[a][c], ss = svv.c[a][c], tt = tv.c[a][c], z = zv.c[a][c];
        xv.c[a][c].re += ar * pp.re - ai * pp.im + wr * ss.re - wi * ss.im;
        xv.c[a][c].im += ar * pp.im + ai * pp.re + wr * ss.im + wi * ss.re;
        const Cx<R> rr = cx<R>(ss.re - (wr * tt.re - wi * tt.im), ss.im - (wr * tt.im + wi * tt.re));
        rv.c[a][c] = rr;
        dr += z.re * rr.re + z.im * rr.im;
        di += z.re * rr.im - z.im * rr.re;
        nn += rr.re * rr.re + rr.im * rr.im;
      }
    store_spinor<P>((char*)x + sb, nullptr, Vh, i, xv);
    store_spinor<P>((char*)r + sb, nullptr, Vh, i, rv);
  }
  __shared__ double red[3][BX / 32];
  double vr = warp_sum((double)dr), vi = warp_sum((double)di), vn = warp_sum((double)nn);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = vr;
    red[1][threadIdx.x >> 5] = vi;
    red[2][threadIdx.x >> 5] = vn;
  }
  __syncthreads();
  if (threadIdx.x == 0 && on) {
    double a0 = 0, a1 = 0, a2 = 0;
    for (int w = 0; w < BX / 32; w++) { a0 += red[0][w]; a1 += red[1][w]; a2 += red[2][w]; }
    cpart[(size_t)j * gridDim.x + blockIdx.x] = make_double2(a0, a1);
    npart[(size_t)j * gridDim.x + blockIdx.x] = a2;
  }
}

// rho_new = (r0, r), |r|^2; beta = (rho_new / rho) (alpha / omega); reliable-update triggers
__global__ void k_bi_beta(const double2* cpart, const double* npart, int nb, int nrhs, CgScal sc, BiScal bs,
                          int max_since, double delta2) {
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs || !sc.active[j]) return;
  const int lane = threadIdx.x & 31;
  double2 d = make_double2(0, 0);
  double n = 0;
  for (int b = lane; b < nb; b += 32) {
    const double2 v = cpart[(size_t)j * nb + b];
    d.x += v.x;
    d.y += v.y;
    n += npart[(size_t)j * nb + b];
  }
  d = warp_sum2(d);
  n = warp_sum(n);
  if (lane == 0) {
    const double2 bt = cmul(cdiv(d, bs.rho[j]), cdiv(bs.alpha[j], bs.omega[j]));
    const bool ok = cfinite(bt) && (d.x != 0.0 || d.y != 0.0);
    bs.beta[j] = ok ? bt : make_double2(0, 0);
    bs.rho[j] = d;
    sc.rr[j] = n;
    sc.iters[j] += 1;
    sc.since[j] += 1;
    if (!isfinite(n)) { sc.active[j] = 0; sc.count[1] = 1; }
    else if (!ok) { sc.ru[j] = 1; bs.brk[j] = 1; }
    else if (n <= sc.stop2[j] || sc.since[j] >= max_since || !(n > 0) || n * delta2 > 1e4 * sc.stop2[j])
      sc.ru[j] = 1;                        // the pause takes effect after the p update (k_pause)
  }
}

// p = r + beta (p - omega v)
template <int P>
__global__ void __launch_bounds__(BX) k_bi_p(int Vh, int nrhs, const void* r, void* p, const void* v, CgScal sc,
                                             BiScal bs) {
  typedef typename PT<P>::R R;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= Vh || !sc.active[j]) return;
  const size_t sb = field_units_per_rhs(P, Vh) * 16 * j;
  const double2 bt = bs.beta[j], om = bs.omega[j];
  const R br = (R)bt.x, bi = (R)bt.y, wr = (R)om.x, wi = (R)om.y;
  const Spinor<R> rv = load_spinor<P>((const char*)r + sb, nullptr, Vh, i);
  const Spinor<R> vv = load_spinor<P>((const char*)v + sb, nullptr, Vh, i);
  Spinor<R> pv = load_spinor<P>((const char*)p + sb, nullptr, Vh, i);
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const Cx<R> vx = vv.c[a][c];
      const Cx<R> d = cx<R>(pv.c[a][c].re - (wr * vx.re - wi * vx.im), pv.c[a][c].im - (wr * vx.im + wi * vx.re));
      pv.c[a][c] = cx<R>(rv.c[a][c].re + br * d.re - bi * d.im, rv.c[a][c].im + br * d.im + bi * d.re);
    }
  store_spinor<P>((char*)p + sb, nullptr, Vh, i, pv);
}

// End of a BiCGStab reliable update in one pass over the updated rhs: r_l = r64 / s_j
// (FP64 -> P); where the shadow residual restarts (rmask) r0 = p = r_l; partials of
// (r0, r_l) and |r_l|^2 for k_bi_resume
template <int P>
__global__ void __launch_bounds__(BX) k_bi_restore(int Vh, int nrhs, const double2* r64, const double* f, void* rl,
                                                   void* r0, void* pl, const int* upd, const int* rmask,
                                                   double2* cpart, double* npart) {
  typedef typename PT<P>::R R;
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y;
  const bool on = upd[j] != 0;
  double dr = 0, di = 0, nn = 0;
  if (i < Vh && on) {
    const size_t so = field_units_per_rhs(P, Vh) * 16 * j;
    const Spinor<double> v = load_spinor<DLMA_FP64>((const char*)r64 + (size_t)192 * Vh * j, nullptr, Vh, i);
    const double ff = f[j] > 0 ? 1.0 / f[j] : 0.0;
    Spinor<R> o;
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) o.c[s][c] = cx<R>((R)(ff * v.c[s][c].re), (R)(ff * v.c[s][c].im));
    store_spinor<P>((char*)rl + so, nullptr, Vh, i, o);
    Spinor<R> a;
    if (rmask[j]) {
      store_spinor<P>((char*)r0 + so, nullptr, Vh, i, o);
      store_spinor<P>((char*)pl + so, nullptr, Vh, i, o);
      a = o;
    } else {
      a = load_spinor<P>((const char*)r0 + so, nullptr, Vh, i);
    }
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const Cx<R> x = a.c[s][c], y = o.c[s][c];
        dr += (double)x.re * y.re + (double)x.im * y.im;
        di += (double)x.re * y.im - (double)x.im * y.re;
        nn += (double)y.re * y.re + (double)y.im * y.im;
      }
  }
  __shared__ double red[3][BX / 32];
  dr = warp_sum(dr);
  di = warp_sum(di);
  nn = warp_sum(nn);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = dr;
    red[1][threadIdx.x >> 5] = di;
    red[2][threadIdx.x >> 5] = nn;
  }
  __syncthreads();
  if (threadIdx.x == 0 && on) {
    double a0 = 0, a1 = 0, a2 = 0;
    for (int w = 0; w < BX / 32; w++) { a0 += red[0][w]; a1 += red[1][w]; a2 += red[2][w]; }
    cpart[(size_t)j * gridDim.x + blockIdx.x] = make_double2(a0, a1);
    npart[(size_t)j * gridDim.x + blockIdx.x] = a2;
  }
}

// resume the updated rhs: rho = (r0, r), |r|^2 from the partials; restart flags consumed
__global__ void k_bi_resume(const double2* cpart, const double* npart, int nb, int nrhs, CgScal sc, BiScal bs,
                            double delta2) {
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (j >= nrhs || !sc.upd[j]) return;
  const int lane = threadIdx.x & 31;
  double2 d = make_double2(0, 0);
  double n = 0;
  for (int b = lane; b < nb; b += 32) {
    const double2 v = cpart[(size_t)j * nb + b];
    d.x += v.x;
    d.y += v.y;
    n += npart[(size_t)j * nb + b];
  }
  d = warp_sum2(d);
  n = warp_sum(n);
  if (lane == 0) {
    sc.upd[j] = 0;
    sc.ru[j] = 0;
    sc.since[j] = 0;
    bs.brk[j] = 0;
    if (!(n > 0) || !isfinite(n) || !cfinite(d)) {
      if (!isfinite(n)) sc.count[1] = 1;
      sc.alive[j] = 0;
      return;
    }
    bs.rho[j] = d;
    sc.rr[j] = n;
    sc.stop2[j] = delta2 * n;
    sc.active[j] = 1;
  }
}

// updated rhs that restart their shadow residual: the stagnating ones and those that broke down
__global__ void k_bi_restart_mask(int nrhs, CgScal sc, BiScal bs, int first, int* rmask) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs) return;
  rmask[j] = sc.upd[j] && (first || sc.rst[j] || bs.brk[j]);
}

}  // namespace

// ---------------------------------------------------------------------------
struct SolveBufs {
  Field b_e, b_o, bh, x64, r64, t64, t64o;     // FP64
  Field xl, rl, pl, ps, q, z, tmp, rhs;        // low precision (pl: vector precision, ps/q/z/tmp/rhs: stencil)
  double *part, *part2;
  CgScal sc;
  // BiCGStab: v = Dhat p (q), s, t = Dhat s (z), shadow residual r0; complex partials
  Field sl, r0;
  double2 *cpart, *cpart2;
  int* rmask;
  int *ru_hi, *ru_lo;   // BiCGStab updates: FP64 operator / FP32 correction of the residual
  BiScal bs;
  // host copies of the set-up
  std::vector<double> bn;
  std::vector<int> alive0;
  double* tmpd = nullptr;
};

static dlma_status rowsum(dlma_ctx* ctx, const double* part, int nb, int nrhs, double* out, int do_sqrt,
                          const int* mask) {
  k_rowsum<<<(nrhs + 3) / 4, 128, 0, ctx->stream>>>(part, nb, nrhs, out, do_sqrt, mask);
  CHECK_LAUNCH();
  return DLMA_OK;
}

template <int PB, int PS>
static dlma_status inner_iteration(dlma_ctx* ctx, SolveBufs& B, int nrhs, int max_since, double delta2) {
  const int Vh = ctx->g.Vh;
  const dim3 gv((Vh + BX - 1) / BX, nrhs);
  const int nbh = hop_grid_x(ctx, PS);
  // q = Dhat p ; |q|^2 partials
  TRY(schur_apply(ctx, B.ps, B.tmp, B.q, 0, B.sc.active, B.part));
  k_cg_alpha<<<(nrhs + 3) / 4, 128, 0, ctx->stream>>>(B.part, nbh, nrhs, B.sc);
  CHECK_LAUNCH();
  // z = Dhat^dag q with the update x += alpha p, r -= alpha z fused into its epilogue
  TRY(schur_dag_cgupdate(ctx, B.q, B.tmp, B.sc.active, B.xl, B.rl, B.pl, B.sc.alpha, B.part2));
  k_cg_beta<<<(nrhs + 3) / 4, 128, 0, ctx->stream>>>(B.part2, nbh, nrhs, B.sc, max_since, delta2);
  CHECK_LAUNCH();
  k_update_p<PB, PS><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.rl.data, B.pl.data, B.ps.data, B.ps.scale, B.sc);
  CHECK_LAUNCH();
  k_pause<<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(nrhs, B.sc);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// Reliable update of the rhs in mask ru: x64 += s x_l, x_l = 0; r64 = bhat - Dhat x64 (FP64);
// retire the converged ones; for the others r_l = Dhat^dag (r64 / s) and resume.
// first: the initial update (nothing to fold); restart: also reset p = r (a plain
// defect-correction restart, used with the FP16 stencil whose rounding makes the
// kept search direction inconsistent with the recomputed residual)
template <int PB, int PS>
static dlma_status reliable_update(dlma_ctx* ctx, SolveBufs& B, int nrhs, double tol_target, double delta2,
                                   bool first, bool restart = false) {
  const int Vh = ctx->g.Vh;
  const dim3 gv((Vh + BX - 1) / BX, nrhs);
  const int* ru = B.sc.ru;
  const int nb1 = (nrhs + 127) / 128;
  if (first) {
    // x64 = 0: the residual is bhat itself, |bhat| = s
    CU(cudaMemcpyAsync(B.r64.data, B.bh.data, field_bytes_per_rhs(DLMA_FP64, Vh) * nrhs, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    CU(cudaMemcpyAsync(B.sc.rnorm, B.sc.scale, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    k_fold<PB><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (double2*)B.x64.data, B.xl.data, B.sc.scale, ru);
    CHECK_LAUNCH();
    TRY(schur_apply(ctx, B.x64, B.t64o, B.t64, 0, ru, nullptr));
    k_sub64<<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (const double2*)B.bh.data, (const double2*)B.t64.data,
                                        (double2*)B.r64.data, ru, B.part2);
    CHECK_LAUNCH();
    TRY(rowsum(ctx, B.part2, gv.x, nrhs, B.sc.rnorm, 1, ru));
  }
  k_mark_exact<<<nb1, 128, 0, ctx->stream>>>(nrhs, B.sc);
  CHECK_LAUNCH();
  k_ru_check<<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(nrhs, B.sc, tol_target);
  CHECK_LAUNCH();
  const int* upd = B.sc.upd;
  // r_l = Dhat^dag (r64 / s) in the stencil precision, then in the vector precision
  k_convert<DLMA_FP64, PS><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.r64.data, nullptr, B.rhs.data, B.rhs.scale,
                                                       B.sc.scale, 1, upd, nullptr);
  CHECK_LAUNCH();
  TRY(schur_apply(ctx, B.rhs, B.tmp, B.z, 1, upd, nullptr));
  k_convert<PS, PB><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.z.data, B.z.scale, B.rl.data, nullptr, nullptr, 0, upd,
                                                B.part2);
  CHECK_LAUNCH();
  TRY(rowsum(ctx, B.part2, gv.x, nrhs, B.sc.rrnew, 0, upd));
  {
    // p = r_l (and its stencil-precision copy): for every updated rhs on the first
    // update or when restarting, otherwise only for the stagnating ones
    const int* pm = (first || restart) ? upd : B.sc.rst;
    k_convert<PB, PB><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.rl.data, nullptr, B.pl.data, nullptr, nullptr, 0, pm,
                                                  nullptr);
    CHECK_LAUNCH();
    if (PS != PB) {
      k_convert<PB, PS><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.rl.data, nullptr, B.ps.data, B.ps.scale, nullptr, 0,
                                                    pm, nullptr);
      CHECK_LAUNCH();
    }
  }
  k_resume<<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(nrhs, B.sc, delta2);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// Set-up shared by the solvers: buffers, per-rhs scalars, the even-odd source
// bhat = b_e - D_eo T_oo^-1 b_o, |b| and s = |bhat| (the low-precision systems
// solve for x / s), and the initial masks.
template <int PB, int PS>
static dlma_status solve_setup(dlma_ctx* ctx, SolveBufs& B, const double* b_dev, int nrhs, bool bicg) {
  const int Vh = ctx->g.Vh;
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
  if (bicg) {
    TRY(field_alloc(ctx, WS_BI_S, PB, nrhs, &B.sl));
    TRY(field_alloc(ctx, WS_BI_R0, PB, nrhs, &B.r0));
  }
  const int nbmax = (Vh + 31) / 32 + 8;
  TRY(workT(ctx, WS_PART, (size_t)2 * nbmax * nrhs, &B.part));
  B.part2 = B.part + (size_t)nbmax * nrhs;
  if (bicg) {
    TRY(workT(ctx, WS_BI_PART, (size_t)2 * nbmax * nrhs, &B.cpart));
    B.cpart2 = B.cpart + (size_t)nbmax * nrhs;
  }
  double* sd;
  TRY(workT(ctx, WS_SCAL, (size_t)10 * nrhs + 64, &sd));
  B.sc.rr = sd;
  B.sc.alpha = sd + nrhs;
  B.sc.beta = sd + 2 * nrhs;
  B.sc.stop2 = sd + 3 * nrhs;
  B.sc.rnorm = sd + 4 * nrhs;
  B.sc.bnorm = sd + 5 * nrhs;
  B.sc.scale = sd + 6 * nrhs;
  B.sc.rrnew = sd + 7 * nrhs;
  B.tmpd = sd + 8 * nrhs;     // 2 nrhs scratch
  TRY(workT(ctx, WS_T0, (size_t)nrhs + 16, &B.sc.rbest));
  int* si;
  TRY(workT(ctx, WS_ACT, (size_t)16 * nrhs + 32, &si));
  B.sc.active = si;
  B.sc.alive = si + nrhs;
  B.sc.ru = si + 2 * nrhs;
  B.sc.upd = si + 3 * nrhs;
  B.sc.iters = si + 4 * nrhs;
  B.sc.since = si + 5 * nrhs;
  B.sc.nupd = si + 6 * nrhs;
  B.sc.stall = si + 7 * nrhs;
  B.sc.rst = si + 8 * nrhs;
  B.sc.cf = si + 9 * nrhs;
  B.sc.exact = si + 10 * nrhs;
  B.ru_hi = si + 11 * nrhs;
  B.bs.brk = si + 12 * nrhs;
  B.rmask = si + 13 * nrhs;
  B.ru_lo = si + 14 * nrhs;
  B.sc.count = si + 16 * nrhs;     // [0] iterating, [1] non-finite, [2] paused, [3] stop reason, [4] passes
  if (bicg) {
    double2* cs;
    TRY(workT(ctx, WS_BI_SCAL, (size_t)4 * nrhs + 16, &cs));
    B.bs.rho = cs;
    B.bs.alpha = cs + nrhs;
    B.bs.omega = cs + 2 * nrhs;
    B.bs.beta = cs + 3 * nrhs;
  }

  const dim3 gv((Vh + BX - 1) / BX, nrhs);
  TRY(pack_parity(ctx, b_dev, 1, 0, B.b_e));
  TRY(pack_parity(ctx, b_dev, 1, 1, B.b_o));
  // |b|^2 over both parities
  k_convert<DLMA_FP64, DLMA_FP64><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.b_e.data, nullptr, B.t64.data, nullptr,
                                                              nullptr, 0, nullptr, B.part);
  CHECK_LAUNCH();
  TRY(rowsum(ctx, B.part, gv.x, nrhs, B.tmpd, 0, nullptr));
  k_convert<DLMA_FP64, DLMA_FP64><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.b_o.data, nullptr, B.t64o.data, nullptr,
                                                              nullptr, 0, nullptr, B.part);
  CHECK_LAUNCH();
  // the timeslices on which b_o is nonzero (for whole-timeslice blocks)
  const int T = ctx->g.T, hsl = ctx->g.Vs / 2;
  const bool ts_blocks = hsl % BX == 0 && T >= 6;
  int* dflag = nullptr;
  std::vector<int> tsf(T, 1);
  if (ts_blocks) {
    TRY(workT(ctx, WS_SUPPORT, (size_t)T, &dflag));
    k_ts_support<<<T, 256, 0, ctx->stream>>>(B.part, gv.x, nrhs, hsl / BX, dflag);
    CHECK_LAUNCH();
    CU(cudaMemcpyAsync(tsf.data(), dflag, sizeof(int) * T, cudaMemcpyDeviceToHost, ctx->stream));
  }
  TRY(rowsum(ctx, B.part, gv.x, nrhs, B.tmpd + nrhs, 0, nullptr));
  CU(cudaStreamSynchronize(ctx->stream));
  // smallest cyclic run of timeslices t0 .. t0 + k - 1 holding every nonzero of b_o
  int t0 = 0, k = T;
  {
    int nz = 0;
    for (int t = 0; t < T; t++) nz += tsf[t] != 0;
    if (nz == 0) k = 0;
    else if (nz < T) {
      int best = T;
      for (int t = 0; t < T; t++) {          // a run ends where the next zero gap begins
        if (!tsf[t] || tsf[(t + T - 1) % T]) continue;
        int last = t, l = 0;
        for (int d = 0; d < T; d++) if (tsf[(t + d) % T]) last = d;
        l = last + 1;
        if (l < best) { best = l; t0 = t; }
      }
      k = best;
    }
  }
  // bhat = b_e - D_eo T_oo^-1 b_o and |bhat|.  With b_o supported on k + 4 < T
  // timeslices (the sources of one source timeslice), T_oo^-1 b_o is formed on those
  // k and zeroed on the two on either side, and the hop changes b_e only on the k + 2
  // timeslices next to them: the rest of bhat is b_e.
  {
    HopOp a;
    a.p_out = 1; a.hop = 0; a.own = 1; a.kout = 3;
    HopOp b;
    b.p_out = 0; b.own = 1; b.kout = 0; b.s = -1.0;
    const size_t fb = field_bytes_per_rhs(DLMA_FP64, Vh) * nrhs;
    if (ts_blocks && k + 4 < T) {
      CU(cudaMemcpyAsync(B.bh.data, B.b_e.data, fb, cudaMemcpyDeviceToDevice, ctx->stream));
      if (k > 0) {
        // zero T_oo^-1 b_o on t0 - 2 .. t0 + k + 1: 12 nrhs rows of double2 per field
        for (int d = -2; d < k + 2; d++) {
          const int t = ((t0 + d) % T + T) % T;
          CU(cudaMemset2DAsync((char*)B.t64o.data + (size_t)t * hsl * 16, (size_t)Vh * 16, 0, (size_t)hsl * 16,
                               (size_t)12 * nrhs, ctx->stream));
        }
        a.site0 = t0 * hsl;
        a.nsites = k * hsl;
        TRY(launch_hop(ctx, a, B.b_o, &B.b_o, B.t64o));
        b.site0 = ((t0 - 1 + T) % T) * hsl;
        b.nsites = (k + 2) * hsl;
        TRY(launch_hop(ctx, b, B.t64o, &B.b_e, B.bh));
      }
    } else {
      TRY(launch_hop(ctx, a, B.b_o, &B.b_o, B.t64o));
      TRY(launch_hop(ctx, b, B.t64o, &B.b_e, B.bh));
    }
  }
  k_convert<DLMA_FP64, DLMA_FP64><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.bh.data, nullptr, B.t64.data, nullptr,
                                                              nullptr, 0, nullptr, B.part);
  CHECK_LAUNCH();
  TRY(rowsum(ctx, B.part, gv.x, nrhs, B.sc.scale, 1, nullptr));
  std::vector<double> hb(2 * nrhs), hs(nrhs);
  CU(cudaMemcpyAsync(hb.data(), B.tmpd, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(hs.data(), B.sc.scale, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  B.bn.assign(nrhs, 0.0);
  B.alive0.assign(nrhs, 0);
  std::vector<int> zeros(nrhs, 0);
  for (int j = 0; j < nrhs; j++) {
    B.bn[j] = sqrt(hb[j] + hb[nrhs + j]);
    if (!isfinite(B.bn[j]) || !isfinite(hs[j])) return set_err(ctx, DLMA_ERR_NONFINITE, "a source holds NaN or Inf");
    B.alive0[j] = B.bn[j] > 0 && hs[j] > 0;
  }
  CU(cudaMemcpyAsync(B.sc.bnorm, B.bn.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemcpyAsync(B.sc.alive, B.alive0.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemcpyAsync(B.sc.ru, B.alive0.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
  for (int* z : {B.sc.active, B.sc.upd, B.sc.iters, B.sc.since, B.sc.nupd, B.sc.stall, B.sc.rst, B.sc.cf,
                 B.sc.exact, B.bs.brk})
    CU(cudaMemcpyAsync(z, zeros.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
  std::vector<double> big(nrhs, 1e300);
  CU(cudaMemcpyAsync(B.sc.rbest, big.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemsetAsync(B.sc.count, 0, 4 * sizeof(int), ctx->stream));
  CU(cudaMemsetAsync(B.x64.data, 0, field_bytes_per_rhs(DLMA_FP64, Vh) * nrhs, ctx->stream));
  CU(cudaMemsetAsync(B.xl.data, 0, field_bytes_per_rhs(PB, Vh) * nrhs, ctx->stream));
  // pack one full-batch right-hand side for the block-shape autotuner before any capture
  k_convert<DLMA_FP64, PS><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.bh.data, nullptr, B.rhs.data, B.rhs.scale,
                                                       B.sc.scale, 1, nullptr, nullptr);
  CHECK_LAUNCH();
  TRY(autotune_hop(ctx, PS, B.rhs, B.tmp, B.z));
  return DLMA_OK;
}

// x_o = T_oo^-1 (b_o - D_oe x_e), the full solution to x_dev, and the reported
// residual of every right-hand side
template <int PB>
static dlma_status solve_finish(dlma_ctx* ctx, SolveBufs& B, double* x_dev, int nrhs, double tol,
                                dlma_solve_info* info, dlma_status st) {
  const int Vh = ctx->g.Vh;
  const dim3 gv((Vh + BX - 1) / BX, nrhs);
  // fold what is left of the low-precision solutions of unconverged rhs
  if (st != DLMA_OK) {
    k_fold<PB><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (double2*)B.x64.data, B.xl.data, B.sc.scale, B.sc.alive);
    CHECK_LAUNCH();
  }
  {
    HopOp r;
    r.p_out = 1; r.own = 1; r.kout = 3; r.s = -1.0;
    TRY(launch_hop(ctx, r, B.x64, &B.b_o, B.t64o));
  }
  TRY(unpack_parity(ctx, B.x64, 1, 0, x_dev));
  TRY(unpack_parity(ctx, B.t64o, 1, 1, x_dev));
  // reported residual ||b - D x|| / ||b||: for an rhs retired on an FP64 residual it is
  // that residual, |bhat - Dhat x_e| (x_o above makes the odd rows of b - D x vanish);
  // the rest (stopped early, or retired on a recursive residual) are evaluated on the
  // full lattice in FP64 here
  k_final_mask<<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(nrhs, B.sc);
  CHECK_LAUNCH();
  const int* fm = B.sc.cf;
  Field xe = B.r64;
  CU(cudaMemcpyAsync(xe.data, B.x64.data, field_bytes_per_rhs(DLMA_FP64, Vh) * nrhs, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  HopOp d;
  d.own = 2; d.kout = 0; d.p_out = 0; d.active = fm;
  TRY(launch_hop(ctx, d, B.t64o, &xe, B.t64));            // (Dx)_e
  k_sub64<<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (const double2*)B.b_e.data, (const double2*)B.t64.data,
                                      (double2*)B.bh.data, fm, B.part);
  CHECK_LAUNCH();
  TRY(rowsum(ctx, B.part, gv.x, nrhs, B.tmpd, 0, fm));
  d.p_out = 1;
  TRY(launch_hop(ctx, d, xe, &B.t64o, B.t64));            // (Dx)_o
  k_sub64<<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (const double2*)B.b_o.data, (const double2*)B.t64.data,
                                      (double2*)B.bh.data, fm, B.part);
  CHECK_LAUNCH();
  TRY(rowsum(ctx, B.part, gv.x, nrhs, B.tmpd + nrhs, 0, fm));
  std::vector<double> h(2 * nrhs), hr(nrhs);
  std::vector<int> hit(nrhs), hup(nrhs), hm(nrhs);
  CU(cudaMemcpyAsync(h.data(), B.tmpd, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(hr.data(), B.sc.rnorm, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(hm.data(), fm, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(hit.data(), B.sc.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(hup.data(), B.sc.nupd, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  bool all = true;
  for (int j = 0; j < nrhs; j++) {
    const double rn = hm[j] ? sqrt(h[j] + h[nrhs + j]) : (B.alive0[j] ? hr[j] : 0.0);
    const double res = B.bn[j] > 0 ? rn / B.bn[j] : 0.0;
    const int conv = res <= tol;
    all = all && conv;
    if (info) {
      info[j].iters_inner = hit[j];
      info[j].iters_outer = hup[j];
      info[j].true_resid = res;
      info[j].converged = conv;
    }
  }
  if (st == DLMA_OK && !all) st = set_err(ctx, DLMA_ERR_NOT_CONVERGED, "true residual above tolerance");
  return st;
}

// The persistent iteration loop shared by the solvers.  After the first reliable
// update (`update(true)`), one CUDA graph runs the whole solve: a WHILE
// conditional node whose body is `chunk` iterations (`body`), the reliable
// update of the rhs paused in them (`update(false)`: every kernel of it is masked
// by the paused / updated rhs, so a pass without pauses costs only empty
// launches) and k_loop, which decides on the device whether to run another pass.
// The host launches the graph once and waits by polling with a wall-clock
// limit; at the limit it raises a stop flag in pinned memory that k_loop reads,
// so the graph ends after the pass in flight and no wait is unbounded.
// With DLMA_SOLVE_GRAPH=0 in the environment of a solve the same
// passes are launched from the host one by one, each followed by a count of the
// iterating rhs: the same kernels and arithmetic, visible one by one to kernel
// profilers that do not look inside conditional graphs.
template <class Body, class Update>
static dlma_status iterate_host(dlma_ctx* ctx, SolveBufs& B, int nrhs, int max_inner, int chunk, Body body,
                                Update update) {
  int* hcount = (int*)ctx->pinned;
  const int max_chunks = std::max(1, max_inner / chunk);
  for (int pass = 0; pass < max_chunks; pass++) {
    for (int k = 0; k < chunk; k++) TRY(body());
    TRY(update(false));
    k_count<<<1, 256, 0, ctx->stream>>>(B.sc.active, B.sc.ru, nrhs, B.sc.count);
    CHECK_LAUNCH();
    CU(cudaMemcpyAsync(hcount, B.sc.count, 8 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (hcount[1]) return set_err(ctx, DLMA_ERR_NONFINITE, "non-finite value in the solve");
    if (hcount[0] == 0 && hcount[2] == 0) return DLMA_OK;
  }
  return set_err(ctx, DLMA_ERR_NOT_CONVERGED, "iteration cap %d reached", max_inner);
}

template <class Body, class Update>
static dlma_status iterate(dlma_ctx* ctx, SolveBufs& B, int nrhs, int max_inner, Body body, Update update) {
  volatile int* hpin = (volatile int*)ctx->pinned;   // [0..7] counts (copied back), [16] stop flag
  int* hcount = (int*)ctx->pinned;
  const int chunk = 8;
  const double wall_limit_s = 600.0;
  TRY(update(true));
  CU(cudaMemsetAsync(B.sc.count, 0, 8 * sizeof(int), ctx->stream));
  // DLMA_SOLVE_GRAPH is read at every solve, so one context can run both forms
  const char* sg = getenv("DLMA_SOLVE_GRAPH");
  if (sg && atoi(sg) == 0) return iterate_host(ctx, B, nrhs, max_inner, chunk, body, update);
  hpin[16] = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  CU(cudaGraphCreate(&graph, 0));
  auto fail = [&](dlma_status s) {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    return s;
  };
  cudaGraphConditionalHandle handle;
  cudaError_t ce = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  if (ce != cudaSuccess) return fail(set_err(ctx, DLMA_ERR_CUDA, "conditional handle: %s", cudaGetErrorString(ce)));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  ce = cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &cp);
  if (ce != cudaSuccess) return fail(set_err(ctx, DLMA_ERR_CUDA, "WHILE node: %s", cudaGetErrorString(ce)));
  cudaGraph_t loop_body = cp.conditional.phGraph_out[0];
  const uint64_t l0 = ctx->launches;
  ce = cudaStreamBeginCaptureToGraph(ctx->stream, loop_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) return fail(set_err(ctx, DLMA_ERR_CUDA, "capture: %s", cudaGetErrorString(ce)));
  dlma_status cs = DLMA_OK;
  for (int k = 0; k < chunk && cs == DLMA_OK; k++) cs = body();
  if (cs == DLMA_OK) cs = update(false);
  if (cs == DLMA_OK) {
    k_loop<<<1, 256, 0, ctx->stream>>>(handle, B.sc.active, B.sc.ru, nrhs, B.sc.count,
                                       std::max(1, max_inner / chunk), (const volatile int*)(hpin + 16));
    ctx->launches++;
  }
  cudaGraph_t captured = nullptr;
  ce = cudaStreamEndCapture(ctx->stream, &captured);
  if (cs != DLMA_OK) return fail(cs);
  if (ce != cudaSuccess) return fail(set_err(ctx, DLMA_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce)));
  const uint64_t body_kernels = ctx->launches - l0;
  ctx->launches = l0;
  ce = cudaGraphInstantiate(&gexec, graph, 0);
  if (ce != cudaSuccess) return fail(set_err(ctx, DLMA_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce)));
  ce = cudaGraphLaunch(gexec, ctx->stream);
  if (ce != cudaSuccess) return fail(set_err(ctx, DLMA_ERR_CUDA, "graph launch: %s", cudaGetErrorString(ce)));
  // bounded wait: poll; at the wall-clock limit ask the device loop to stop
  const auto t_start = std::chrono::steady_clock::now();
  bool stopped = false;
  while (true) {
    const cudaError_t q = cudaStreamQuery(ctx->stream);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return fail(set_err(ctx, DLMA_ERR_CUDA, "solve graph: %s", cudaGetErrorString(q)));
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (!stopped && el > wall_limit_s) {
      hpin[16] = 1;
      stopped = true;
    }
    if (stopped && el > 2 * wall_limit_s)
      return fail(set_err(ctx, DLMA_ERR_TIMEOUT, "solve graph did not stop after the wall-clock limit"));
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  CU(cudaMemcpyAsync(hcount, B.sc.count, 8 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->launches += body_kernels * (uint64_t)std::max(0, hcount[4]);
  cudaGraphExecDestroy(gexec);
  cudaGraphDestroy(graph);
  if (hcount[1]) return set_err(ctx, DLMA_ERR_NONFINITE, "non-finite value in the solve");
  if (hcount[3] == 2) return set_err(ctx, DLMA_ERR_TIMEOUT, "solve exceeded %.0f s", wall_limit_s);
  if (hcount[3] == 1) return set_err(ctx, DLMA_ERR_NOT_CONVERGED, "iteration cap %d reached", max_inner);
  return DLMA_OK;
}

template <int PB, int PS>
static dlma_status solve_batch(dlma_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, double tol,
                               dlma_solve_info* info, double delta, int max_inner, int max_since) {
  SolveBufs B;
  TRY((solve_setup<PB, PS>(ctx, B, b_dev, nrhs, false)));
  const double tol_target = 0.5 * tol;
  const double delta2 = delta * delta;
  // the first "update" sets r_l = Dhat^dag (bhat / s) and p = r_l
  dlma_status st = iterate(
      ctx, B, nrhs, max_inner, [&]() { return inner_iteration<PB, PS>(ctx, B, nrhs, max_since, delta2); },
      [&](bool first) {
        return reliable_update<PB, PS>(ctx, B, nrhs, tol_target, delta2, first, !first && PS == DLMA_FP16S);
      });
  if (st != DLMA_OK && st != DLMA_ERR_NOT_CONVERGED && st != DLMA_ERR_TIMEOUT) return st;
  return solve_finish<PB>(ctx, B, x_dev, nrhs, tol, info, st);
}

// ---- BiCGStab on the Schur system, FP32 (or FP64) vectors and stencil ------
// Per iteration: v = Dhat p with (r0, v); alpha = rho / (r0, v); s = r - alpha v;
// t = Dhat s with (s, t) and |t|^2; omega = (t, s) / |t|^2; x += alpha p + omega s;
// r = s - omega t with (r0, r) and |r|^2; beta = (rho' / rho)(alpha / omega);
// p = r + beta (p - omega v).  Two operator applications per iteration, the inner
// products in the stencil's and the vector kernels' epilogues.
template <int P>
static dlma_status bicg_iteration(dlma_ctx* ctx, SolveBufs& B, int nrhs, int max_since, double delta2) {
  const int Vh = ctx->g.Vh;
  const dim3 gv((Vh + BX - 1) / BX, nrhs);
  const int nbh = hop_grid_x(ctx, P);
  const int nw = (nrhs + 3) / 4;
  // v = Dhat p (into q) with the partials of (r0, v)
  TRY(schur_apply_dot(ctx, B.pl, B.tmp, B.q, B.sc.active, B.r0, B.cpart, nullptr));
  k_bi_alpha<<<nw, 128, 0, ctx->stream>>>(B.cpart, nbh, nrhs, B.sc, B.bs);
  CHECK_LAUNCH();
  k_bi_s<P><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.rl.data, B.q.data, B.sl.data, B.sc, B.bs);
  CHECK_LAUNCH();
  // t = Dhat s (into z) with the partials of sum conj(s) t and |t|^2
  TRY(schur_apply_dot(ctx, B.sl, B.tmp, B.z, B.sc.active, B.sl, B.cpart, B.part));
  k_bi_omega<<<nw, 128, 0, ctx->stream>>>(B.cpart, B.part, nbh, nrhs, B.sc, B.bs);
  CHECK_LAUNCH();
  k_bi_xr<P><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.xl.data, B.rl.data, B.pl.data, B.sl.data, B.z.data, B.r0.data,
                                         B.sc, B.bs, B.cpart2, B.part2);
  CHECK_LAUNCH();
  k_bi_beta<<<nw, 128, 0, ctx->stream>>>(B.cpart2, B.part2, gv.x, nrhs, B.sc, B.bs, max_since, delta2);
  CHECK_LAUNCH();
  k_bi_p<P><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, B.rl.data, B.pl.data, B.q.data, B.sc, B.bs);
  CHECK_LAUNCH();
  k_pause<<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(nrhs, B.sc);
  CHECK_LAUNCH();
  return DLMA_OK;
}

// Reliable update of the paused rhs: x64 += s x_l, x_l = 0, r64 = bhat - Dhat x64 in
// FP64; the converged retire; the rest continue with r_l = r64 / s and rho = (r0, r_l),
// restarting r0 = p = r_l on the first update, after a breakdown or on stagnation.
template <int P>
static dlma_status bicg_update(dlma_ctx* ctx, SolveBufs& B, int nrhs, double tol_target, double delta2, bool first) {
  const int Vh = ctx->g.Vh;
  const dim3 gv((Vh + BX - 1) / BX, nrhs);
  const int* ru = B.sc.ru;
  const int nb1 = (nrhs + 127) / 128;
  if (first) {
    CU(cudaMemcpyAsync(B.r64.data, B.bh.data, field_bytes_per_rhs(DLMA_FP64, Vh) * nrhs, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    CU(cudaMemcpyAsync(B.sc.rnorm, B.sc.scale, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
  } else if (P == DLMA_FP32) {
    // x64 += s x_l.  r64 = bhat - Dhat x64 changes by -s Dhat x_l: for rhs whose last
    // residual is below theta |b| that change is applied with the FP32 operator, whose
    // relative rounding (~1e-6 with the cancellation between hop and clover terms)
    // leaves an error below 1e-3 of the target tolerance; the others evaluate the
    // residual with the FP64 operator
    const double theta = 1e-3 * tol_target / 1.2e-7;
    k_split_ru<<<nb1, 128, 0, ctx->stream>>>(nrhs, B.sc, theta, B.ru_hi, B.ru_lo);
    CHECK_LAUNCH();
    TRY(schur_apply(ctx, B.xl, B.tmp, B.q, 0, B.ru_lo, nullptr));
    k_fold<P><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (double2*)B.x64.data, B.xl.data, B.sc.scale, ru);
    CHECK_LAUNCH();
    TRY(schur_apply(ctx, B.x64, B.t64o, B.t64, 0, B.ru_hi, nullptr));
    k_sub64<<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (const double2*)B.bh.data, (const double2*)B.t64.data,
                                        (double2*)B.r64.data, B.ru_hi, B.part2);
    CHECK_LAUNCH();
    k_corr64<P><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (double2*)B.r64.data, B.q.data, B.sc.scale, B.ru_lo,
                                            B.part2);
    CHECK_LAUNCH();
    TRY(rowsum(ctx, B.part2, gv.x, nrhs, B.sc.rnorm, 1, ru));
  } else {
    k_fold<P><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (double2*)B.x64.data, B.xl.data, B.sc.scale, ru);
    CHECK_LAUNCH();
    TRY(schur_apply(ctx, B.x64, B.t64o, B.t64, 0, ru, nullptr));
    k_sub64<<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (const double2*)B.bh.data, (const double2*)B.t64.data,
                                        (double2*)B.r64.data, ru, B.part2);
    CHECK_LAUNCH();
    TRY(rowsum(ctx, B.part2, gv.x, nrhs, B.sc.rnorm, 1, ru));
  }
  k_mark_exact<<<nb1, 128, 0, ctx->stream>>>(nrhs, B.sc);
  CHECK_LAUNCH();
  k_ru_check<<<nb1, 128, 0, ctx->stream>>>(nrhs, B.sc, tol_target);
  CHECK_LAUNCH();
  const int* upd = B.sc.upd;
  k_bi_restart_mask<<<nb1, 128, 0, ctx->stream>>>(nrhs, B.sc, B.bs, first ? 1 : 0, B.rmask);
  CHECK_LAUNCH();
  k_bi_restore<P><<<gv, BX, 0, ctx->stream>>>(Vh, nrhs, (const double2*)B.r64.data, B.sc.scale, B.rl.data, B.r0.data,
                                               B.pl.data, upd, B.rmask, B.cpart2, B.part2);
  CHECK_LAUNCH();
  k_bi_resume<<<(nrhs + 3) / 4, 128, 0, ctx->stream>>>(B.cpart2, B.part2, gv.x, nrhs, B.sc, B.bs, delta2);
  CHECK_LAUNCH();
  return DLMA_OK;
}

template <int P>
static dlma_status solve_batch_bicg(dlma_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, double tol,
                                    dlma_solve_info* info, double delta, int max_inner, int max_since) {
  SolveBufs B;
  TRY((solve_setup<P, P>(ctx, B, b_dev, nrhs, true)));
  const double tol_target = 0.5 * tol;
  const double delta2 = delta * delta;
  dlma_status st = iterate(
      ctx, B, nrhs, max_inner, [&]() { return bicg_iteration<P>(ctx, B, nrhs, max_since, delta2); },
      [&](bool first) { return bicg_update<P>(ctx, B, nrhs, tol_target, delta2, first); });
  if (st != DLMA_OK && st != DLMA_ERR_NOT_CONVERGED && st != DLMA_ERR_TIMEOUT) return st;
  return solve_finish<P>(ctx, B, x_dev, nrhs, tol, info, st);
}

// One batch with the context's solver choice.  BiCGStab serves FP32 inner solves;
// right-hand sides it leaves above the tolerance are solved again with CGNE.
static dlma_status solve_one_batch(dlma_ctx* ctx, const double* b, double* x, int n, double tol, dlma_prec inner,
                                   dlma_solve_info* inf) {
  // delta: reduction of the iterated residual between FP64 reliable updates
  if (inner == DLMA_FP64) return solve_batch<DLMA_FP64, DLMA_FP64>(ctx, b, x, n, tol, inf, 1e-6, 200000, 100000);
  if (inner == DLMA_FP16S) return solve_batch<DLMA_FP32, DLMA_FP16S>(ctx, b, x, n, tol, inf, 3e-3, 40000, 400);
  if (ctx->solver != DLMA_SOLVER_BICGSTAB)
    return solve_batch<DLMA_FP32, DLMA_FP32>(ctx, b, x, n, tol, inf, 3e-4, 40000, 400);
  std::vector<dlma_solve_info> li(n);
  // the reduction of |r| between FP64 updates (DLMA_BICG_DELTA overrides it for tuning)
  double delta = 3e-4;
  if (const char* e = getenv("DLMA_BICG_DELTA")) delta = std::min(0.5, std::max(1e-8, atof(e)));
  dlma_status s = solve_batch_bicg<DLMA_FP32>(ctx, b, x, n, tol, li.data(), delta, 20000, 200);
  if (s != DLMA_OK && s != DLMA_ERR_NOT_CONVERGED && s != DLMA_ERR_TIMEOUT) return s;
  std::vector<int> bad;
  for (int j = 0; j < n; j++)
    if (!li[j].converged) bad.push_back(j);
  if (!bad.empty()) {
    // gather the unconverged sources, solve them with CGNE, scatter the solutions back
    const size_t fb = (size_t)ctx->g.V * 24 * sizeof(double);
    double *gb, *gx;
    TRY(workT(ctx, WS_RETRY_B, bad.size() * fb / sizeof(double), &gb));
    TRY(workT(ctx, WS_RETRY_X, bad.size() * fb / sizeof(double), &gx));
    for (size_t q = 0; q < bad.size(); q++)
      CU(cudaMemcpyAsync((char*)gb + q * fb, (const char*)b + bad[q] * fb, fb, cudaMemcpyDeviceToDevice, ctx->stream));
    std::vector<dlma_solve_info> ri(bad.size());
    s = solve_batch<DLMA_FP32, DLMA_FP32>(ctx, gb, gx, (int)bad.size(), tol, ri.data(), 3e-4, 40000, 400);
    if (s != DLMA_OK && s != DLMA_ERR_NOT_CONVERGED && s != DLMA_ERR_TIMEOUT) return s;
    for (size_t q = 0; q < bad.size(); q++) {
      CU(cudaMemcpyAsync((char*)x + bad[q] * fb, (const char*)gx + q * fb, fb, cudaMemcpyDeviceToDevice, ctx->stream));
      ri[q].iters_inner += li[bad[q]].iters_inner;
      ri[q].iters_outer += li[bad[q]].iters_outer;
      li[bad[q]] = ri[q];
    }
    CU(cudaStreamSynchronize(ctx->stream));
  }
  bool all = true;
  for (int j = 0; j < n; j++) all = all && li[j].converged;
  if (inf) memcpy(inf, li.data(), sizeof(dlma_solve_info) * n);
  return all ? DLMA_OK : set_err(ctx, DLMA_ERR_NOT_CONVERGED, "true residual above tolerance");
}

// Batch-size autotuner: the stencil's time per right-hand side at the largest
// batch memory allows (nb) and at nb / 2, nb / 4, measured once per precision on
// the context's own lattice (the choice is kept until a larger batch fits); the
// solves then run in batches of the cheapest size.  Links and clover are shared
// by every right-hand side of a batch, so larger batches usually win; the
// measurement decides where L2 reuse or occupancy says otherwise.
static dlma_status autotune_batch(dlma_ctx* ctx, dlma_prec prec, int nb, int* out) {
  if (ctx->batch_tuned[prec] && nb <= ctx->batch_tuned_nb[prec]) {
    *out = std::min(nb, ctx->batch_rhs[prec]);
    return DLMA_OK;
  }
  Field in, tmp, res;
  TRY(field_alloc(ctx, WS_CG_RHS, prec, nb, &in));
  TRY(field_alloc(ctx, WS_CG_TMP, prec, nb, &tmp));
  TRY(field_alloc(ctx, WS_CG_Z, prec, nb, &res));
  CU(cudaMemsetAsync(in.data, 0, field_bytes_per_rhs(prec, ctx->g.Vh) * nb, ctx->stream));
  TRY(autotune_hop(ctx, prec, in, tmp, res));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  int best_k = nb;
  double best = 1e300;
  for (int k : {nb, (nb + 1) / 2, (nb + 3) / 4}) {
    Field a = in, t = tmp, r = res;
    a.nrhs = t.nrhs = r.nrhs = k;
    float tmin = 1e30f;
    for (int rep = 0; rep < 3; rep++) {
      CU(cudaEventRecord(e0, ctx->stream));
      TRY(schur_apply(ctx, a, t, r, 0, nullptr, nullptr));
      CU(cudaEventRecord(e1, ctx->stream));
      CU(cudaEventSynchronize(e1));
      float ms = 0;
      CU(cudaEventElapsedTime(&ms, e0, e1));
      tmin = std::min(tmin, ms);
    }
    const double per = tmin / k;
    if (per < 0.97 * best) { best = per; best_k = k; }    // a smaller batch must win clearly
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->batch_rhs[prec] = best_k;
  ctx->batch_tuned_nb[prec] = nb;
  ctx->batch_tuned[prec] = 1;
  *out = std::min(nb, best_k);
  return DLMA_OK;
}

dlma_status solve_fields(dlma_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, double tol, dlma_prec inner,
                         dlma_solve_info* info) {
  // batch size bounded by the memory cap (or 85% of free memory)
  const size_t Vh = ctx->g.Vh;
  size_t per_rhs = field_bytes_per_rhs(DLMA_FP64, Vh) * 7;
  const int pb = inner == DLMA_FP64 ? DLMA_FP64 : DLMA_FP32;
  per_rhs += field_bytes_per_rhs(pb, Vh) * 5 + field_bytes_per_rhs(inner, Vh) * 5;
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  size_t budget = (size_t)(0.85 * (double)(freeb + ctx->work_bytes));
  if (ctx->memcap) budget = ctx->memcap;
  int nb = (int)std::min<size_t>((size_t)nrhs, budget / per_rhs);
  if (nb < 1) return set_err(ctx, DLMA_ERR_OOM, "one right-hand side needs %zu bytes", per_rhs);
  if (inner != DLMA_FP64 && nb > 16) TRY(autotune_batch(ctx, inner, nb, &nb));
  dlma_status worst = DLMA_OK;
  for (int j0 = 0; j0 < nrhs; j0 += nb) {
    const int n = std::min(nb, nrhs - j0);
    const double* b = b_dev + (size_t)j0 * ctx->g.V * 24;
    double* x = x_dev + (size_t)j0 * ctx->g.V * 24;
    dlma_solve_info* inf = info ? info + j0 : nullptr;
    const dlma_status s = solve_one_batch(ctx, b, x, n, tol, inner, inf);
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
  const size_t bytes = (size_t)nrhs * ctx->g.V * 12 * 16;
  const double* db;
  TRY(copy_in(ctx, WS_SRC, b, bytes, mem, &db));
  double* dx = x;
  if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_SOL, bytes / 8, &dx));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, ctx->stream));
  const dlma_status s = solve_fields(ctx, db, dx, nrhs, tol, inner, info);
  CU(cudaEventRecord(e1, ctx->stream));
  if (s == DLMA_OK || s == DLMA_ERR_NOT_CONVERGED) {
    const dlma_status c = copy_out(ctx, x, dx, bytes, mem);
    if (c != DLMA_OK) return c;
  }
  CU(cudaStreamSynchronize(ctx->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  for (int i = 0; i < kTimingSlots; i++) ctx->timing[i] = 0;
  ctx->timing[0] = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}
