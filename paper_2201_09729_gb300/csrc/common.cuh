// Shared device / host helpers of the dlma library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>
#include <string.h>
#include <vector>
#include <string>

#include "../../include/dlma.h"

// ---------------------------------------------------------------------------
// complex arithmetic on (re, im) pairs, templated on the real type
template <class R> struct Cx { R re, im; };

template <class R> __host__ __device__ __forceinline__ Cx<R> cx(R a, R b) { Cx<R> z; z.re = a; z.im = b; return z; }
template <class R> __host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return cx<R>(a.re + b.re, a.im + b.im); }
template <class R> __host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return cx<R>(a.re - b.re, a.im - b.im); }
template <class R> __host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a) { return cx<R>(-a.re, -a.im); }
template <class R> __host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return cx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R> __host__ __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return cx<R>(s * a.re, s * a.im); }
template <class R> __host__ __device__ __forceinline__ Cx<R> conj(Cx<R> a) { return cx<R>(a.re, -a.im); }
// i * a
template <class R> __host__ __device__ __forceinline__ Cx<R> mul_i(Cx<R> a) { return cx<R>(-a.im, a.re); }
// a += b * c
template <class R> __host__ __device__ __forceinline__ void fma_acc(Cx<R>& a, Cx<R> b, Cx<R> c) {
  a.re = fma(b.re, c.re, a.re); a.re = fma(-b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im); a.im = fma(b.im, c.re, a.im);
}
// a += conj(b) * c
template <class R> __host__ __device__ __forceinline__ void fma_conj_acc(Cx<R>& a, Cx<R> b, Cx<R> c) {
  a.re = fma(b.re, c.re, a.re); a.re = fma(b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im); a.im = fma(-b.im, c.re, a.im);
}
template <class R> __host__ __device__ __forceinline__ R norm2(Cx<R> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------------------
// lattice geometry: even-odd compressed index <-> coordinates.
// Site s = x + L (y + L (z + L t)); parity p = (x+y+z+t) & 1; for even L the
// compressed index of s within its parity is s >> 1.
struct Geom {
  int L, T, V, Vh, Vs;
};

struct Coord { int x, y, z, t; };

__host__ __device__ __forceinline__ Coord eo_coords(const Geom& g, int p, int i) {
  int s0 = 2 * i;
  Coord c;
  int x0 = s0 % g.L;
  int r = s0 / g.L;
  c.y = r % g.L; r /= g.L;
  c.z = r % g.L;
  c.t = r / g.L;
  c.x = x0 + ((c.y + c.z + c.t + p) & 1);
  return c;
}
__host__ __device__ __forceinline__ int lex_of(const Geom& g, int x, int y, int z, int t) {
  return x + g.L * (y + g.L * (z + g.L * t));
}
// neighbour in direction mu (0 t, 1 x, 2 y, 3 z), sign +1 / -1, periodic wrap; lexicographic index
__host__ __device__ __forceinline__ int nbr_lex(const Geom& g, Coord c, int mu, int sgn) {
  int x = c.x, y = c.y, z = c.z, t = c.t;
  if (mu == 0) { t += sgn; t = t < 0 ? g.T - 1 : (t >= g.T ? 0 : t); }
  else if (mu == 1) { x += sgn; x = x < 0 ? g.L - 1 : (x >= g.L ? 0 : x); }
  else if (mu == 2) { y += sgn; y = y < 0 ? g.L - 1 : (y >= g.L ? 0 : y); }
  else { z += sgn; z = z < 0 ? g.L - 1 : (z >= g.L ? 0 : z); }
  return lex_of(g, x, y, z, t);
}

// ---------------------------------------------------------------------------
// device buffers owned by the context (grow-on-demand work space)
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// slots of dlma_last_timing (meaning per call: see include/dlma.h)
constexpr int kTimingSlots = 8;

struct dlma_ctx {
  Geom g;
  int bc_t = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;      // created by dlma_create when the caller passed NULL
  char err[512];
  uint64_t launches = 0;
  uint64_t memcap = 0;
  uint64_t work_bytes = 0;      // bytes currently held in work buffers
  double timing[kTimingSlots] = {0};
  // stencil block shape (sites x right-hand sides) per precision, chosen by autotune_hop
  int hop_sx[3] = {64, 64, 64}, hop_sy[3] = {4, 4, 4}, hop_tuned[3] = {0, 0, 0};
  int hop_l18[3] = {0, 0, 0};   // FP32: read 18-real links instead of rebuilding row 2
  int hop_chunk[3] = {64, 64, 64};   // right-hand sides per chunk of the stencil's block order
  int hop_nr[3] = {1, 1, 1};    // FP32: right-hand sides per thread (1 or 2)
  // the Laplacian eigensolver's FP64 phase computes its Gram matrices and rotations
  // in double-float (dfloat.cuh) for tol >= 1e-11; DLMA_DF_EIGS=0 at context
  // creation keeps FP64 arithmetic
  int df_eigs = 1;
  // solve batch size per precision, chosen by autotune_batch (valid up to batch_tuned_nb)
  int batch_rhs[3] = {0, 0, 0}, batch_tuned_nb[3] = {0, 0, 0}, batch_tuned[3] = {0, 0, 0};

  bool have_gauge = false, have_params = false;
  double m0 = 0, csw = 0;
  int solver = DLMA_SOLVER_BICGSTAB;   // Krylov method of the FP32 inner solves
  // generations of the gauge field and of the cached modes: a checkpoint taken
  // under one generation is stale under the next
  uint64_t gauge_gen = 0, eig_gen = 0;

  // gauge: U_mu(x) for x in parity p, SoA over the compressed site index
  double2* Ucan = nullptr;  // [V][4][3][3] canonical copy (clover build)
  double2* U64 = nullptr;   // [2][4][9][Vh]
  float4* U32 = nullptr;    // [2][4][3][Vh]  rows 0, 1 (12 reals)
  float4* U32f = nullptr;   // [2][4][5][Vh]  all 9 entries (18 reals + 2 pad): no reconstruction
  uint4* U16a = nullptr;    // [2][4][Vh]     halves 0..7 of rows 0, 1
  uint2* U16b = nullptr;    // [2][4][Vh]     halves 8..11
  double2* U3 = nullptr;    // [3][9][V]      spatial links, lexicographic, for the Laplacian
  float4* U3f = nullptr;    // [3][3][V]      spatial links 12-real fp32
  // clover: 2 hermitian 6x6 blocks per site packed as 72 reals
  // (per block: 6 real diagonal entries, then the 15 complex entries below the diagonal, row-major)
  double2* C64 = nullptr;   // [2][36][Vh]  T(x)
  double2* Ci64 = nullptr;  // [2][36][Vh]  T(x)^-1
  float4* C32 = nullptr;    // [2][18][Vh]
  float4* Ci32 = nullptr;
  uint4* C16 = nullptr;     // [2][9][Vh]
  uint4* Ci16 = nullptr;
  int* flag = nullptr;      // device status flags [16]
  // neighbour table of the stencil: for output parity p, int4 words w = 0, 1 hold
  // directions 4w .. 4w+3 (direction 2 mu + 0 forward / 1 backward): the compressed
  // index of the neighbour in parity 1 - p; bit 31 set when the hop picks up the
  // antiperiodic time phase.  Layout int4 [2][2][V/2].
  int4* nbr_tab = nullptr;

  // cached Laplacian modes (all timeslices)
  int eig_N = 0;
  double2* eig_V = nullptr;       // [N][T][Vs][3]
  std::vector<double> eig_lam;    // [T][N]
  std::vector<int> eig_have;      // [T] modes cached for timeslice t

  // cached Dirac low modes (eigenvectors of g5 Dhat on the even sites), FP64 [N][12][V/2]
  int dirac_N = 0;
  double2* dirac_V = nullptr;

  // checkpointed forward solutions of dlma_correlators (for the backward):
  // [4N distillation, then phi_r, phibar_r per noise][V][4][3] complex
  int checkpoint = 0;
  double* ckpt = nullptr;
  int ckpt_J = 0, ckpt_N = 0, ckpt_nn = 0, ckpt_tsrc = -1;
  // state the checkpointed forward ran under, and its serial number (0: none)
  double ckpt_m0 = 0, ckpt_csw = 0;
  uint64_t ckpt_gauge_gen = 0, ckpt_eig_gen = 0, ckpt_serial = 0, ckpt_count = 0;

  // named work buffers
  DevBuf wb[64];
  void* pinned = nullptr;         // small pinned host staging area
};

enum WorkSlot {
  WS_IN = 0, WS_OUT, WS_T0, WS_T1, WS_T2,
  WS_SOLVE_B, WS_SOLVE_X64, WS_SOLVE_R64, WS_SOLVE_BH, WS_SOLVE_TMP64,
  WS_CG_X, WS_CG_R, WS_CG_P, WS_CG_PLO, WS_CG_Q, WS_CG_Z, WS_CG_TMP, WS_CG_RHS,
  WS_SCAL, WS_PART, WS_ACT, WS_ITERS,
  WS_EIG_X, WS_EIG_Y, WS_EIG_Y2, WS_EIG_W, WS_EIG_G, WS_EIG_PART, WS_EIG_S, WS_EIG_AUX,
  WS_PROJ_V, WS_PROJ_PART, WS_PROJ_C, WS_CON, WS_CON2, WS_SRC, WS_SOL, WS_ETA,
  WS_BI_S, WS_BI_R0, WS_BI_PART, WS_BI_SCAL, WS_RETRY_B, WS_RETRY_X,
  WS_TC_A, WS_TC_B, WS_TC_E, WS_SUPPORT,
  WS_COUNT
};

// ---------------------------------------------------------------------------
// error handling
dlma_status set_err(dlma_ctx* ctx, dlma_status st, const char* fmt, ...);

#define CU(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return set_err(ctx, DLMA_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, \
                     cudaGetErrorString(e_));                                      \
  } while (0)

#define CHECK_LAUNCH()                                                              \
  do {                                                                              \
    cudaError_t e_ = cudaGetLastError();                                            \
    if (e_ != cudaSuccess)                                                          \
      return set_err(ctx, DLMA_ERR_CUDA, "%s:%d launch: %s", __FILE__, __LINE__,      \
                     cudaGetErrorString(e_));                                       \
    ctx->launches++;                                                                \
  } while (0)

#define TRY(call)                       \
  do {                                  \
    dlma_status s_ = (call);            \
    if (s_ != DLMA_OK) return s_;       \
  } while (0)

// work buffer of at least `bytes` in slot `slot` (contents not preserved on growth)
dlma_status work(dlma_ctx* ctx, int slot, size_t bytes, void** out);
template <class T> dlma_status workT(dlma_ctx* ctx, int slot, size_t count, T** out) {
  void* p;
  dlma_status s = work(ctx, slot, count * sizeof(T), &p);
  *out = (T*)p;
  return s;
}

// ---------------------------------------------------------------------------
// internal fields: even-odd half-lattice spinors in one precision, SoA over
// the compressed site index.  Per right-hand side:
//   FP64  double2 [12][Vh]
//   FP32  float4  [6][Vh]      (complex components 2q, 2q+1 in one float4)
//   FP16S uint4   [3][Vh]      (complex components 4q..4q+3) + float scale [Vh]
struct Field {
  void* data = nullptr;
  float* scale = nullptr;
  int prec = DLMA_FP64;
  int nrhs = 0;
  int Vh = 0;
};

__host__ __device__ inline size_t field_units_per_rhs(int prec, int Vh) {
  return prec == DLMA_FP64 ? (size_t)12 * Vh : prec == DLMA_FP32 ? (size_t)6 * Vh : (size_t)3 * Vh;
}
inline size_t field_bytes_per_rhs(int prec, int Vh) {
  return prec == DLMA_FP64 ? (size_t)12 * Vh * 16 : prec == DLMA_FP32 ? (size_t)6 * Vh * 16
                                                                      : (size_t)3 * Vh * 16 + (size_t)Vh * 4;
}
dlma_status field_alloc(dlma_ctx* ctx, int slot, int prec, int nrhs, Field* f);

// ---------------------------------------------------------------------------
// cross-file internal entry points
dlma_status copy_in(dlma_ctx* ctx, int slot, const double* p, size_t bytes, dlma_mem mem, const double** dev);
dlma_status copy_out(dlma_ctx* ctx, double* dst, const double* dev, size_t bytes, dlma_mem mem);

// pack canonical complex128 [nrhs][V][4][3] (full lattice) parity p -> field
dlma_status pack_parity(dlma_ctx* ctx, const double* src, int full, int p, Field& f);
// unpack field parity p -> canonical complex128 (full lattice or half)
dlma_status unpack_parity(dlma_ctx* ctx, const Field& f, int full, int p, double* dst);

// stencil (hop) launch: out_p = Kout * (Kown * own + s * hop(in_{1-p}))
struct HopOp {
  int p_out;          // parity of the output sites
  int g5_in = 0;      // apply gamma_5 to the hopping input
  int g5_hop = 0;     // apply gamma_5 to the hopping result
  int own = 0;        // 0: no own-site term, 1: identity, 2: clover T_p, 3: clover inverse T_p^-1
  int kout = 0;       // 0: none, 2: T_p, 3: T_p^-1 applied to the sum
  int hop = 1;        // include the hopping term
  double s = 1.0;     // sign / factor of the hopping term
  double* norm_part = nullptr;   // if set: per (rhs, block) partial |out|^2
  const int* active = nullptr;   // per-rhs mask (nullptr = all)
  // fused CG update instead of storing the output (Schur step B of the adjoint):
  // x += alpha p, r -= alpha out, partial |r|^2 into norm_part
  void* cg_x = nullptr;
  void* cg_r = nullptr;
  const void* cg_p = nullptr;
  const double* cg_alpha = nullptr;
  // DOT epilogue (Schur step B, no gamma_5 on the hop): per (rhs, site tile)
  // partial of sum conj(w) out into dot_part; w is a field in the output precision
  const struct Field* dot_w = nullptr;
  double2* dot_part = nullptr;
  // output sites: the compressed indices site0 .. site0 + nsites - 1 (cyclic modulo
  // V/2; nsites < 0: all).  Whole timeslices are contiguous ranges, so a source
  // supported on few timeslices needs few sites; no partial sums with a range.
  int site0 = 0, nsites = -1;
};
dlma_status launch_hop(dlma_ctx* ctx, const HopOp& op, const Field& in, const Field* own, Field& out,
                       int* nblocks_out = nullptr);
int hop_grid_x(dlma_ctx* ctx, int prec);

// Schur operator on even fields: out = Dhat in (dagger: gamma5 Dhat gamma5), tmp: odd work field
dlma_status schur_apply(dlma_ctx* ctx, const Field& in, Field& tmp, Field& out, int dagger,
                        const int* active, double* norm_part);
dlma_status autotune_hop(dlma_ctx* ctx, int prec, const Field& in, Field& tmp, Field& out);
// out = Dhat in with the partials of sum conj(w) out (dot_part, double2) and, if
// norm_part is set, |out|^2 per (rhs, site tile)
dlma_status schur_apply_dot(dlma_ctx* ctx, const Field& in, Field& tmp, Field& out, const int* active,
                            const Field& w, double2* dot_part, double* norm_part);
// z = Dhat^dag q fused with the CG update x += alpha p, r -= alpha z (x, r, p in the
// vector precision); partial |r|^2 per (rhs, site tile) into part
dlma_status schur_dag_cgupdate(dlma_ctx* ctx, const Field& q, Field& tmp, const int* active, Field& x, Field& r,
                               const Field& p, const double* alpha, double* part);

void gamma_matrices(double G[4][4][4][2]);
dlma_status solve_fields(dlma_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, double tol,
                         dlma_prec inner, dlma_solve_info* info);
// V^dag psi on the tensor cores, FP64-accurate (split-precision digits): coeff[j][Tsel][4][N]
dlma_status project_tc(dlma_ctx* ctx, const double2* VT, int N, int Tsel, const double* psi, size_t stride_sites,
                       int site_t0, int nrhs, double2* coeff);
// sum over kappa of conj(B_k) A_r per timeslice on the tensor cores (tcproj.cu):
// omode 1 writes out[t][k][r], omode 2 out[t][r][k]
dlma_status tc_block_product(dlma_ctx* ctx, int omode, const double2* a_src, size_t a_st, size_t a_sr, size_t a_sk,
                             int R, const double2* b_src, int b_conj, int N, int K, int T, double2* out);

// per-context event timer helper
struct EvTimer {
  cudaEvent_t a = nullptr, b = nullptr;
};

// Phase timer: events recorded on the context's stream at phase boundaries; the
// time between consecutive marks is charged to the phase opened by the earlier
// mark.  collect() (after a stream synchronisation) adds the elapsed times to
// acc[phase] and recycles the events.
struct PhaseTimer {
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, cudaEvent_t>> marks;
  double acc[kTimingSlots] = {0};
  int used = 0;
  explicit PhaseTimer(cudaStream_t s) : st(s) {}
  ~PhaseTimer() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
  void mark(int phase) {
    if (used == (int)pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      pool.push_back(e);
    }
    cudaEvent_t e = pool[used++];
    cudaEventRecord(e, st);
    marks.push_back({phase, e});
  }
  // open `phase` unless it is already the open one
  void enter(int phase) {
    if (!marks.empty() && marks.back().first == phase) return;
    mark(phase);
  }
  // the stream must have passed the last mark
  void collect() {
    for (size_t i = 0; i + 1 < marks.size(); i++) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, marks[i].second, marks[i + 1].second) == cudaSuccess && marks[i].first >= 0 &&
          marks[i].first < kTimingSlots)
        acc[marks[i].first] += ms;
    }
    if (!marks.empty()) {
      // keep the last mark open: its phase continues
      std::pair<int, cudaEvent_t> last = marks.back();
      marks.clear();
      for (int k = 0; k < used; k++)
        if (pool[k] == last.second) { std::swap(pool[k], pool[0]); break; }
      used = 1;
      marks.push_back(last);
    }
  }
};
