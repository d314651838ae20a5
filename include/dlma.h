/*
 * dlma.h -- C ABI of the GB300 (sm_103a) distillation low-mode-averaging
 * library (arXiv:2201.09729, "Implementing noise reduction techniques into
 * the OpenQ*D package").
 *
 * The calls follow the paper's statement of the problem:
 *   set the gauge field and the Wilson-clover parameters (Sec. 2, Table 1),
 *   compute the low modes of the spatial Laplacian per timeslice (Eq. 1,
 *   Sec. 2), apply / invert the Dirac operator on distillation and noise
 *   sources (Eq. 4 and the text after Eq. 3), project solutions on V(t)
 *   (Eq. 1, Eq. 3) and contract into C_rest, C_mixed and C_dist (Eqs. 2-3).
 *
 * Conventions (all calls):
 *   Complex numbers are interleaved (re, im) doubles.  Site index
 *   s = x + L (y + L (z + L t)), so every timeslice is a contiguous block of
 *   L^3 sites.  Spinors are [site][spin 4][colour 3] complex; links are
 *   [site][mu 4][row 3][col 3] complex with mu = 0 time and mu = 1, 2, 3 the
 *   x, y, z directions.  Colour vectors on a timeslice are [L^3][3] complex.
 *   Dirac matrices are in the chiral basis: gamma_5 = diag(1, 1, -1, -1),
 *   gamma_0 = -[[0, 1], [1, 0]], gamma_k = [[0, -i sigma_k], [i sigma_k, 0]].
 *
 *   Memory: every data pointer is host or device memory as the dlma_mem
 *   argument says; device pointers must belong to the context's device.  The
 *   caller owns every array it passes; the library owns the context, its
 *   copies of the gauge and clover fields, the cached Laplacian modes and all
 *   work space.  Calls are ordered on the context's stream and synchronous on
 *   return.  A context is not thread-safe.
 *
 *   Errors: every call returns a dlma_status; nothing is thrown across the
 *   ABI.  dlma_last_error() gives a one-line description of the last failure.
 *   On DLMA_ERR_NOT_CONVERGED the outputs hold the best iterate and the info
 *   records its true residual.
 */
#ifndef DLMA_H
#define DLMA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dlma_ctx dlma_ctx;

typedef enum {
  DLMA_OK = 0,
  DLMA_ERR_INVALID_ARG = 1,   /* bad size, pointer, precision or state of the input */
  DLMA_ERR_NOT_CONVERGED = 2, /* iteration cap reached before the tolerance */
  DLMA_ERR_NONFINITE = 3,     /* NaN / Inf met in the gauge field or in an iterate */
  DLMA_ERR_SINGULAR = 4,      /* a clover block could not be inverted */
  DLMA_ERR_OOM = 5,           /* device allocation failed or exceeds the memory cap */
  DLMA_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  DLMA_ERR_TIMEOUT = 7,       /* host-side wall-clock limit hit while waiting */
  DLMA_ERR_STATE = 8          /* call made before its prerequisites (gauge, params) */
} dlma_status;

typedef enum {
  DLMA_FP64 = 0,   /* double precision, 18-real links */
  DLMA_FP32 = 1,   /* single precision, 12-real links (third row rebuilt) */
  DLMA_FP16S = 2   /* half precision spinors with a per-site fp32 scale, 12-real fp16 links */
} dlma_prec;

typedef enum { DLMA_MEM_HOST = 0, DLMA_MEM_DEVICE = 1 } dlma_mem;

typedef enum {
  DLMA_SOLVER_CGNE = 0,      /* CG on the normal equations of the Schur system */
  DLMA_SOLVER_BICGSTAB = 1   /* BiCGStab on the Schur system (FP32 inner solves; default) */
} dlma_solver;

typedef struct {
  int L;      /* spatial extent (even, >= 2) */
  int T;      /* temporal extent (even, >= 2) */
  int bc_t;   /* 0 periodic, 1 antiperiodic quark fields in time */
} dlma_lattice;

typedef struct {
  int iters_inner;     /* inner (low-precision) Krylov iterations summed over restarts */
  int iters_outer;     /* FP64 reliable updates (residual replacements) */
  double true_resid;   /* ||b - D x||_2 / ||b||_2 in FP64: the even-odd Schur residual
                          |bhat - Dhat x_e| of the final FP64 update (the odd rows of
                          b - D x vanish by construction of x_o), or, for a solve stopped
                          before converging, b - D x evaluated on the full lattice */
  int converged;       /* 1 if true_resid <= tol */
} dlma_solve_info;

/* ---- context -------------------------------------------------------------
 * dlma_create: a context for an L^3 x T lattice on CUDA device `device`;
 * `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).
 * Allocates the index / gauge / clover storage for the lattice.
 * Errors: INVALID_ARG (odd or < 2 extents, device out of range), OOM, CUDA. */
dlma_status dlma_create(const dlma_lattice* lat, int device, void* cuda_stream, dlma_ctx** out);
dlma_status dlma_destroy(dlma_ctx* ctx);
const char* dlma_last_error(const dlma_ctx* ctx);
/* Free the context's work space (solver, eigensolver and contraction buffers
 * grow on demand and are kept between calls); the gauge and clover fields, the
 * cached modes and any checkpoint stay.  Errors: INVALID_ARG. */
dlma_status dlma_release_workspace(dlma_ctx* ctx);
/* Cap on the library's own device work space in bytes (0 = no cap); solves
 * that would exceed it run in smaller batches, or fail with OOM if one
 * right-hand side does not fit. */
dlma_status dlma_set_memory_cap(dlma_ctx* ctx, uint64_t bytes);

/* ---- gauge field and parameters ----------------------------------------
 * dlma_set_gauge: copy the links U_mu(x) (complex [V][4][3][3]) into the
 * context and derive the even-odd, 12-real (fp32 / fp16) and spatial-link
 * copies.  Links are expected in SU(3); the 12-real forms rebuild the third
 * row as the conjugated cross product of the first two.
 * Errors: INVALID_ARG (null), NONFINITE (a NaN / Inf link), CUDA. */
dlma_status dlma_set_gauge(dlma_ctx* ctx, const double* links, dlma_mem mem);

/* dlma_set_params: Wilson-clover parameters of the O(a)-improved Wilson
 * operator named in the abstract and Sec. 2 (m0-normalised form)
 *   D psi(x) = T(x) psi(x) - 1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x+mu)
 *                                       + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu)],
 *   T(x) = (4 + m0) + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} Fhat_{mu nu}(x),
 * Fhat = (Q_{mu nu} - Q_{nu mu}) / 8 from the four plaquette leaves; m0 =
 * 1/(2 kappa) - 4.  Builds the clover field and the inverse of its odd-site
 * blocks (2 hermitian 6x6 chirality blocks per site).
 * Errors: STATE (no gauge field), SINGULAR (a block not invertible), CUDA. */
dlma_status dlma_set_params(dlma_ctx* ctx, double m0, double c_sw);

/* ---- Dirac operator -------------------------------------------------------
 * dlma_apply_Dw: out = D in for nrhs full-lattice spinor fields
 * (complex [nrhs][V][4][3]), computed in precision `prec` (inputs and
 * outputs are always complex128; FP32 / FP16S round the fields on entry).
 * Errors: STATE, INVALID_ARG, OOM, CUDA. */
dlma_status dlma_apply_Dw(dlma_ctx* ctx, const double* in, double* out, int nrhs,
                          dlma_prec prec, dlma_mem mem);

/* dlma_apply_schur: the even-odd Schur operator on even-site fields
 * (complex [nrhs][V/2][4][3], even sites in lexicographic order):
 *   dagger = 0: out = Dhat in,  Dhat = T_ee - D_eo T_oo^-1 D_oe
 *   dagger = 1: out = Dhat^dag in = gamma_5 Dhat gamma_5 in.
 * Errors: STATE, INVALID_ARG, OOM, CUDA. */
dlma_status dlma_apply_schur(dlma_ctx* ctx, const double* in, double* out, int nrhs, int dagger,
                             dlma_prec prec, dlma_mem mem);

/* dlma_apply_schur_noalloc: the same operator as dlma_apply_schur with
 * dagger 0 / 1, in FP64, for callers that must not allocate device memory:
 * a framework that owns all device memory through its own pool and forbids
 * allocations it does not track, or a caller that cannot afford the
 * device-wide synchronisation cudaMalloc / cudaFree may cause.  The paper has
 * no counterpart; it is a library-usage variant.  `in` and `out` are DEVICE
 * pointers (complex [nrhs][V/2][4][3], even sites), owned by the caller.  The
 * work space is a fixed 64 MiB array in the library's device memory, held by
 * every GPU that has loaded it until the process exits; nothing else is
 * allocated.  The library's device code is loaded lazily (per device, on first
 * use), so the 64 MiB are reserved on a device by the first call there, which
 * also looks up the array's device address: make that first call before any
 * stream capture.  Three FP64 even-odd fields of nrhs right-hand sides must
 * fit in it (3 * 192 * nrhs * V/2 bytes <= 64 MiB), else DLMA_ERR_INVALID_ARG
 * with a message.  All calls share the one
 * array: calls that overlap on the GPU race on it.
 * Errors: STATE, INVALID_ARG, CUDA. */
dlma_status dlma_apply_schur_noalloc(dlma_ctx* ctx, const double* in, double* out, int nrhs, int dagger);

/* dlma_solve: x = D^-1 b for nrhs full-lattice sources (complex
 * [nrhs][V][4][3]); the propagator solves of Eq. 4 and of the perambulator
 * (text after Eq. 3).  Even-odd Schur system, multi-RHS CG on the normal
 * equations (or BiCGStab on the Schur system for FP32 inner solves, see
 * dlma_set_solver); `inner` = DLMA_FP64 runs it in double precision, DLMA_FP32 /
 * DLMA_FP16S run the Krylov iteration in that precision (FP16: storage, FP32
 * arithmetic) with FP64 reliable updates: when a right-hand side's iterated
 * residual has dropped by a fixed factor since its last update, its solution
 * is folded into FP64 and its residual recomputed in FP64 (for BiCGStab's
 * last update see dlma_set_solver).  Each right-hand side stops when its
 * FP64 true residual ||b - D x|| / ||b|| <= tol and is retired from the batch.  `info` (may be
 * NULL) receives nrhs records.  A zero source gives x = 0.
 * Errors: STATE, INVALID_ARG (tol <= 0, nrhs < 1), NOT_CONVERGED, NONFINITE,
 * OOM, CUDA. */
dlma_status dlma_solve(dlma_ctx* ctx, const double* b, double* x, int nrhs, double tol,
                       dlma_prec inner, dlma_solve_info* info, dlma_mem mem);

/* dlma_set_solver: Krylov method of the inner solves with inner = DLMA_FP32
 * (the FP64 and FP16S inner solves always run CGNE).  DLMA_SOLVER_BICGSTAB
 * (the default) iterates BiCGStab on the Schur system Dhat x_e = bhat with
 * FP32 vectors and the same FP64 reliable updates (residual replacement when
 * |r| has dropped by 3e-4 since the last update, DLMA_BICG_DELTA in the
 * environment overriding the factor; restart of the shadow residual after a
 * breakdown or a stagnating update).  The iteration aims at tol / 2; once a
 * right-hand side's FP64 residual is below 1e-3 (tol / 2) / 1.2e-7 times |b|,
 * its next update subtracts the FP32 operator's image of the FP32 solution
 * increment from that residual instead of applying the FP64 operator: the
 * FP32 rounding of the small product stays below 1e-3 (tol / 2) |b|.  Two operator
 * applications per iteration and about half as many as CGNE needs on these
 * systems.  Right-hand sides it leaves above the tolerance are solved again
 * with CGNE in the same call; their info sums both iteration counts.
 * DLMA_SOLVER_CGNE selects CGNE throughout.  Errors: INVALID_ARG. */
dlma_status dlma_set_solver(dlma_ctx* ctx, dlma_solver solver);

/* dlma_solve_adjoint: y = D^-dag g for nrhs full-lattice fields, computed as
 * gamma_5 D^-1 gamma_5 g (gamma_5-hermiticity; the D^-1^dag of Eq. 3) with the
 * solver of dlma_solve (same arguments and errors).  The backward pass of a
 * differentiable solve: for x = D^-1 b, grad_b = D^-dag grad_x and, since
 * dD/dm0 = 1, dL/dm0 = -Re <D^-dag grad_x, x>. */
dlma_status dlma_solve_adjoint(dlma_ctx* ctx, const double* g, double* y, int nrhs, double tol,
                               dlma_prec inner, dlma_solve_info* info, dlma_mem mem);

/* dlma_real_dot: *out = Re sum_i conj(a_i) b_i over n complex numbers (a, b
 * in `mem`; out HOST).  Errors: INVALID_ARG, CUDA. */
dlma_status dlma_real_dot(dlma_ctx* ctx, const double* a, const double* b, uint64_t n, double* out,
                          dlma_mem mem);

/* ---- spatial Laplacian (Eq. 1) --------------------------------------------
 * dlma_apply_laplacian: out = lap(t) in on every timeslice at once for nvec
 * colour fields over the whole lattice (complex [nvec][V][3]):
 *   (lap v)(m, t) = -6 v + sum_j [U_j(m,t) v(m+j) + U_j(m-j,t)^dag v(m-j)].
 * Errors: STATE, INVALID_ARG, CUDA. */
dlma_status dlma_apply_laplacian(dlma_ctx* ctx, const double* in, double* out, int nvec, dlma_mem mem);

/* dlma_laplacian_eigs: the N lowest eigenpairs of -lap(t) (Eq. 1; "low-lying
 * modes", Sec. 2), for one timeslice t or for all timeslices at once
 * (t = -1).  Eigenvalues (of -lap, ascending, in [0, 12]) go to evals
 * ([N], or [T][N] for t = -1; always HOST memory); eigenvectors, normalised,
 * go to evecs (complex [N][L^3][3], or [T][N][L^3][3]) in `mem`; evecs may be
 * NULL.  The modes of every computed timeslice are also cached in the
 * context.  Each pair meets ||lap v - lam v|| <= tol * max(|lam|, 1).  The
 * iteration keeps N + min(max(N, 16), 64) vectors per timeslice, at most 510.
 * An iteration that stops improving before tol returns NOT_CONVERGED with
 * the residual reached.
 * Errors: STATE, INVALID_ARG (N < 1, N > 3 L^3 / 2, or the block above 510
 * vectors or 2^31 entries), NOT_CONVERGED, CUDA. */
dlma_status dlma_laplacian_eigs(dlma_ctx* ctx, int t, int N, double tol, double* evals,
                                double* evecs, dlma_mem mem);

/* ---- distillation sources, projections, contractions ------------------------
 * dlma_make_sources: the 4N + 5 n_noise sources of one source timeslice
 * t_src (complex [4N + 5 n_noise][V][4][3], zero off t_src), from the
 * modes V (complex [N][L^3][3] of t_src) and the noise eta (complex
 * [n_noise][L^3][4][3]):
 *   source 4k + alpha            = v_k (x) e_alpha                 (perambulator)
 *   source 4N + 5r + 0           = eta_r                           (Eq. 4, phi)
 *   source 4N + 5r + 1           = (1 - Box(t')) eta_r             (Eq. 4, phibar)
 *   source 4N + 5r + 1 + k       = gamma_5 gamma_k (1 - Box(t')) eta_r, k = 1..3
 * (the last three give the vector-channel left vectors of the one-end
 * estimator with an undiluted noise).  Errors: INVALID_ARG, CUDA. */
dlma_status dlma_make_sources(dlma_ctx* ctx, int t_src, int N, const double* V, int n_noise,
                              const double* eta, double* b, dlma_mem mem);

/* dlma_project: coefficients c = V(t)^dag psi(t) per spin (Eq. 1, Eq. 3),
 * for one timeslice t or every timeslice (t = -1):
 *   coeff[j][t][alpha][k] = sum_{m, c} conj(V_t[k][m][c]) psi_j(m, t, alpha, c)
 * V is complex [N][L^3][3] (t >= 0) or [T][N][L^3][3] (t = -1); psi complex
 * [nrhs][V][4][3]; coeff complex [nrhs][T or 1][4][N].
 * Errors: INVALID_ARG, CUDA. */
dlma_status dlma_project(dlma_ctx* ctx, int t, const double* V, int N, const double* psi, int nrhs,
                         double* coeff, dlma_mem mem);

/* dlma_contract: the correlator parts of Eqs. 2-3 for one source timeslice,
 * from the solutions of dlma_make_sources' sources (phi complex
 * [4N + 5 n_noise][V][4][3], in that order) and the modes of every timeslice
 * (V complex [T][N][L^3][3]).  For the four channels G in (gamma_5, gamma_1,
 * gamma_2, gamma_3), with sink and source Gamma equal:
 *   C_dist(t)      = tr[g5 G tau(t) G g5 tau(t)^dag],  tau = V(t)^dag D^-1 V(t')
 *   C_mixed(t)     = 1/N_r sum_r sum_{x in t} chi_r^dag g5 G Box(t) phi_r
 *   C_rest(t)      = 1/N_r sum_r sum_{x in t} chi_r^dag g5 G (1 - Box(t)) phi_r
 *   C_mixed_src(t) = tr[g5 G (1 - Box(t)) S G g5 Box(t') S^dag], S = D^-1(t, t'):
 *                    the other mixed term of Eq. 2 (Box at the source, 1 - Box
 *                    at the sink), exact and noise-free from the distillation
 *                    solutions phi^(k,b):  sum_{k,b,b'} (G g5)_{b'b}
 *                    <phi^(k,b), g5 G phi^(k,b')>_t - C_dist(t)
 *   C_full(t)      = C_rest + 2 C_mixed + C_dist, the total of Eq. 2 (the two
 *                    mixed terms merged by time reversal as the paper does;
 *                    C_mixed - C_mixed_src measures what that merge neglects
 *                    on one configuration)
 * chi_r = phibar_r (G = g5) or the gamma_5 gamma_k solution (G = g_k).
 * Outputs are complex [4][T] (channel-major), always HOST memory; C_mixed_src
 * and C_full may be NULL.  Errors: INVALID_ARG, CUDA. */
dlma_status dlma_contract(dlma_ctx* ctx, int t_src, int N, const double* V, int n_noise,
                          const double* phi, double* C_dist, double* C_rest, double* C_mixed,
                          double* C_mixed_src, double* C_full, dlma_mem mem);

/* dlma_correlators: the whole per-source-timeslice pipeline on the device --
 * sources, solves (precision `inner`, tolerance tol, in batches that fit the
 * memory cap), projections and contractions -- using the modes cached by
 * dlma_laplacian_eigs(t = -1, N).  eta complex [n_noise][L^3][4][3] in
 * `mem`; outputs complex [4][T] HOST as in dlma_contract (C_mixed_src and
 * C_full may be NULL); info (may be NULL) gets 4N + 5 n_noise records.
 * Errors: STATE (no cached modes for N), plus those of dlma_solve. */
dlma_status dlma_correlators(dlma_ctx* ctx, int t_src, int N, int n_noise, const double* eta,
                             double tol, dlma_prec inner, double* C_dist, double* C_rest,
                             double* C_mixed, double* C_mixed_src, double* C_full,
                             dlma_solve_info* info, dlma_mem mem);

/* dlma_correlators_diluted: the same pipeline with the noise treatment of the
 * paper's measurements (Sec. 3: six colour and even-odd diluted wall sources
 * per noise vector, solved for each of the four source spins -- the 24 wall
 * sources of Fig. 1).  eta complex [n_noise][L^3][3] in `mem`: one Z2 x Z2
 * number per site and colour of t_src, no spin index.  Piece d = 2 c + p keeps
 * colour c on the sites of t_src with (x + y + z + t_src) mod 2 = p; every
 * piece eta_d is solved as eta_d (x) e_beta and (1 - Box(t_src)) eta_d (x) e_beta
 * (48 solves per noise vector), and with B = G g5 on the source spin
 *   C_P(t) = 1/N_r sum_{r,d} sum_{beta,beta'} B[beta][beta'] sum_{x in t}
 *            phibar_{d,beta'}^dag g5 G P_t phi_{d,beta},
 * P_t = 1 - Box(t) (C_rest) or Box(t) (C_mixed): Eq. 3 with eta eta^dag
 * replaced by sum_d eta_d eta_d^dag.  C_dist, C_mixed_src and C_full as in
 * dlma_contract.  Outputs complex [4][T] HOST (channels PS, V1, V2, V3; the
 * last two may be NULL); info (may be NULL) gets 4N + 48 n_noise records: the
 * 4N distillation solves, then for noise r, piece d, the rows
 * 4N + 48 r + 8 d + beta (phi) and + 4 + beta (phibar).  Solves run in batches
 * of whole noise vectors within the memory cap.  Errors: STATE (no cached
 * modes for N), INVALID_ARG (n_noise < 1), plus those of dlma_solve. */
dlma_status dlma_correlators_diluted(dlma_ctx* ctx, int t_src, int N, int n_noise, const double* eta,
                                     double tol, dlma_prec inner, double* C_dist, double* C_rest,
                                     double* C_mixed, double* C_mixed_src, double* C_full,
                                     dlma_solve_info* info, dlma_mem mem);

/* dlma_correlators_plain: the plain one-end stochastic estimator of the same
 * correlator without distillation (no Box anywhere): the comparison the
 * paper draws in Fig. 1.  diluted = 0: eta complex [n_noise][L^3][4][3]
 * (undiluted Z2 x Z2 noise on t_src), 4 solves per noise vector, phi_r =
 * D^-1 eta_r and chi_{r,k} = D^-1 g5 g_k eta_r, and
 *   C(t) = 1/N_r sum_r sum_{x in t} chi_r^dag g5 G phi_r   (chi_r = phi_r for G = g5);
 * info rows 4 r + q (q = 0: phi_r, q = k: chi_{r,k}).  diluted = 1: eta
 * complex [n_noise][L^3][3] diluted as in dlma_correlators_diluted, 24 solves
 * per noise vector (rows 24 r + 4 d + beta: phi_{d,beta}) and
 *   C(t) = 1/N_r sum_{r,d} sum_{beta,beta'} (G g5)[beta][beta'] sum_{x in t}
 *          phi_{d,beta'}^dag g5 G phi_{d,beta}.
 * Needs no Laplacian modes.  C complex [4][T] HOST (channels PS, V1, V2, V3).
 * Errors: STATE (no gauge / params), INVALID_ARG, plus those of dlma_solve. */
dlma_status dlma_correlators_plain(dlma_ctx* ctx, int t_src, int n_noise, const double* eta, int diluted,
                                   double tol, dlma_prec inner, double* C, dlma_solve_info* info,
                                   dlma_mem mem);

/* ---- conventional low-mode averaging with Dirac low modes (the control) ----
 * Sec. 1 and the remark after Eq. 2: were Box built from eigenmodes of the
 * Dirac operator, Box and the propagator would commute and C_mixed would
 * vanish.  dlma_dirac_eigs: the N eigenpairs of the hermitian even-odd
 * operator Qhat = g5 Dhat (even sites, Dhat the Schur complement of
 * dlma_apply_schur) with the smallest |lambda|, in that order, found by
 * Chebyshev-filtered subspace iteration on Qhat^2 = Dhat^dag Dhat in FP64 and a
 * Rayleigh-Ritz of Qhat in the converged span.  evals [N] HOST (signed
 * lambda); evecs complex [N][V/2][4][3] (even sites, lexicographic) in `mem`,
 * may be NULL.  The modes are cached in the context until the gauge field or
 * the parameters change.  Each pair meets ||Qhat u - lambda u|| <= tol
 * max(1, |lambda|).  Errors: STATE, INVALID_ARG (N < 1, block N + max(8, N)
 * above 510 or V/2 * 6), NOT_CONVERGED, CUDA. */
dlma_status dlma_dirac_eigs(dlma_ctx* ctx, int N, double tol, double* evals, double* evecs, dlma_mem mem);

/* dlma_dirac_project: out = P in (conj_g5 = 0) or g5 P g5 in (conj_g5 = 1) for
 * even-site fields (complex [nrhs][V/2][4][3]), P = sum_i u_i u_i^dag over the
 * cached Dirac low modes.  Since the even-even block of D^-1 is Dhat^-1 =
 * Qhat^-1 g5, P Dhat^-1 (1 - g5 P g5) = 0: the mixed term of Eq. 2 with these
 * modes vanishes.  Errors: STATE (no cached modes), INVALID_ARG, CUDA. */
dlma_status dlma_dirac_project(dlma_ctx* ctx, const double* in, double* out, int nrhs, int conj_g5, dlma_mem mem);

/* dlma_set_checkpoint: on != 0 makes dlma_correlators keep its forward
 * solutions (the 4N distillation solutions and phi_r, phibar_r of every noise
 * vector; the Krylov iterates are never kept) for dlma_correlators_backward;
 * on = 0 releases them.  The checkpoint holds (4N + 2 n_noise) V 192 bytes of
 * device memory from the first checkpointed forward until it is released;
 * while on, every dlma_correlators call also pays the device-to-device copies
 * into it.  Each checkpointed forward overwrites the previous checkpoint and
 * gets a new serial number (dlma_checkpoint_serial). */
dlma_status dlma_set_checkpoint(dlma_ctx* ctx, int on);

/* dlma_checkpoint_serial: serial number of the checkpoint currently held
 * (1, 2, ... per checkpointed dlma_correlators call), 0 if none.  A caller
 * that ran several forwards before their backwards compares it with the
 * serial seen after its own forward and re-runs that forward if another one
 * has replaced the checkpoint. */
uint64_t dlma_checkpoint_serial(const dlma_ctx* ctx);

/* dlma_correlators_backward: gradients of L = sum_t w(t) Re C_PS(t), C_PS the
 * pseudoscalar total C_rest + 2 C_mixed + C_dist of the last checkpointed
 * dlma_correlators call with the same (t_src, N, n_noise): dL/dm0 (one real,
 * HOST) and dL/deta (complex [n_noise][L^3][4][3] in `mem`, written as
 * dL/dRe + i dL/dIm).  w is real [T] in `mem`.  It runs 4N + 2 n_noise adjoint
 * solves y_j = D^-dag G_j of the adjoint sources G(phi_j) = 2 w Box phi_j
 * (distillation), G(phi_r) = w/N_r (1 + Box) phibar_r, G(phibar_r) =
 * w/N_r (1 + Box) phi_r; then dL/dm0 = -sum_j Re <y_j, phi_j> and
 * dL/deta_r = y_{phi_r} + (1 - Box(t')) y_{phibar_r} on t'.  info (may be NULL)
 * gets 4N + 2 n_noise records.  The gradients belong to the state the
 * checkpointed forward ran under: if m0, c_sw, the gauge field or the cached
 * modes changed since, the call fails with STATE instead of differentiating
 * the wrong operator.  Errors: STATE (no checkpoint / modes, or state changed
 * since the checkpoint), INVALID_ARG, plus those of dlma_solve. */
dlma_status dlma_correlators_backward(dlma_ctx* ctx, int t_src, int N, int n_noise, const double* w,
                                      double tol, dlma_prec inner, double* dL_dm0, double* dL_deta,
                                      dlma_solve_info* info, dlma_mem mem);

/* ---- introspection ---------------------------------------------------------
 * dlma_index_tables: the device's even-odd index arithmetic written out:
 * eo_index[V] (compressed index of every site within its parity) and
 * nbr[2][8][V/2] (for output parity p, direction d = 2 mu + (0 fwd, 1 bwd),
 * the compressed index of the neighbour in parity 1 - p).  HOST memory.
 * Errors: INVALID_ARG, CUDA. */
dlma_status dlma_index_tables(dlma_ctx* ctx, int32_t* eo_index, int32_t* nbr);

/* dlma_kernel_launches: number of kernels the library launched on this
 * context since creation (graph-replayed kernels included). */
uint64_t dlma_kernel_launches(const dlma_ctx* ctx);

/* dlma_last_timing: figures of the last timed call, measured with CUDA
 * events on the context's stream (milliseconds unless stated); out[0 .. n-1]
 * receives slots 0 .. n-1 (slots past 7 are 0).  Slot 0 is the device time of
 * the whole call for every call below; the others depend on the call:
 *   dlma_apply_schur          1 the two stencil launches, 2 their number (2)
 *   dlma_solve, _adjoint      -
 *   dlma_dirac_eigs           1 subspace iterations
 *   dlma_laplacian_eigs       1 FP32 filter iterations, 2 FP64 iterations,
 *                             3 Laplacian applications (the matvec of Table 2),
 *                             4 orthogonalisation: Gram matrices, small
 *                               eigenproblems, rotations, residuals,
 *                             5 host steps and transfers
 *   dlma_correlators, _diluted, _plain
 *                             1 source construction, 2 solves, 3 projections,
 *                             4 contractions
 * Errors: INVALID_ARG. */
dlma_status dlma_last_timing(const dlma_ctx* ctx, double* out, int n);

#ifdef __cplusplus
}
#endif
#endif /* DLMA_H */
