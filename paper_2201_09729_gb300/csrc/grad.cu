// Differentiation of the solves and of the pseudoscalar correlator.
//
// Adjoint solve (gamma_5-hermiticity of the Wilson-clover operator, Eq. 3 uses
// D^-1^dag):  y = D^-dag g = gamma_5 D^-1 gamma_5 g.
//
// For the scalar L = sum_t w(t) Re C_PS(t), C_PS = C_rest + 2 C_mixed + C_dist
// (Eq. 2 with Gamma = gamma_5, so g5 G = G g5 = 1):
//   C_dist(t)            = sum_{j dist} |V(t)^dag phi_j(t)|^2
//   C_rest + 2 C_mixed   = 1/N_r sum_r <phibar_r, (1 + Box(t)) phi_r>_t
// With gradients written as G(z) = dL/dRe z + i dL/dIm z (the convention of
// PyTorch), the adjoint sources of the checkpointed solutions are
//   G(phi_j)     = 2 w(t) Box(t) phi_j                       (distillation)
//   G(phi_r)     = w(t)/N_r (1 + Box(t)) phibar_r,   G(phibar_r) = w(t)/N_r (1 + Box(t)) phi_r,
// y_j = D^-dag G(phi_j), and since dD/dm0 = 1 and the sources are linear in eta:
//   dL/dm0  = - sum_j Re <y_j, phi_j>
//   dL/deta = [y_{phi_r} + (1 - Box(t')) y_{phibar_r}] restricted to t'.
#include "common.cuh"
#include <algorithm>

namespace {

// out = gamma_5 in for canonical spinors (chiral basis: spins 2, 3 change sign)
__global__ void k_gamma5(const double2* in, double2* out, size_t nsites) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nsites * 12) return;
  const int comp = e % 12;
  const double2 v = in[e];
  out[e] = comp >= 6 ? make_double2(-v.x, -v.y) : v;
}

// partial sums of Re sum conj(a) b
__global__ void k_real_dot(const double2* __restrict__ a, const double2* __restrict__ b, size_t n, double* part) {
  double s = 0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double2 x = a[e], y = b[e];
    s += x.x * y.x + x.y * y.y;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Box(t) psi_j from the coefficients: out[j][site][alpha][c] = sum_k v_k(m, c; t) coeff[j][t][alpha][k]
// (VT [Tsel][3 Vs][N]: V transposed; sites of the timeslices t0 .. t0 + Tsel - 1, stride_sites per j)
__global__ void k_backproject(const double2* __restrict__ VT, const double2* __restrict__ coeff, int N, int Vs,
                              int Tsel, int t0, int nj, size_t stride_sites, double2* out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)Tsel * Vs * 12;
  if (e >= per * nj) return;
  const int c = e % 3, a = (e / 3) % 4;
  const size_t site = (e / 12) % ((size_t)Tsel * Vs);
  const size_t j = e / per;
  const int t = site / Vs, m = site % Vs;
  const double2* vt = VT + (size_t)t * 3 * Vs * N + (size_t)(m * 3 + c) * N;
  const double2* co = coeff + (((size_t)j * Tsel + t) * 4 + a) * N;
  Cx<double> s = cx<double>(0, 0);
  for (int k = 0; k < N; k++) fma_acc(s, cx<double>(vt[k].x, vt[k].y), cx<double>(co[k].x, co[k].y));
  out[((size_t)j * stride_sites + (size_t)t0 * Vs + site) * 12 + a * 3 + c] = make_double2(s.re, s.im);
}

// adjoint sources G_j = w(t) (alpha_j sol_{p(j)} + beta_j box_{p(j)})
__global__ void k_adjoint_src(const double2* __restrict__ sol, const double2* __restrict__ box,
                              const double* __restrict__ w, const int* __restrict__ partner,
                              const double* __restrict__ ab, int nj, size_t V, int Vs, double2* G) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nj * V * 12) return;
  const size_t j = e / (V * 12);
  const size_t rest = e % (V * 12);
  const int t = (rest / 12) / Vs;
  const size_t src = (size_t)partner[j] * V * 12 + rest;
  const double f = w[t], al = ab[2 * j], be = ab[2 * j + 1];
  const double2 x = sol[src], bx = box[src];
  G[e] = make_double2(f * (al * x.x + be * bx.x), f * (al * x.y + be * bx.y));
}

// deta[r] = y_phi_r + y_phibar_r - box(y_phibar_r) on timeslice t'
__global__ void k_eta_grad(const double2* __restrict__ y, const double2* __restrict__ boxp, int nn, int N4, size_t V,
                           int Vs, int tsrc, double2* deta) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nn * Vs * 12) return;
  const size_t r = e / ((size_t)Vs * 12), rest = e % ((size_t)Vs * 12);
  const size_t off = (size_t)tsrc * Vs * 12 + rest;
  const double2 a = y[((size_t)N4 + 2 * r) * V * 12 + off];
  const double2 b = y[((size_t)N4 + 2 * r + 1) * V * 12 + off];
  const double2 c = boxp[r * (size_t)Vs * 12 + rest];
  deta[e] = make_double2(a.x + b.x - c.x, a.y + b.y - c.y);
}

}  // namespace

// internal: projection helpers of contract.cu
dlma_status contract_transpose_V(dlma_ctx* ctx, const double* V, int st_t, int st_k, int Tsel, int t0, int N,
                                 double2** VT, int slot);
dlma_status contract_project(dlma_ctx* ctx, const double2* VT, int N, int Tsel, const double* psi,
                             size_t stride_sites, int site_t0, int nrhs, double2* coeff);

static dlma_status gamma5_inplace(dlma_ctx* ctx, double* p, size_t nsites) {
  const size_t tot = nsites * 12;
  k_gamma5<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>((const double2*)p, (double2*)p, nsites);
  CHECK_LAUNCH();
  return DLMA_OK;
}

static dlma_status real_dot(dlma_ctx* ctx, const double* a, const double* b, size_t n, double* out) {
  double* part;
  TRY(workT(ctx, WS_T0, 1024, &part));
  k_real_dot<<<1024, 256, 0, ctx->stream>>>((const double2*)a, (const double2*)b, n, part);
  CHECK_LAUNCH();
  std::vector<double> h(1024);
  CU(cudaMemcpyAsync(h.data(), part, sizeof(double) * 1024, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  double s = 0;
  for (double v : h) s += v;
  *out = s;
  return DLMA_OK;
}

extern "C" dlma_status dlma_solve_adjoint(dlma_ctx* ctx, const double* g, double* y, int nrhs, double tol,
                                          dlma_prec inner, dlma_solve_info* info, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!ctx->have_gauge || !ctx->have_params) return set_err(ctx, DLMA_ERR_STATE, "gauge / params not set");
  if (!g || !y || nrhs < 1 || !(tol > 0) || inner < DLMA_FP64 || inner > DLMA_FP16S)
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_solve_adjoint");
  CU(cudaSetDevice(ctx->device));
  const size_t nsites = (size_t)nrhs * ctx->g.V;
  const size_t bytes = nsites * 12 * 16;
  double *dg, *dy;
  TRY(workT(ctx, WS_SRC, bytes / 8, &dg));
  CU(cudaMemcpyAsync(dg, g, bytes, mem == DLMA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                     ctx->stream));
  TRY(gamma5_inplace(ctx, dg, nsites));
  dy = y;
  if (mem == DLMA_MEM_HOST) TRY(workT(ctx, WS_SOL, bytes / 8, &dy));
  const dlma_status s = solve_fields(ctx, dg, dy, nrhs, tol, inner, info);
  if (s != DLMA_OK && s != DLMA_ERR_NOT_CONVERGED) return s;
  TRY(gamma5_inplace(ctx, dy, nsites));
  TRY(copy_out(ctx, y, dy, bytes, mem));
  CU(cudaStreamSynchronize(ctx->stream));
  return s;
}

extern "C" dlma_status dlma_real_dot(dlma_ctx* ctx, const double* a, const double* b, uint64_t n, double* out,
                                     dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!a || !b || !out) return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_real_dot");
  CU(cudaSetDevice(ctx->device));
  const double *da, *db;
  TRY(copy_in(ctx, WS_IN, a, n * 16, mem, &da));
  TRY(copy_in(ctx, WS_OUT, b, n * 16, mem, &db));
  return real_dot(ctx, da, db, n, out);
}

extern "C" dlma_status dlma_set_checkpoint(dlma_ctx* ctx, int on) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  ctx->checkpoint = on ? 1 : 0;
  if (!on) {
    if (ctx->ckpt) {
      cudaSetDevice(ctx->device);
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->ckpt);
    }
    ctx->ckpt = nullptr;
    ctx->ckpt_J = 0;
    ctx->ckpt_serial = 0;
  }
  return DLMA_OK;
}

extern "C" dlma_status dlma_correlators_backward(dlma_ctx* ctx, int t_src, int N, int n_noise, const double* w,
                                                 double tol, dlma_prec inner, double* dL_dm0, double* dL_deta,
                                                 dlma_solve_info* info, dlma_mem mem) {
  if (!ctx) return DLMA_ERR_INVALID_ARG;
  if (!w || !dL_dm0 || (n_noise && !dL_deta) || N < 1 || n_noise < 0 || t_src < 0 || t_src >= ctx->g.T ||
      !(tol > 0))
    return set_err(ctx, DLMA_ERR_INVALID_ARG, "bad argument to dlma_correlators_backward");
  if (!ctx->ckpt || ctx->ckpt_N != N || ctx->ckpt_nn != n_noise || ctx->ckpt_tsrc != t_src)
    return set_err(ctx, DLMA_ERR_STATE, "no checkpointed forward solutions for these arguments");
  if (ctx->eig_N != N) return set_err(ctx, DLMA_ERR_STATE, "no cached Laplacian modes for N = %d", N);
  // the adjoint solves use the current operator and modes: they must be the ones
  // the checkpointed forward ran with
  if (!ctx->have_params || ctx->m0 != ctx->ckpt_m0 || ctx->csw != ctx->ckpt_csw)
    return set_err(ctx, DLMA_ERR_STATE, "m0 / c_sw changed since the checkpointed forward (m0 %g -> %g, c_sw %g -> %g)",
                   ctx->ckpt_m0, ctx->m0, ctx->ckpt_csw, ctx->csw);
  if (ctx->gauge_gen != ctx->ckpt_gauge_gen)
    return set_err(ctx, DLMA_ERR_STATE, "the gauge field changed since the checkpointed forward");
  if (ctx->eig_gen != ctx->ckpt_eig_gen)
    return set_err(ctx, DLMA_ERR_STATE, "the Laplacian modes were recomputed since the checkpointed forward");
  CU(cudaSetDevice(ctx->device));
  const int T = ctx->g.T, Vs = ctx->g.Vs;
  const size_t V = ctx->g.V;
  const int J2 = 4 * N + 2 * n_noise;
  const size_t fb = V * 12 * 16;
  // modes, coefficients and Box of every checkpointed solution
  double2 *VT, *VTs, *coeff, *box, *G;
  TRY(contract_transpose_V(ctx, (const double*)ctx->eig_V, 1, T, T, 0, N, &VT, WS_PROJ_PART));
  TRY(contract_transpose_V(ctx, (const double*)ctx->eig_V, 1, T, 1, t_src, N, &VTs, WS_PROJ_V));
  TRY(workT(ctx, WS_PROJ_C, (size_t)J2 * T * 4 * N, &coeff));
  TRY(contract_project(ctx, VT, N, T, (const double*)ctx->ckpt, V, 0, J2, coeff));
  TRY(workT(ctx, WS_CON, (size_t)J2 * V * 12, &box));
  {
    const size_t tot = (size_t)J2 * T * Vs * 12;
    k_backproject<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(VT, coeff, N, Vs, T, 0, J2, V, box);
    CHECK_LAUNCH();
  }
  // adjoint sources
  std::vector<int> partner(J2);
  std::vector<double> ab(2 * J2);
  for (int j = 0; j < 4 * N; j++) { partner[j] = j; ab[2 * j] = 0.0; ab[2 * j + 1] = 2.0; }
  for (int r = 0; r < n_noise; r++) {
    const int jp = 4 * N + 2 * r, jb = jp + 1;
    partner[jp] = jb; ab[2 * jp] = ab[2 * jp + 1] = 1.0 / n_noise;
    partner[jb] = jp; ab[2 * jb] = ab[2 * jb + 1] = 1.0 / n_noise;
  }
  double* aux;
  TRY(workT(ctx, WS_T2, (size_t)T + 2 * J2 + J2 + 16, &aux));
  double* dw = aux;
  double* dab = aux + T;
  int* dpart = (int*)(aux + T + 2 * J2);
  const double* wdev = w;
  if (mem == DLMA_MEM_HOST) {
    CU(cudaMemcpyAsync(dw, w, sizeof(double) * T, cudaMemcpyHostToDevice, ctx->stream));
    wdev = dw;
  }
  CU(cudaMemcpyAsync(dab, ab.data(), sizeof(double) * 2 * J2, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemcpyAsync(dpart, partner.data(), sizeof(int) * J2, cudaMemcpyHostToDevice, ctx->stream));
  TRY(workT(ctx, WS_SRC, (size_t)J2 * V * 12, &G));
  {
    const size_t tot = (size_t)J2 * V * 12;
    k_adjoint_src<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>((const double2*)ctx->ckpt, box, wdev,
                                                                          dpart, dab, J2, V, Vs, G);
    CHECK_LAUNCH();
  }
  // adjoint solves y = g5 D^-1 g5 G (the solver reads G, writes y into the Box buffer)
  TRY(gamma5_inplace(ctx, (double*)G, (size_t)J2 * V));
  double* y = (double*)box;
  const dlma_status s = solve_fields(ctx, (const double*)G, y, J2, tol, inner, info);
  if (s != DLMA_OK && s != DLMA_ERR_NOT_CONVERGED) return s;
  TRY(gamma5_inplace(ctx, y, (size_t)J2 * V));
  // dL/dm0 = - sum_j Re <y_j, phi_j>
  double dot = 0;
  TRY(real_dot(ctx, y, (const double*)ctx->ckpt, (size_t)J2 * V * 12, &dot));
  *dL_dm0 = -dot;
  // dL/deta
  if (n_noise) {
    const size_t ebytes = (size_t)n_noise * Vs * 12 * 16;
    double2 *cy, *boxp, *deta;
    TRY(workT(ctx, WS_CON2, (size_t)n_noise * 4 * N, &cy));
    // coefficients of y_phibar_r on t' (rows 4N + 2r + 1: stride 2 V sites from row 4N + 1)
    TRY(contract_project(ctx, VTs, N, 1, y + ((size_t)4 * N + 1) * V * 24, 2 * V, t_src, n_noise, cy));
    TRY(workT(ctx, WS_ETA, (size_t)n_noise * Vs * 12 * 2, &boxp));
    {
      const size_t tot = (size_t)n_noise * Vs * 12;
      k_backproject<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(VTs, cy, N, Vs, 1, 0, n_noise, Vs, boxp);
      CHECK_LAUNCH();
    }
    deta = boxp + (size_t)n_noise * Vs * 12;
    if (mem == DLMA_MEM_DEVICE) deta = (double2*)dL_deta;
    {
      const size_t tot = (size_t)n_noise * Vs * 12;
      k_eta_grad<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>((const double2*)y, boxp, n_noise, 4 * N, V,
                                                                         Vs, t_src, deta);
      CHECK_LAUNCH();
    }
    if (mem == DLMA_MEM_HOST) TRY(copy_out(ctx, dL_deta, (const double*)deta, ebytes, mem));
  }
  CU(cudaStreamSynchronize(ctx->stream));
  (void)fb;
  return s;
}
