// Spatial covariant Laplacian of Eq. 1 and its low modes (placeholder for the
// eigensolver; the stencil is complete).
#include "common.cuh"

__global__ void k_lap(Geom g, const double2* __restrict__ U3, const double2* __restrict__ in, double2* out, int nvec,
                      size_t vstride) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (s >= g.V || j >= nvec) return;
  int x = s % g.L, y = (s / g.L) % g.L, z = (s / (g.L * g.L)) % g.L, t = s / g.Vs;
  Coord c{x, y, z, t};
  const double2* v = in + (size_t)j * vstride;
  Cx<double> acc[3];
  for (int a = 0; a < 3; a++) {
    double2 e = v[(size_t)s * 3 + a];
    acc[a] = cx<double>(-6.0 * e.x, -6.0 * e.y);
  }
  for (int k = 0; k < 3; k++) {
    int nf = nbr_lex(g, c, k + 1, +1), nb = nbr_lex(g, c, k + 1, -1);
    Cx<double> vf[3], vb[3];
    for (int a = 0; a < 3; a++) {
      double2 e = v[(size_t)nf * 3 + a];
      vf[a] = cx<double>(e.x, e.y);
      e = v[(size_t)nb * 3 + a];
      vb[a] = cx<double>(e.x, e.y);
    }
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double2 uf = U3[((size_t)k * 9 + a * 3 + b) * g.V + s];
        double2 ub = U3[((size_t)k * 9 + b * 3 + a) * g.V + nb];
        fma_acc(acc[a], cx<double>(uf.x, uf.y), vf[b]);
        fma_conj_acc(acc[a], cx<double>(ub.x, ub.y), vb[b]);
      }
  }
  double2* o = out + (size_t)j * vstride;
  for (int a = 0; a < 3; a++) o[(size_t)s * 3 + a] = make_double2(acc[a].re, acc[a].im);
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
  dim3 grid((ctx->g.V + 127) / 128, nvec);
  k_lap<<<grid, 128, 0, ctx->stream>>>(ctx->g, ctx->U3, (const double2*)din, (double2*)dout, nvec,
                                       (size_t)ctx->g.V * 3);
  CHECK_LAUNCH();
  TRY(copy_out(ctx, out, dout, bytes, mem));
  CU(cudaStreamSynchronize(ctx->stream));
  return DLMA_OK;
}

extern "C" dlma_status dlma_laplacian_eigs(dlma_ctx* ctx, int t, int N, double tol, double* evals, double* evecs,
                                           dlma_mem mem) {
  (void)t; (void)N; (void)tol; (void)evals; (void)evecs; (void)mem;
  return set_err(ctx, DLMA_ERR_STATE, "eigensolver not built yet");
}
