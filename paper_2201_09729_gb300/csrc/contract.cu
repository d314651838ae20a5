// Distillation sources, projections and contractions (placeholders).
#include "common.cuh"

extern "C" dlma_status dlma_make_sources(dlma_ctx* ctx, int t_src, int N, const double* V, int n_noise,
                                         const double* eta, double* b, dlma_mem mem) {
  (void)t_src; (void)N; (void)V; (void)n_noise; (void)eta; (void)b; (void)mem;
  return set_err(ctx, DLMA_ERR_STATE, "not built yet");
}
extern "C" dlma_status dlma_project(dlma_ctx* ctx, int t, const double* V, int N, const double* psi, int nrhs,
                                    double* coeff, dlma_mem mem) {
  (void)t; (void)V; (void)N; (void)psi; (void)nrhs; (void)coeff; (void)mem;
  return set_err(ctx, DLMA_ERR_STATE, "not built yet");
}
extern "C" dlma_status dlma_contract(dlma_ctx* ctx, int t_src, int N, const double* V, int n_noise,
                                     const double* phi, double* C_dist, double* C_rest, double* C_mixed,
                                     dlma_mem mem) {
  (void)t_src; (void)N; (void)V; (void)n_noise; (void)phi; (void)C_dist; (void)C_rest; (void)C_mixed; (void)mem;
  return set_err(ctx, DLMA_ERR_STATE, "not built yet");
}
extern "C" dlma_status dlma_correlators(dlma_ctx* ctx, int t_src, int N, int n_noise, const double* eta, double tol,
                                        dlma_prec inner, double* C_dist, double* C_rest, double* C_mixed,
                                        dlma_solve_info* info, dlma_mem mem) {
  (void)t_src; (void)N; (void)n_noise; (void)eta; (void)tol; (void)inner; (void)C_dist; (void)C_rest; (void)C_mixed;
  (void)info; (void)mem;
  return set_err(ctx, DLMA_ERR_STATE, "not built yet");
}
