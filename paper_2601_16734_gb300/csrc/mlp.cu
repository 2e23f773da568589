// Learned local preconditioner for the PCG solve (placeholder until the
// network kernels land): every entry point reports SEEMPS_ERR_UNSUPPORTED.
#include "contract.cuh"

seemps_status mlp_precond_prepare(seemps_ctx* ctx, const seemps_mlp* mlp, const seemps_pair_dims* dm,
                                  const double* L, const double* W1, const double* W2,
                                  const double* R, const double* diag, void** state) {
  (void)mlp; (void)dm; (void)L; (void)W1; (void)W2; (void)R; (void)diag; (void)state;
  seemps_set_error(ctx, "MLP preconditioner not available in this build");
  return SEEMPS_ERR_UNSUPPORTED;
}

seemps_status mlp_precond_apply(seemps_ctx* ctx, void* state, const double* r, double* z,
                                const int* skip) {
  (void)state; (void)r; (void)z; (void)skip;
  seemps_set_error(ctx, "MLP preconditioner not available in this build");
  return SEEMPS_ERR_UNSUPPORTED;
}
