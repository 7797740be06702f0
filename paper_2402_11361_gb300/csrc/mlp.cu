// Learned preconditioner correction (kind 2): placeholder until a network is loaded.
#include "internal.cuh"

int mlp_apply(mehdg_ctx* ctx, const double* r, double* z) {
  (void)r;
  (void)z;
  if (!ctx->mlp) return ctx_fail(ctx, MEHDG_ERR_ARG, "preconditioner kind 2 needs a loaded MLP");
  return MEHDG_OK;
}
