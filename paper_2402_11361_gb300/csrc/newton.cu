// a11-a12: nonlinear solves on the device-resident state.
//
// Steady (stage 0): pseudo-transient continuation (Sec. 3.1).  The pseudo-time
// term adds (1/dtau)(I (x) M) to A_uu only, so it vanishes from the residual at the
// linearisation point.  SER step update (eq. C31222, read with the ratio of
// successive |R_U| as in Mulder and van Leer): dtau <- min(max(dtau |R_U^m| /
// |R_U^{m+1}|, tau_init), tau_max).  Stop when |R_F| <= max(rtol |R_F^0|, atol).
// DIRK (stages 1..3, eq. C242): Alexander's 3-stage L-stable, stiffly accurate
// scheme; stage i solves the residual with time term d_ii/dt u + hist,
// hist = -d_ii/dt u^n + sum_{j<i} d_ij (u^{n,j} - u^n)/dt (d = a^-1), by Newton.
// Each Newton step: assemble -> condense + factor -> FGMRES -> recover -> update.
#include <chrono>
#include <cmath>

#include "internal.cuh"

namespace {

struct Dirk3 {
  double a[3][3], dinv[3][3];
  Dirk3() {
    // alpha: root of x^3 - 3x^2 + 3x/2 - 1/6 in (1/6, 1/2), by bisection
    double lo = 1.0 / 6.0, hi = 0.5;
    auto f = [](double x) { return x * x * x - 3 * x * x + 1.5 * x - 1.0 / 6.0; };
    for (int i = 0; i < 200; ++i) {
      double mid = 0.5 * (lo + hi);
      if ((f(lo) < 0) == (f(mid) < 0)) lo = mid; else hi = mid;
    }
    double al = 0.5 * (lo + hi);
    double b1 = -(6 * al * al - 16 * al + 1) / 4.0, b2 = (6 * al * al - 20 * al + 5) / 4.0;
    double A[3][3] = {{al, 0, 0}, {(1 - al) / 2, al, 0}, {b1, b2, al}};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) { a[i][j] = A[i][j]; dinv[i][j] = 0.0; }
    // inverse of the lower-triangular A by forward substitution
    for (int c = 0; c < 3; ++c)
      for (int i = 0; i < 3; ++i) {
        double s = (i == c) ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) s -= a[i][k] * dinv[k][c];
        dinv[i][c] = s / a[i][i];
      }
  }
};

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int newton_step(mehdg_ctx* ctx, double shift, double* u, double* q, double* uh, mehdg_solve_stats* st) {
  int rc;
  double t0 = now();
  if ((rc = condense_all(ctx, shift, ctx->bhat))) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  double t1 = now();
  rc = linear_solve_impl(ctx, ctx->bhat, ctx->duh, st);
  if (rc && rc != MEHDG_ERR_NOT_CONVERGED) return rc;
  double t2 = now();
  if ((rc = recover_impl(ctx, ctx->duh, ctx->du, ctx->dq))) return rc;
  const long long nu = (long long)ctx->E * ctx->Nu;
  if ((rc = vec_axpy(ctx, nu, 1.0, ctx->du, u))) return rc;
  if ((rc = vec_axpy(ctx, nu * ctx->d, 1.0, ctx->dq, q))) return rc;
  if ((rc = vec_axpy(ctx, ctx->ntr, 1.0, ctx->duh, uh))) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  phase_harvest(ctx);
  double t3 = now();
  if (st) {
    st->t_condense += t1 - t0;
    st->t_krylov += t2 - t1;
    st->t_recover += t3 - t2;
  }
  return MEHDG_OK;
}

bool stage_converged(const mehdg_ctx* ctx) {
  return ctx->stage_norms[3] <= std::max(ctx->opt.newton_rtol * ctx->stage_R0, ctx->opt.newton_atol);
}

}  // namespace

extern "C" int mehdg_stage_begin(mehdg_ctx* ctx, int stage, double dt, double* u, double* q, double* uh,
                                 mehdg_solve_stats* st) {
  if (!ctx || !u || !q || !uh || stage < 0 || stage > 3) return MEHDG_ERR_ARG;
  if (stage > 0 && !(dt > 0.0)) return MEHDG_ERR_ARG;
  mehdg_solve_stats local{};
  if (!st) st = &local;
  *st = mehdg_solve_stats{};
  const long long nu = (long long)ctx->E * ctx->Nu;
  int rc;
  ctx->stage_tt = mehdg_time_term{0.0, nullptr, 0};
  if (stage > 0) {
    static const Dirk3 dk;
    const int i = stage - 1;
    if (stage == 1) {
      if ((rc = vec_copy(ctx, nu, u, ctx->un))) return rc;
    }
    const double coef = dk.dinv[i][i] / dt;
    // hist = -coef u^n + sum_{j<i} dinv[i][j] (u^{n,j} - u^n) / dt
    double cn = -coef;
    for (int j = 0; j < i; ++j) cn -= dk.dinv[i][j] / dt;
    if ((rc = vec_lincomb(ctx, nu, cn, ctx->un, 0.0, ctx->un, ctx->hist))) return rc;
    for (int j = 0; j < i; ++j)
      if ((rc = vec_axpy(ctx, nu, dk.dinv[i][j] / dt, ctx->ustage + (size_t)j * nu, ctx->hist))) return rc;
    ctx->stage_tt = mehdg_time_term{coef, ctx->hist, 1};
  }
  ctx->cur_stage = -1;
  double t0 = now();
  if ((rc = assemble_all(ctx, u, q, uh, stage > 0 ? &ctx->stage_tt : nullptr, ctx->stage_norms))) return rc;
  st->t_assemble += now() - t0;
  if (!std::isfinite(ctx->stage_norms[3])) return ctx_fail(ctx, MEHDG_ERR_NAN, "non-finite residual");
  ctx->cur_stage = stage;
  ctx->stage_dt = dt;
  ctx->stage_R0 = ctx->stage_norms[3];
  ctx->stage_dtau = ctx->opt.tau_init;
  ctx->stage_newton = 0;
  st->res0 = st->res = ctx->stage_R0;
  st->status = stage_converged(ctx) ? 2 : 0;
  return MEHDG_OK;
}

extern "C" int mehdg_newton_step(mehdg_ctx* ctx, double* u, double* q, double* uh, mehdg_solve_stats* st) {
  if (!ctx || !u || !q || !uh) return MEHDG_ERR_ARG;
  if (ctx->cur_stage < 0) return ctx_fail(ctx, MEHDG_ERR_ARG, "mehdg_newton_step before mehdg_stage_begin");
  mehdg_solve_stats local{};
  if (!st) st = &local;
  *st = mehdg_solve_stats{};
  const int stage = ctx->cur_stage;
  st->res0 = ctx->stage_norms[3];
  const double shift = (stage == 0) ? 1.0 / ctx->stage_dtau : 0.0;
  int rc = newton_step(ctx, shift, u, q, uh, st);
  if (rc) return rc;
  const double RU_old = ctx->stage_norms[1];
  double t0 = now();
  if ((rc = assemble_all(ctx, u, q, uh, stage > 0 ? &ctx->stage_tt : nullptr, ctx->stage_norms))) return rc;
  st->t_assemble += now() - t0;
  ++ctx->stage_newton;
  st->newton_steps = 1;
  st->res = ctx->stage_norms[3];
  if (!std::isfinite(st->res)) return ctx_fail(ctx, MEHDG_ERR_NAN, "non-finite residual");
  if (stage == 0)
    ctx->stage_dtau = std::min(std::max(ctx->stage_dtau * RU_old / std::max(ctx->stage_norms[1], 1e-300),
                                        ctx->opt.tau_init), ctx->opt.tau_max);
  st->status |= stage_converged(ctx) ? 2 : 0;
  return MEHDG_OK;
}

extern "C" int mehdg_stage_end(mehdg_ctx* ctx, const double* u) {
  if (!ctx || !u) return MEHDG_ERR_ARG;
  if (ctx->cur_stage < 0) return ctx_fail(ctx, MEHDG_ERR_ARG, "mehdg_stage_end before mehdg_stage_begin");
  const int stage = ctx->cur_stage;
  int rc;
  if (stage > 0) {
    const long long nu = (long long)ctx->E * ctx->Nu;
    if ((rc = vec_copy(ctx, nu, u, ctx->ustage + (size_t)(stage - 1) * nu))) return rc;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->cur_stage = -1;
  return MEHDG_OK;
}

extern "C" int mehdg_dirk_stage(mehdg_ctx* ctx, int stage, double dt, double* u, double* q, double* uh,
                                mehdg_solve_stats* st) {
  if (!ctx || !u || !q || !uh || stage < 0 || stage > 3) return MEHDG_ERR_ARG;
  if (stage > 0 && !(dt > 0.0)) return MEHDG_ERR_ARG;
  mehdg_solve_stats local{}, one{};
  if (!st) st = &local;
  *st = mehdg_solve_stats{};
  int rc = mehdg_stage_begin(ctx, stage, dt, u, q, uh, &one);
  if (rc) return rc;
  st->res0 = one.res0;
  st->t_assemble += one.t_assemble;
  int steps = 0;
  while (!stage_converged(ctx) && steps < ctx->opt.max_newton) {
    rc = mehdg_newton_step(ctx, u, q, uh, &one);
    if (rc) return rc;
    st->fgmres_iters += one.fgmres_iters;
    st->t_assemble += one.t_assemble;
    st->t_condense += one.t_condense;
    st->t_krylov += one.t_krylov;
    st->t_recover += one.t_recover;
    st->status |= one.status & 1;
    ++steps;
  }
  st->newton_steps = steps;
  st->res = ctx->stage_norms[3];
  const bool ok = stage_converged(ctx);
  if ((rc = mehdg_stage_end(ctx, u))) return rc;
  if (!ok) return ctx_fail(ctx, MEHDG_ERR_NOT_CONVERGED, "Newton iteration cap reached");
  return MEHDG_OK;
}
