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
  double t3 = now();
  if (st) {
    st->t_condense += t1 - t0;
    st->t_krylov += t2 - t1;
    st->t_recover += t3 - t2;
  }
  return MEHDG_OK;
}

}  // namespace

extern "C" int mehdg_dirk_stage(mehdg_ctx* ctx, int stage, double dt, double* u, double* q, double* uh,
                                mehdg_solve_stats* st) {
  if (!ctx || !u || !q || !uh || stage < 0 || stage > 3) return MEHDG_ERR_ARG;
  if (stage > 0 && !(dt > 0.0)) return MEHDG_ERR_ARG;
  mehdg_solve_stats local{};
  if (!st) st = &local;
  *st = mehdg_solve_stats{};
  const long long nu = (long long)ctx->E * ctx->Nu;
  int rc;
  double norms[4];
  mehdg_time_term tt{0.0, nullptr, 0};
  const mehdg_time_term* ttp = nullptr;
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
    tt.coef = coef;
    tt.hist = ctx->hist;
    tt.supg_time = 1;
    ttp = &tt;
  }
  double t0 = now();
  if ((rc = assemble_all(ctx, u, q, uh, ttp, norms))) return rc;
  st->t_assemble += now() - t0;
  const double R0 = norms[3];
  st->res0 = R0;
  double dtau = ctx->opt.tau_init;
  int steps = 0;
  while (norms[3] > std::max(ctx->opt.newton_rtol * R0, ctx->opt.newton_atol) && steps < ctx->opt.max_newton) {
    if (!std::isfinite(norms[3])) return ctx_fail(ctx, MEHDG_ERR_NAN, "non-finite residual");
    double shift = (stage == 0) ? 1.0 / dtau : 0.0;
    rc = newton_step(ctx, shift, u, q, uh, st);
    if (rc) return rc;
    double RU_old = norms[1];
    t0 = now();
    if ((rc = assemble_all(ctx, u, q, uh, ttp, norms))) return rc;
    st->t_assemble += now() - t0;
    ++steps;
    if (stage == 0)
      dtau = std::min(std::max(dtau * RU_old / std::max(norms[1], 1e-300), ctx->opt.tau_init), ctx->opt.tau_max);
  }
  st->newton_steps = steps;
  st->res = norms[3];
  if (stage > 0) {
    if ((rc = vec_copy(ctx, nu, u, ctx->ustage + (size_t)(stage - 1) * nu))) return rc;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (norms[3] > std::max(ctx->opt.newton_rtol * R0, ctx->opt.newton_atol))
    return ctx_fail(ctx, MEHDG_ERR_NOT_CONVERGED, "Newton iteration cap reached");
  return MEHDG_OK;
}
