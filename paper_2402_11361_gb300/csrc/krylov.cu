// a8-a9: FGMRES on the condensed trace system and its preconditioners (Sec. 4.2).
//
// Flexible GMRES(restart) with right preconditioning: the Krylov basis V and the
// preconditioned directions Z live on the device in FP64; the Arnoldi step uses
// classical Gram-Schmidt applied twice (the paper's iterated CGS); dot products
// are block-reduced in a fixed order, so results are reproducible run to run.
// The (restart+1) x restart Hessenberg matrix and its Givens rotations stay on
// the host.  Preconditioners: kind 0 applies (A_uhuh)^-1 face block by face block
// with the LU factors made in mehdg_condense_factor; kind 1 runs inner_iters
// steps of GMRES on A^, left-preconditioned by kind 0 (the paper's multi-level
// preconditioner, a variable operator that FGMRES tolerates); kind 2 adds the
// learned correction to kind 0.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "lu.cuh"

namespace {

constexpr int RB = 512;   // reduction blocks
constexpr size_t RED_OUT = (size_t)RB * 128;   // dred layout: partials [128][RB], results, coefficients

__global__ void k_mdot_part(const double* __restrict__ V, long long ldv, int nv, const double* __restrict__ w,
                            long long n, double* __restrict__ part) {
  __shared__ double red[256 / 32];
  const int i = blockIdx.y;
  const double* v = V + (size_t)i * ldv;
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    s += v[k] * w[k];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    part[(size_t)i * RB + blockIdx.x] = t;
  }
}
__global__ void k_mdot_final(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[RB];
  const int i = blockIdx.x;
  red[threadIdx.x] = part[(size_t)i * RB + threadIdx.x];
  __syncthreads();
  for (int s = RB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = red[0];
}
// y += sum_i c_i V_i  (c on the device)
__global__ void k_maxpy(const double* __restrict__ V, long long ldv, int nv, const double* __restrict__ c,
                        double* __restrict__ y, long long n, double sign) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = 0.0;
  for (int i = 0; i < nv; ++i) s += c[i] * V[(size_t)i * ldv + k];
  y[k] += sign * s;
}
__global__ void k_axpy(long long n, double a, const double* x, double* y) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) y[k] += a * x[k];
}
__global__ void k_scal(long long n, double a, double* x) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) x[k] *= a;
}
__global__ void k_lincomb(long long n, double a, const double* x, double b, const double* y, double* z) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) z[k] = a * x[k] + b * y[k];
}

// block-Jacobi: z_f = (A_uhuh,f)^-1 r_f
__global__ void __launch_bounds__(128) k_block_jacobi(const double* __restrict__ fblk, const int* __restrict__ fperm,
                                                      const double* __restrict__ r, double* __restrict__ z, int nfb) {
  extern __shared__ double sy[];
  const int f = blockIdx.x;
  const double* rf = r + (size_t)f * nfb;
  const int* pf = fperm + (size_t)f * nfb;
  for (int i = threadIdx.x; i < nfb; i += blockDim.x) sy[i] = rf[pf[i]];
  __syncthreads();
  lu_solve_block<double>(fblk + (size_t)f * nfb * nfb, nfb, sy);
  for (int i = threadIdx.x; i < nfb; i += blockDim.x) z[(size_t)f * nfb + i] = sy[i];
}

// z_f = Minv_f r_f with an explicit FP32 inverse per face block (mixed precision)
__global__ void __launch_bounds__(256) k_block_gemv(const float* __restrict__ Minv, const double* __restrict__ r,
                                                    double* __restrict__ z, int nfb) {
  __shared__ float xs[512];
  const int f = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < nfb; i += blockDim.x) xs[i] = (float)r[(size_t)f * nfb + i];
  __syncthreads();
  const float* Mf = Minv + (size_t)f * nfb * nfb;
  for (int row = w; row < nfb; row += nw) {
    const float* mr = Mf + (size_t)row * nfb;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int c = lane;
    for (; c + 96 < nfb; c += 128) {
      s0 += mr[c] * xs[c];
      s1 += mr[c + 32] * xs[c + 32];
      s2 += mr[c + 64] * xs[c + 64];
      s3 += mr[c + 96] * xs[c + 96];
    }
    for (; c < nfb; c += 32) s0 += mr[c] * xs[c];
    float s = (s0 + s1) + (s2 + s3);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) z[(size_t)f * nfb + row] = (double)s;
  }
}

int mdot(mehdg_ctx* ctx, const double* V, long long ldv, int nv, const double* w, long long n, double* host) {
  dim3 grid(RB, nv);
  k_mdot_part<<<grid, 256, 0, ctx->stream>>>(V, ldv, nv, w, n, ctx->dred);
  k_mdot_final<<<nv, RB, 0, ctx->stream>>>(ctx->dred, ctx->dred + RED_OUT);
  CKL();
  CK(cudaMemcpyAsync(ctx->hred, ctx->dred + RED_OUT, sizeof(double) * nv, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < nv; ++i) host[i] = ctx->hred[i];
  return MEHDG_OK;
}

int maxpy(mehdg_ctx* ctx, const double* V, long long ldv, int nv, const double* chost, double* y, long long n,
          double sign) {
  double* dc = ctx->dred + RED_OUT + 128;
  CK(cudaMemcpyAsync(dc, chost, sizeof(double) * nv, cudaMemcpyHostToDevice, ctx->stream));
  k_maxpy<<<(n + 255) / 256, 256, 0, ctx->stream>>>(V, ldv, nv, dc, y, n, sign);
  CKL();
  // the host buffer chost must stay valid until the copy ran
  CK(cudaStreamSynchronize(ctx->stream));
  return MEHDG_OK;
}

// Givens-based least squares for the small Hessenberg problem (host)
struct Hess {
  int m;
  std::vector<double> H, cs, sn, g;
  explicit Hess(int m_) : m(m_), H((m_ + 1) * m_, 0.0), cs(m_, 0.0), sn(m_, 0.0), g(m_ + 1, 0.0) {}
  double& h(int i, int j) { return H[(size_t)i * m + j]; }
  // rotate column j (already holding the new Arnoldi coefficients); returns |residual|
  double rotate(int j) {
    for (int i = 0; i < j; ++i) {
      double t = cs[i] * h(i, j) + sn[i] * h(i + 1, j);
      h(i + 1, j) = -sn[i] * h(i, j) + cs[i] * h(i + 1, j);
      h(i, j) = t;
    }
    double rr = std::hypot(h(j, j), h(j + 1, j));
    if (rr == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
    else { cs[j] = h(j, j) / rr; sn[j] = h(j + 1, j) / rr; }
    h(j, j) = rr;
    h(j + 1, j) = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    return std::fabs(g[j + 1]);
  }
  std::vector<double> solve(int k) {
    std::vector<double> y(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int c = i + 1; c < k; ++c) s -= h(i, c) * y[c];
      y[i] = (h(i, i) != 0.0) ? s / h(i, i) : 0.0;
    }
    return y;
  }
};

// CGS2 step: orthogonalise w against V[0..j], H column j, then normalise into V[j+1]
int arnoldi_cgs2(mehdg_ctx* ctx, double* V, int j, double* w, long long n, Hess& hs, double* hnorm) {
  std::vector<double> h(j + 1);
  for (int pass = 0; pass < 2; ++pass) {
    int rc = mdot(ctx, V, n, j + 1, w, n, h.data());
    if (rc) return rc;
    rc = maxpy(ctx, V, n, j + 1, h.data(), w, n, -1.0);
    if (rc) return rc;
    for (int i = 0; i <= j; ++i) hs.h(i, j) += h[i];
  }
  double nn;
  int rc = mdot(ctx, w, n, 1, w, n, &nn);
  if (rc) return rc;
  nn = std::sqrt(nn);
  hs.h(j + 1, j) = nn;
  *hnorm = nn;
  if (nn > 0.0) {
    k_lincomb<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, 1.0 / nn, w, 0.0, w, V + (size_t)(j + 1) * n);
    CKL();
  }
  return MEHDG_OK;
}

}  // namespace

int vec_dot(mehdg_ctx* ctx, const double* a, const double* b, long long n, double* out) {
  return mdot(ctx, a, n, 1, b, n, out);
}
int vec_axpy(mehdg_ctx* ctx, long long n, double a, const double* x, double* y) {
  k_axpy<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, a, x, y);
  CKL();
  return MEHDG_OK;
}
int vec_scal(mehdg_ctx* ctx, long long n, double a, double* x) {
  k_scal<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, a, x);
  CKL();
  return MEHDG_OK;
}
int vec_copy(mehdg_ctx* ctx, long long n, const double* x, double* y) {
  CK(cudaMemcpyAsync(y, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  return MEHDG_OK;
}
int vec_lincomb(mehdg_ctx* ctx, long long n, double a, const double* x, double b, const double* y, double* z) {
  k_lincomb<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, a, x, b, y, z);
  CKL();
  return MEHDG_OK;
}

static int block_jacobi(mehdg_ctx* ctx, const double* r, double* z) {
  size_t smem = sizeof(double) * ctx->nfb;
  if (ctx->finv32) {
    phase_begin(ctx, PH_PRECOND);
    k_block_gemv<<<ctx->F, 256, 0, ctx->stream>>>(ctx->finv32, r, z, ctx->nfb);
    CKL();
    phase_end(ctx, PH_PRECOND);
    return MEHDG_OK;
  }
  phase_begin(ctx, PH_PRECOND);
  k_block_jacobi<<<ctx->F, 128, smem, ctx->stream>>>(ctx->fblk, ctx->fperm, r, z, ctx->nfb);
  CKL();
  phase_end(ctx, PH_PRECOND);
  return MEHDG_OK;
}

// kind 1: nu steps of GMRES on A^ left-preconditioned by block-Jacobi, from z = 0
static int inner_gmres(mehdg_ctx* ctx, const double* r, double* z) {
  const long long n = ctx->ntr;
  const int nu = std::min(120, std::max(1, ctx->opt.inner_iters));
  int rc;
  double* IV = ctx->iV;
  if ((rc = block_jacobi(ctx, r, ctx->iw))) return rc;
  double beta;
  if ((rc = vec_dot(ctx, ctx->iw, ctx->iw, n, &beta))) return rc;
  beta = std::sqrt(beta);
  CK(cudaMemsetAsync(z, 0, sizeof(double) * n, ctx->stream));
  if (beta == 0.0) return MEHDG_OK;
  if ((rc = vec_lincomb(ctx, n, 1.0 / beta, ctx->iw, 0.0, ctx->iw, IV))) return rc;
  Hess hs(nu);
  hs.g[0] = beta;
  int k = 0;
  for (int j = 0; j < nu; ++j) {
    if ((rc = apply_trace_impl(ctx, IV + (size_t)j * n, ctx->tv))) return rc;
    if ((rc = block_jacobi(ctx, ctx->tv, ctx->iw))) return rc;
    double hn;
    if ((rc = arnoldi_cgs2(ctx, IV, j, ctx->iw, n, hs, &hn))) return rc;
    hs.rotate(j);
    k = j + 1;
    if (hn == 0.0) break;
  }
  std::vector<double> y = hs.solve(k);
  return maxpy(ctx, IV, n, k, y.data(), z, n, 1.0);
}

int precond_impl(mehdg_ctx* ctx, int kind, const double* r, double* z) {
  if (!ctx->condensed) return ctx_fail(ctx, MEHDG_ERR_ARG, "precondition before mehdg_condense_factor");
  if (kind == 0) return block_jacobi(ctx, r, z);
  if (kind == 1) return inner_gmres(ctx, r, z);
  if (kind == 2) {
    int rc = block_jacobi(ctx, r, z);
    if (rc) return rc;
    return mlp_apply(ctx, r, z);
  }
  return ctx_fail(ctx, MEHDG_ERR_ARG, "unknown preconditioner kind");
}

int linear_solve_impl(mehdg_ctx* ctx, const double* b, double* x, mehdg_solve_stats* st) {
  const long long n = ctx->ntr;
  const int m = ctx->restart;
  int rc;
  double bnorm;
  if ((rc = vec_dot(ctx, b, b, n, &bnorm))) return rc;
  bnorm = std::sqrt(bnorm);
  const double tol = std::max(ctx->opt.lin_rtol * bnorm, ctx->opt.lin_atol);
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
  if ((rc = vec_copy(ctx, n, b, ctx->rv))) return rc;
  double beta = bnorm;
  int its = 0;
  bool conv = beta <= tol;
  int kind = ctx->opt.precond;
  // learned preconditioner fallback: switch to the multi-level preconditioner when the
  // residual falls by less than 10x over 20 iterations
  double watch = beta;
  int watch_it = 0;
  Hess last(m);
  int last_k = 0;
  while (!conv && its < ctx->opt.max_iters) {
    if ((rc = vec_copy(ctx, n, x, ctx->xstart))) return rc;
    if ((rc = vec_lincomb(ctx, n, 1.0 / beta, ctx->rv, 0.0, ctx->rv, ctx->V))) return rc;
    Hess hs(m);
    hs.g[0] = beta;
    int k = 0;
    bool fallback = false;
    for (int j = 0; j < m; ++j) {
      double* Zj = ctx->Zk + (size_t)j * n;
      if ((rc = precond_impl(ctx, kind, ctx->V + (size_t)j * n, Zj))) return rc;
      if ((rc = apply_trace_impl(ctx, Zj, ctx->wv))) return rc;
      double hn;
      if ((rc = arnoldi_cgs2(ctx, ctx->V, j, ctx->wv, n, hs, &hn))) return rc;
      double res = hs.rotate(j);
      ++its;
      k = j + 1;
      if (!std::isfinite(res)) return ctx_fail(ctx, MEHDG_ERR_NAN, "non-finite FGMRES residual");
      if (res <= tol || its >= ctx->opt.max_iters || hn == 0.0) break;
      if (kind == 2 && its - watch_it >= 20) {
        if (res > 0.1 * watch) {
          fallback = true;
          break;
        }
        watch = res;
        watch_it = its;
      }
    }
    std::vector<double> y = hs.solve(k);
    if ((rc = maxpy(ctx, ctx->Zk, n, k, y.data(), x, n, 1.0))) return rc;
    if ((rc = apply_trace_impl(ctx, x, ctx->wv))) return rc;
    if ((rc = vec_lincomb(ctx, n, 1.0, b, -1.0, ctx->wv, ctx->rv))) return rc;
    if ((rc = vec_dot(ctx, ctx->rv, ctx->rv, n, &beta))) return rc;
    beta = std::sqrt(beta);
    conv = beta <= tol;
    last = hs;
    last_k = k;
    if (fallback) {
      kind = 1;
      if (st) st->status |= 1;   // bit 0: the learned preconditioner fell back
    }
  }
  if (st) {
    st->fgmres_iters += its;
    st->res = beta;
  }
  if (!conv) return ctx_fail(ctx, MEHDG_ERR_NOT_CONVERGED, "FGMRES reached its iteration cap");
  if (mlp_recording(ctx) && last_k > 0) {
    // (residual, error) pairs of iterates of the last cycle: x_i = x_start + Z y_i,
    // y_i from the rotated Hessenberg of that cycle (its first i columns are final)
    const int npairs = std::min(8, last_k);
    int prev = -1;
    for (int q = 0; q < npairs; ++q) {
      int i = (int)((long long)q * last_k / npairs);
      if (i == prev) continue;
      prev = i;
      if ((rc = vec_copy(ctx, n, ctx->xstart, ctx->tv2))) return rc;
      if (i > 0) {
        std::vector<double> yi = last.solve(i);
        if ((rc = maxpy(ctx, ctx->Zk, n, i, yi.data(), ctx->tv2, n, 1.0))) return rc;
      }
      if ((rc = apply_trace_impl(ctx, ctx->tv2, ctx->wv))) return rc;
      if ((rc = vec_lincomb(ctx, n, 1.0, b, -1.0, ctx->wv, ctx->rv))) return rc;
      if ((rc = vec_lincomb(ctx, n, 1.0, x, -1.0, ctx->tv2, ctx->tv))) return rc;
      if ((rc = mlp_record_pair(ctx, ctx->rv, ctx->tv))) return rc;
    }
  }
  return MEHDG_OK;
}

extern "C" int mehdg_precondition(mehdg_ctx* ctx, int kind, const double* r, double* z) {
  if (!ctx || !r || !z || r == z) return MEHDG_ERR_ARG;
  return precond_impl(ctx, kind, r, z);
}

extern "C" int mehdg_linear_solve(mehdg_ctx* ctx, const double* b, double* x, mehdg_solve_stats* st) {
  if (!ctx || !b || !x || b == x) return MEHDG_ERR_ARG;
  return linear_solve_impl(ctx, b, x, st);
}
