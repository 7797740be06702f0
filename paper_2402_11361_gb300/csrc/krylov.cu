// a8-a9: FGMRES on the condensed trace system and its preconditioners (Sec. 4.2).
//
// Flexible GMRES(restart) with right preconditioning: the Krylov basis V and the
// preconditioned directions Z live on the device in FP64; the Arnoldi step uses
// classical Gram-Schmidt applied twice (the paper's iterated CGS); dot products
// are block-reduced in a fixed order, so results are reproducible run to run.
// The (restart+1) x restart Hessenberg matrix and its Givens rotations live on the
// device; the host reads one residual estimate per outer iteration and copies the
// rotated Hessenberg back at the end of a cycle for the back-substitution.
// Preconditioners: kind 0 applies (A_uhuh)^-1 face block by face block (FP64 LU
// factors, or explicit FP32/BF16 inverses in the mixed path); kind 1 runs inner_iters
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
// block tickets of the one-launch reductions: 129 unsigned counters (one per vector of a
// multi-dot, one for the norm of k_maxpy_norm), zero between launches; the context
// clears the whole reduction buffer when it is made
constexpr size_t RED_CNT = RED_OUT + 1024;
constexpr int CNT_NORM = 128;

// Dot products out[i] = V_i . w (i < nv) in one launch: block (x, i) of the (RB, nv)
// grid sums its grid-strided share of vector i and stores the partial; the block that
// finishes vector i last (a ticket from an atomic counter, no waiting) adds the RB
// partials in a fixed tree order, so the result does not depend on which block came
// last.  With H, also H[i][col] (= or +=).  The last block resets its counter.
__device__ __forceinline__ double block_sum_256(double s, double* red8) {
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < 8; ++k) t += red8[k];
  return t;   // valid in thread 0
}
// the last of the blocks that stored a partial in part[0..RB) (counter *cnt) returns
// the fixed-order sum of those partials in thread 0 and true in every thread
__device__ __forceinline__ bool last_block_sum(const double* part, unsigned int* cnt, unsigned int nblk, double* red,
                                               double& total) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(cnt, 1u) == nblk - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // RB = 2 x 256 partials: the pairwise tree of a 512-wide reduction
  red[threadIdx.x] = __ldcg(part + threadIdx.x) + __ldcg(part + threadIdx.x + 256);
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    total = red[0];
    *cnt = 0u;
  }
  return true;
}
__global__ void __launch_bounds__(256) k_mdot(const double* __restrict__ V, long long ldv, const double* __restrict__ w,
                                              long long n, double* __restrict__ part, unsigned int* __restrict__ cnt,
                                              double* __restrict__ out, double* __restrict__ H, int ldh, int col,
                                              int accumulate) {
  __shared__ double red8[8];
  __shared__ double red[256];
  const int i = blockIdx.y;
  const double* v = V + (size_t)i * ldv;
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    s += v[k] * w[k];
  s = block_sum_256(s, red8);
  if (threadIdx.x == 0) part[(size_t)i * RB + blockIdx.x] = s;
  double t;
  if (!last_block_sum(part + (size_t)i * RB, cnt + i, gridDim.x, red, t)) return;
  if (threadIdx.x == 0) {
    out[i] = t;
    if (H) H[(size_t)i * ldh + col] = accumulate ? H[(size_t)i * ldh + col] + t : t;
  }
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
// w -= sum_i c_i V_i over an (RB)-block grid-strided range, and *dot = |w|^2 of the
// updated w by the same fixed-order reduction as k_mdot
__global__ void __launch_bounds__(256) k_maxpy_norm(const double* __restrict__ V, long long ldv, int nv,
                                                    const double* __restrict__ c, double* __restrict__ w, long long n,
                                                    double* __restrict__ part, unsigned int* __restrict__ cnt,
                                                    double* __restrict__ dot) {
  __shared__ double red8[8];
  __shared__ double red[256];
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a += c[i] * V[(size_t)i * ldv + k];
    const double y = w[k] - a;
    w[k] = y;
    s += y * y;
  }
  s = block_sum_256(s, red8);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  double t;
  if (!last_block_sum(part, cnt, gridDim.x, red, t)) return;
  if (threadIdx.x == 0) *dot = t;
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

// ---------------------------------------------------------------- device-side Arnoldi
// The orthogonalisation coefficients, the Hessenberg matrix and the Givens rotations
// stay on the device, so an Arnoldi step needs no host round trip: the outer FGMRES
// reads back one residual estimate per iteration, and the inner GMRES of the
// multi-level preconditioner (a fixed number of steps) runs as one CUDA graph.

// v = w / sqrt(*dot) (v = 0 if the norm is 0); thread 0 stores the norm in *nrm
__global__ void k_normalize(long long n, const double* __restrict__ dot, const double* __restrict__ w,
                            double* __restrict__ v, double* __restrict__ nrm) {
  const double s = sqrt(fmax(*dot, 0.0));
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k == 0 && nrm) *nrm = s;
  if (k < n) v[k] = w[k] * inv;
}
__global__ void k_set(double* p, double v) { *p = v; }
// Hessenberg block on the device: H [(m+1) x m] row-major, cs [m], sn [m], g [m+1]
struct DevHess {
  double *H, *cs, *sn, *g;
  int m;
};
__device__ void givens_column(DevHess h, int j) {
  const int m = h.m;
  for (int i = 0; i < j; ++i) {
    const double a = h.H[(size_t)i * m + j], b = h.H[(size_t)(i + 1) * m + j];
    h.H[(size_t)i * m + j] = h.cs[i] * a + h.sn[i] * b;
    h.H[(size_t)(i + 1) * m + j] = -h.sn[i] * a + h.cs[i] * b;
  }
  const double a = h.H[(size_t)j * m + j], b = h.H[(size_t)(j + 1) * m + j];
  const double rr = hypot(a, b);
  if (rr == 0.0) { h.cs[j] = 1.0; h.sn[j] = 0.0; }
  else { h.cs[j] = a / rr; h.sn[j] = b / rr; }
  h.H[(size_t)j * m + j] = rr;
  h.H[(size_t)(j + 1) * m + j] = 0.0;
  h.g[j + 1] = -h.sn[j] * h.g[j];
  h.g[j] = h.cs[j] * h.g[j];
}
// rotate column j; out[0] = |residual estimate|, out[1] = H[j+1][j] before the rotation
__global__ void k_givens_step(DevHess h, int j, double* out) {
  out[1] = h.H[(size_t)(j + 1) * h.m + j];
  givens_column(h, j);
  out[0] = fabs(h.g[j + 1]);
}
// least squares of a fresh (unrotated) k-column Hessenberg: rotate, back-substitute -> y
__global__ void k_lsq(DevHess h, int k, const double* __restrict__ beta, double* __restrict__ y) {
  for (int i = 0; i <= k; ++i) h.g[i] = 0.0;
  h.g[0] = *beta;
  for (int j = 0; j < k; ++j) givens_column(h, j);
  for (int i = k - 1; i >= 0; --i) {
    double s = h.g[i];
    for (int c = i + 1; c < k; ++c) s -= h.H[(size_t)i * h.m + c] * y[c];
    const double d = h.H[(size_t)i * h.m + i];
    y[i] = (d != 0.0) ? s / d : 0.0;
  }
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

// z_f = Minv_f r_f with an explicit inverse per face block (mixed precision).  Persistent
// grid: each CTA takes a contiguous range of the F * nfb rows and stages r_f (FP32, in
// dynamic shared memory of nfb floats) per face block.
// FP32 inverses [F nfb][nfb]: one warp per row.
__global__ void __launch_bounds__(256) k_block_gemv(const float* __restrict__ Minv, const double* __restrict__ r,
                                                    double* __restrict__ z, int nfb, int F, long long rows_per_cta) {
  extern __shared__ __align__(16) float xs[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long total = (long long)F * nfb, g0 = (long long)blockIdx.x * rows_per_cta;
  const long long g1 = min(g0 + rows_per_cta, total);
  for (long long gs = g0; gs < g1;) {
    const int f = (int)(gs / nfb);
    const long long ge = min(g1, (long long)(f + 1) * nfb);
    __syncthreads();
    for (int i = threadIdx.x; i < nfb; i += blockDim.x) xs[i] = (float)r[(size_t)f * nfb + i];
    __syncthreads();
    for (long long gr = gs + w; gr < ge; gr += nw) {
      const float* mr = Minv + (size_t)gr * nfb;
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = lane + 32 * u;
        v[u] = (c < nfb) ? __ldg(mr + c) : 0.f;
      }
      float s = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = lane + 32 * u;
        if (c < nfb) s += v[u] * xs[c];
      }
      for (int c = lane + 128; c < nfb; c += 32) s += __ldg(mr + c) * xs[c];
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) z[gr] = (double)s;
    }
    gs = ge;
  }
}
// BF16 inverses (raw 16-bit words) with rows padded to ld (a multiple of 32, zeros beyond
// nfb): eight lanes per row, four rows per warp.  Lane l of a row reads the 4-entry
// chunks at 32t + 4l (one 8-byte load each, 64 contiguous bytes per row and t) and the
// matching x chunk as one float4 (128 contiguous bytes per 8 lanes: no bank conflict);
// FP32 accumulation, a 3-step reduction within the 8 lanes.  For rows of up to 128
// entries the next four rows are requested before the current ones are multiplied, and
// a face block's first four rows before its x is gathered.
// FROM_SLOT: r is not a trace vector but the per-macro slots of an apply, and r_f is
// summed from the face's (up to two) owners on the fly (the face reduction fused in).
struct SlotMap {
  const int* owner;
  int Nt, Nth, Nfn, nf;   // nf: faces per macro-element
};
__device__ __forceinline__ float bf16x4_dot(uint2 v, float4 x) {
  return __uint_as_float(v.x << 16) * x.x + __uint_as_float(v.x & 0xFFFF0000u) * x.y +
         __uint_as_float(v.y << 16) * x.z + __uint_as_float(v.y & 0xFFFF0000u) * x.w;
}
template <bool FROM_SLOT>
__global__ void __launch_bounds__(256) k_block_gemv_bf16(const unsigned short* __restrict__ Minv, int ld,
                                                         const double* __restrict__ r, SlotMap sm,
                                                         double* __restrict__ z, int nfb, int F,
                                                         long long rows_per_cta) {
  extern __shared__ __align__(16) float xs[];   // ld floats, zero beyond nfb
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int q = lane >> 3, l8 = lane & 7, nch = ld >> 5;
  const long long total = (long long)F * nfb, g0 = (long long)blockIdx.x * rows_per_cta;
  const long long g1 = min(g0 + rows_per_cta, total);
  for (long long gs = g0; gs < g1;) {
    const int f = (int)(gs / nfb);
    const long long ge = min(g1, (long long)(f + 1) * nfb);
    // the first four rows' loads go out before x is gathered
    const bool pipe = nch <= 4;
    uint2 cur[4];
    if (pipe) {
      const long long gr = gs + 4 * w + q;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        cur[u] = (gr < ge && u < nch) ? __ldg(reinterpret_cast<const uint2*>(Minv + (size_t)gr * ld) + 8 * u + l8)
                                      : make_uint2(0u, 0u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ld; i += blockDim.x) {
      float v = 0.f;
      if (i < nfb) {
        if (FROM_SLOT) {
          const int s = i / sm.Nfn, j = i - s * sm.Nfn;
          double a = 0.0;
          for (int o = 0; o < 2; ++o) {
            const int ow = sm.owner[2 * f + o];
            if (ow < 0) continue;
            const int e = ow / sm.nf, fl = ow % sm.nf;
            a += r[(size_t)e * sm.Nt + (size_t)s * sm.Nth + fl * sm.Nfn + j];
          }
          v = (float)a;
        } else {
          v = (float)r[(size_t)f * nfb + i];
        }
      }
      xs[i] = v;
    }
    __syncthreads();
    if (pipe) {
      for (long long g4 = gs + 4 * w; g4 < ge; g4 += 4 * nw) {
        const long long gr = g4 + q, gn = gr + 4 * nw;
        uint2 nxt[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          nxt[u] = (gn < ge && u < nch) ? __ldg(reinterpret_cast<const uint2*>(Minv + (size_t)gn * ld) + 8 * u + l8)
                                        : make_uint2(0u, 0u);
        float s = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < nch) s += bf16x4_dot(cur[u], *reinterpret_cast<const float4*>(xs + 32 * u + 4 * l8));
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (gr < ge && l8 == 0) z[gr] = (double)s;
#pragma unroll
        for (int u = 0; u < 4; ++u) cur[u] = nxt[u];
      }
    } else {
      for (long long g4 = gs + 4 * w; g4 < ge; g4 += 4 * nw) {
        const long long gr = g4 + q;
        const bool act = gr < ge;
        float s = 0.f;
        if (act) {
          const uint2* mr = reinterpret_cast<const uint2*>(Minv + (size_t)gr * ld);
          for (int t0 = 0; t0 < nch; t0 += 4) {
            uint2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = (t0 + u < nch) ? __ldg(mr + 8 * (t0 + u) + l8) : make_uint2(0u, 0u);
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (t0 + u < nch) s += bf16x4_dot(v[u], *reinterpret_cast<const float4*>(xs + 32 * (t0 + u) + 4 * l8));
          }
        }
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (act && l8 == 0) z[gr] = (double)s;
      }
    }
    gs = ge;
  }
}

unsigned int* red_cnt(mehdg_ctx* ctx) { return reinterpret_cast<unsigned int*>(ctx->dred + RED_CNT); }

int mdot(mehdg_ctx* ctx, const double* V, long long ldv, int nv, const double* w, long long n, double* host) {
  dim3 grid(RB, nv);
  k_mdot<<<grid, 256, 0, ctx->stream>>>(V, ldv, w, n, ctx->dred, red_cnt(ctx), ctx->dred + RED_OUT, nullptr, 0, 0, 0);
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

// scratch in dred after the reduction results: [RED_OUT .. +128) results, +128 coefficients
constexpr size_t RED_SCAL = RED_OUT + 256;   // device scalars (norms, residual estimates)

// out[0..nv) = V_i . w, on the device (no host copy); with H, also H[i][col]
int mdot_dev(mehdg_ctx* ctx, const double* V, long long ldv, int nv, const double* w, long long n, double* out,
             double* H = nullptr, int ldh = 0, int col = 0, int accumulate = 0) {
  dim3 grid(RB, nv);
  k_mdot<<<grid, 256, 0, ctx->stream>>>(V, ldv, w, n, ctx->dred, red_cnt(ctx), out, H, ldh, col, accumulate);
  CKL();
  return MEHDG_OK;
}

// CGS2 step on the device: w -= V[0..j] (V^T w) twice (coefficients summed into H[.][j]),
// H[j+1][j] = |w|, V[j+1] = w / |w|
int arnoldi_dev(mehdg_ctx* ctx, double* V, int j, double* w, long long n, DevHess h) {
  double* coef = ctx->dred + RED_OUT;
  int rc;
  double* dot = ctx->dred + RED_SCAL;
  for (int pass = 0; pass < 2; ++pass) {
    if ((rc = mdot_dev(ctx, V, n, j + 1, w, n, coef, h.H, h.m, j, pass))) return rc;
    if (pass == 0) {
      k_maxpy<<<(n + 255) / 256, 256, 0, ctx->stream>>>(V, n, j + 1, coef, w, n, -1.0);
    } else {
      // second update fused with |w|^2
      k_maxpy_norm<<<RB, 256, 0, ctx->stream>>>(V, n, j + 1, coef, w, n, ctx->dred, red_cnt(ctx) + CNT_NORM, dot);
    }
    CKL();
  }
  k_normalize<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, dot, w, V + (size_t)(j + 1) * n,
                                                         h.H + (size_t)(j + 1) * h.m + j);
  CKL();
  return MEHDG_OK;
}

DevHess dev_hess(double* base, int m) {
  DevHess h;
  h.m = m;
  h.H = base;
  h.cs = base + (size_t)(m + 1) * m;
  h.sn = h.cs + m;
  h.g = h.sn + m;
  return h;
}

// host copy of a rotated Hessenberg (upper triangular part) and its right-hand side,
// for the back-substitution of a cycle's iterates
struct Hess {
  int m;
  std::vector<double> H, g;
  explicit Hess(int m_) : m(m_), H((m_ + 1) * m_, 0.0), g(m_ + 1, 0.0) {}
  double& h(int i, int j) { return H[(size_t)i * m + j]; }
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

// from_slot: r holds the per-macro slots of an apply (BF16 face inverses only)
static int block_jacobi(mehdg_ctx* ctx, const double* r, double* z, bool from_slot = false) {
  size_t smem = sizeof(double) * ctx->nfb;
  if (ctx->finv32) {
    const bool lowp = ctx->lowp_apply && ctx->finv16;
    if (from_slot && !lowp) return ctx_fail(ctx, MEHDG_ERR_ARG, "slot input needs the BF16 face inverses");
    int& grid = lowp ? ctx->bj_grid16 : ctx->bj_grid;
    const size_t xsm = sizeof(float) * (size_t)(lowp ? ctx->ldf16 : ctx->nfb);
    if (grid <= 0) {
      int dev = 0, sms = 0, per = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      if (lowp) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_block_gemv_bf16<true>, 256, xsm));
      else CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_block_gemv, 256, xsm));
      grid = std::max(1, sms * std::max(1, per));
    }
    const long long total = (long long)ctx->F * ctx->nfb, rows = (total + grid - 1) / grid;
    phase_begin(ctx, PH_PRECOND);
    const SlotMap sm{ctx->owner, ctx->Nt, ctx->Nth, ctx->Nfn, ctx->nf};
    if (lowp && from_slot)
      k_block_gemv_bf16<true><<<grid, 256, xsm, ctx->stream>>>(ctx->finv16, ctx->ldf16, r, sm, z, ctx->nfb, ctx->F,
                                                               rows);
    else if (lowp)
      k_block_gemv_bf16<false><<<grid, 256, xsm, ctx->stream>>>(ctx->finv16, ctx->ldf16, r, sm, z, ctx->nfb, ctx->F,
                                                                rows);
    else
      k_block_gemv<<<grid, 256, xsm, ctx->stream>>>(ctx->finv32, r, z, ctx->nfb, ctx->F, rows);
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

// kind 1: nu steps of GMRES on A^ left-preconditioned by block-Jacobi, from z = 0,
// entirely on the device (fixed step count: no convergence test, no host round trip)
static int inner_gmres_dev(mehdg_ctx* ctx, const double* r, double* z) {
  const long long n = ctx->ntr;
  const int nu = std::min(120, std::max(1, ctx->opt.inner_iters));
  int rc;
  double* IV = ctx->iV;
  DevHess h = dev_hess(ctx->dHi, nu);
  double* beta = ctx->dred + RED_SCAL + 1;
  double* dot = ctx->dred + RED_SCAL + 2;
  double* y = ctx->dred + RED_SCAL + 8;
  CK(cudaMemsetAsync(h.H, 0, sizeof(double) * (size_t)(nu + 1) * nu, ctx->stream));
  if ((rc = block_jacobi(ctx, r, ctx->iw))) return rc;
  if ((rc = mdot_dev(ctx, ctx->iw, n, 1, ctx->iw, n, dot))) return rc;
  k_normalize<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, dot, ctx->iw, IV, beta);
  CKL();
  const bool slots = apply_bf16_slots_available(ctx);
  for (int j = 0; j < nu; ++j) {
    ctx->lowp_apply = true;   // the BF16 operator and face-inverse copies, when the context keeps them
    if (slots) {
      // BF16 apply into the per-macro slots; the block-Jacobi product sums the owners
      rc = apply_bf16_slots(ctx, IV + (size_t)j * n);
      if (rc == MEHDG_OK) rc = block_jacobi(ctx, ctx->slot, ctx->iw, true);
    } else {
      rc = apply_trace_impl(ctx, IV + (size_t)j * n, ctx->tv);
      if (rc == MEHDG_OK) rc = block_jacobi(ctx, ctx->tv, ctx->iw);
    }
    ctx->lowp_apply = false;
    if (rc) return rc;
    if ((rc = arnoldi_dev(ctx, IV, j, ctx->iw, n, h))) return rc;
  }
  k_lsq<<<1, 1, 0, ctx->stream>>>(h, nu, beta, y);
  CKL();
  CK(cudaMemsetAsync(z, 0, sizeof(double) * n, ctx->stream));
  k_maxpy<<<(n + 255) / 256, 256, 0, ctx->stream>>>(IV, n, nu, y, z, n, 1.0);
  CKL();
  return MEHDG_OK;
}

// The inner GMRES is captured once per context into a CUDA graph on fixed input and
// output buffers (all other pointers are fixed for the context's lifetime); each call
// copies r in, replays the graph and copies z out.
static int inner_gmres(mehdg_ctx* ctx, const double* r, double* z) {
  const long long n = ctx->ntr;
  if (!ctx->ig_exec && !ctx->ig_failed) {
    cudaGraph_t graph = nullptr;
    const long long l0 = ctx->launches;
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      ctx->capturing = true;
      int rc = inner_gmres_dev(ctx, ctx->gin, ctx->gout);
      ctx->capturing = false;
      cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
      if (rc == MEHDG_OK && ec == cudaSuccess && graph &&
          cudaGraphInstantiate(&ctx->ig_exec, graph, 0) == cudaSuccess) {
        ctx->ig_nodes = ctx->launches - l0;
      } else {
        ctx->ig_exec = nullptr;
        ctx->ig_failed = true;
      }
      if (graph) cudaGraphDestroy(graph);
      ctx->launches = l0;
      cudaGetLastError();
    } else {
      ctx->ig_failed = true;
      cudaGetLastError();
    }
  }
  if (!ctx->ig_exec) return inner_gmres_dev(ctx, r, z);
  CK(cudaMemcpyAsync(ctx->gin, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaGraphLaunch(ctx->ig_exec, ctx->stream));
  ctx->launches += ctx->ig_nodes;
  ++ctx->ig_replays;
  ++ctx->ig_total;
  CK(cudaMemcpyAsync(z, ctx->gout, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  return MEHDG_OK;
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

// GMRES(k) left-preconditioned by the block-Jacobi (A_uhuh)^-1 of the macro-faces: the
// baseline solver of Sec. 4.2 (the first option there, GMRES with a fixed preconditioner;
// compared with FGMRES and the multi-level preconditioner in the paper's Table 2).  Arnoldi
// (CGS2, FP64, on the device) runs on M^-1 A^; the iterate is x = x_start + V y; the
// stopping test is on the preconditioned residual |M^-1 (b - A^ x)| <= max(rtol |M^-1 b|, atol).
static int gmres_left_impl(mehdg_ctx* ctx, const double* b, double* x, mehdg_solve_stats* st) {
  const long long n = ctx->ntr;
  const int m = ctx->restart;
  int rc;
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
  if ((rc = block_jacobi(ctx, b, ctx->rv))) return rc;
  double beta;
  if ((rc = vec_dot(ctx, ctx->rv, ctx->rv, n, &beta))) return rc;
  beta = std::sqrt(beta);
  const double tol = std::max(ctx->opt.lin_rtol * beta, ctx->opt.lin_atol);
  int its = 0;
  bool conv = beta <= tol;
  while (!conv && its < ctx->opt.max_iters) {
    if ((rc = vec_lincomb(ctx, n, 1.0 / beta, ctx->rv, 0.0, ctx->rv, ctx->V))) return rc;
    Hess hs(m);
    hs.g[0] = beta;
    DevHess dh = dev_hess(ctx->dHo, m);
    CK(cudaMemsetAsync(dh.H, 0, sizeof(double) * ((size_t)(m + 1) * m + 3 * (size_t)m + 1), ctx->stream));
    k_set<<<1, 1, 0, ctx->stream>>>(dh.g, beta);
    CKL();
    double* est = ctx->dred + RED_SCAL + 4;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      if ((rc = apply_trace_impl(ctx, ctx->V + (size_t)j * n, ctx->tv))) return rc;
      if ((rc = block_jacobi(ctx, ctx->tv, ctx->wv))) return rc;
      if ((rc = arnoldi_dev(ctx, ctx->V, j, ctx->wv, n, dh))) return rc;
      k_givens_step<<<1, 1, 0, ctx->stream>>>(dh, j, est);
      CKL();
      CK(cudaMemcpyAsync(ctx->hred + 200, est, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      phase_harvest(ctx);
      const double res = ctx->hred[200], hn = ctx->hred[201];
      ++its;
      k = j + 1;
      if (!std::isfinite(res)) return ctx_fail(ctx, MEHDG_ERR_NAN, "non-finite GMRES residual");
      if (res <= tol || its >= ctx->opt.max_iters || hn == 0.0) break;
    }
    CK(cudaMemcpyAsync(hs.H.data(), dh.H, sizeof(double) * hs.H.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hs.g.data(), dh.g, sizeof(double) * hs.g.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<double> y = hs.solve(k);
    if ((rc = maxpy(ctx, ctx->V, n, k, y.data(), x, n, 1.0))) return rc;
    // restart residual M^-1 (b - A^ x)
    if ((rc = apply_trace_impl(ctx, x, ctx->wv))) return rc;
    if ((rc = vec_lincomb(ctx, n, 1.0, b, -1.0, ctx->wv, ctx->tv))) return rc;
    if ((rc = block_jacobi(ctx, ctx->tv, ctx->rv))) return rc;
    if ((rc = vec_dot(ctx, ctx->rv, ctx->rv, n, &beta))) return rc;
    beta = std::sqrt(beta);
    conv = beta <= tol;
  }
  if (st) {
    st->fgmres_iters += its;
    st->res = beta;
  }
  if (!conv) return ctx_fail(ctx, MEHDG_ERR_NOT_CONVERGED, "GMRES reached its iteration cap");
  return MEHDG_OK;
}

int linear_solve_impl(mehdg_ctx* ctx, const double* b, double* x, mehdg_solve_stats* st) {
  if (ctx->opt.solver == 1) return gmres_left_impl(ctx, b, x, st);
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
    DevHess dh = dev_hess(ctx->dHo, m);
    CK(cudaMemsetAsync(dh.H, 0, sizeof(double) * ((size_t)(m + 1) * m + 3 * (size_t)m + 1), ctx->stream));
    k_set<<<1, 1, 0, ctx->stream>>>(dh.g, beta);
    CKL();
    double* est = ctx->dred + RED_SCAL + 4;
    int k = 0;
    bool fallback = false;
    for (int j = 0; j < m; ++j) {
      double* Zj = ctx->Zk + (size_t)j * n;
      if ((rc = precond_impl(ctx, kind, ctx->V + (size_t)j * n, Zj))) return rc;
      if ((rc = apply_trace_impl(ctx, Zj, ctx->wv))) return rc;
      if ((rc = arnoldi_dev(ctx, ctx->V, j, ctx->wv, n, dh))) return rc;
      k_givens_step<<<1, 1, 0, ctx->stream>>>(dh, j, est);
      CKL();
      CK(cudaMemcpyAsync(ctx->hred + 200, est, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      phase_harvest(ctx);
      const double res = ctx->hred[200], hn = ctx->hred[201];
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
    // rotated Hessenberg and right-hand side of this cycle to the host
    CK(cudaMemcpyAsync(hs.H.data(), dh.H, sizeof(double) * hs.H.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hs.g.data(), dh.g, sizeof(double) * hs.g.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
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

extern "C" int mehdg_set_precond(mehdg_ctx* ctx, int kind) {
  if (!ctx || kind < 0 || kind > 2) return MEHDG_ERR_ARG;
  if (kind == 2 && !ctx->mlp) return ctx_fail(ctx, MEHDG_ERR_ARG, "kind 2 needs mehdg_mlp_setup");
  ctx->opt.precond = kind;
  return MEHDG_OK;
}
