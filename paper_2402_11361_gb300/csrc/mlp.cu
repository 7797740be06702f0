// Learned preconditioner correction (preconditioner kind 2).  Not part of the
// paper: FGMRES accepts a variable preconditioner (Sec. 4.2), so the block-Jacobi
// output z0 = (A_uhuh)^-1 r is corrected face by face by a small network,
//   z_f = z0_f + |z0_f| MLP(r_f / |r_f|, z0_f / |z0_f| [, z0_g / |z0_f| for the faces g
//                                                         of the face's owners]),
// MLP: n_in -> hid (ReLU) -> hid (ReLU) -> n_out with n_out = ns Nfn rounded up to a
// multiple of 32 and n_in = 2 n_out (the two normalised face vectors), or (2 + 2 (2d - 1))
// n_out with the neighbouring faces' block-Jacobi outputs (the error that block-Jacobi
// leaves is carried by the coupling through the two owner macro-elements).  Weights are
// stored in BF16 for the products, with FP32 master copies, FP32 biases and FP32
// accumulation everywhere.  Training pairs (residual r, error e) come from the plain
// FGMRES solves; the target of face f is (e_f - z0_f) / |z0_f|, what block-Jacobi
// misses relative to its own output.  Forward, backward and Adam run in the kernels
// below.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace {

struct Mlp {
  int nin, nh, nout, nfb, F;
  int nnb = 0;                   // neighbouring faces per face in the input (0: the face alone)
  int* nbr = nullptr;            // [F][nnb] their face ids, -1 where absent
  long long np;                  // parameter count
  long long oW1, ob1, oW2, ob2, oW3, ob3;
  float *P = nullptr, *G = nullptr, *Mm = nullptr, *Vv = nullptr;   // master params, grads, Adam moments
  __nv_bfloat16* Ph = nullptr;   // BF16 copy of the parameters
  float *X = nullptr, *T = nullptr;   // recorded samples [cap][nin], targets [cap][nout]
  int cap = 0, count = 0;
  int wcap = 0;                       // rows of the work buffers
  float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *dH1 = nullptr, *dH2 = nullptr,
        *Xin = nullptr;
  double* nrm = nullptr;              // per-face norms |z0_f|
  double* dloss = nullptr;
  long long step = 0;
  bool trained = false;
  bool recording = false;
};

// C[m][n] = act(sum_k A(m,k) B(k,n) + bias[n]) (then optionally masked) + beta C[m][n]
// A(m,k) = TA ? A[k lda + m] : A[m lda + k];  B(k,n) = TB ? B[n ldb + k] : B[k ldb + n]
template <class BT, bool TA, bool TB>
__global__ void __launch_bounds__(256) k_mm(int M, int N, int K, const float* __restrict__ A, int lda,
                                            const BT* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                            const float* __restrict__ bias, int relu, const float* __restrict__ mask,
                                            float beta) {
  __shared__ float sA[16][65];
  __shared__ float sB[16][65];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = threadIdx.x; i < 64 * 16; i += 256) {
      int r = i / 16, c = i % 16;   // r: m or n within tile, c: k within chunk
      int gm = m0 + r, gk = k0 + c;
      float av = 0.f;
      if (gm < M && gk < K) av = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      sA[c][r] = av;
      int gn = n0 + r;
      float bv = 0.f;
      if (gn < N && gk < K) bv = (float)(TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]);
      sB[c][r] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) {
        float v = acc[i][j] + (bias ? bias[n] : 0.f);
        if (relu) v = fmaxf(v, 0.f);
        if (mask && mask[(size_t)m * ldc + n] <= 0.f) v = 0.f;
        float* p = C + (size_t)m * ldc + n;
        *p = (beta == 0.f) ? v : v + beta * *p;
      }
    }
}

// column sums: out[n] = sum_m A[m][n]
__global__ void k_colsum(const float* __restrict__ A, int M, int N, float* __restrict__ out) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += A[(size_t)m * N + n];
  out[n] = s;
}

// dY = 2 (Y - T) / (rows * nout), loss partial sums
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                      long long n, float scale, double* __restrict__ loss) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float d = Y[i] - T[i];
    dY[i] = 2.f * d * scale;
    s += (double)d * d;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(loss, t);
  }
}

__global__ void k_adam(float* P, const float* G, float* Mm, float* Vv, __nv_bfloat16* Ph, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float g = G[i];
  float m = b1 * Mm[i] + (1.f - b1) * g;
  float v = b2 * Vv[i] + (1.f - b2) * g * g;
  Mm[i] = m;
  Vv[i] = v;
  float p = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
  P[i] = p;
  Ph[i] = __float2bfloat16(p);
}

__global__ void k_to_bf16(const float* P, __nv_bfloat16* Ph, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) Ph[i] = __float2bfloat16(P[i]);
}

// per face: normalised inputs [r_f/|r_f|, z0_f/|z0_f|], |z0_f|, and (when recording)
// the target (e_f - z0_f)/|z0_f|
__global__ void k_face_samples(const double* __restrict__ r, const double* __restrict__ e,
                               const double* __restrict__ z0, float* __restrict__ X, float* __restrict__ T,
                               double* __restrict__ nrm, int nfb, int nin, int nout, const int* __restrict__ nbr,
                               int nnb) {
  __shared__ double red[2][8];
  const int f = blockIdx.x;
  const double* rf = r + (size_t)f * nfb;
  const double* zf = z0 + (size_t)f * nfb;
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < nfb; i += blockDim.x) {
    s += rf[i] * rf[i];
    t += zf[i] * zf[i];
  }
  for (int o = 16; o; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = t;
  }
  __syncthreads();
  double sr = 0.0, sz = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    sr += red[0][w];
    sz += red[1][w];
  }
  const double ir = sr > 0.0 ? 1.0 / sqrt(sr) : 0.0;
  const double nz = sqrt(sz);
  const double iz = nz > 0.0 ? 1.0 / nz : 0.0;
  if (threadIdx.x == 0 && nrm) nrm[f] = nz;
  for (int i = threadIdx.x; i < nin; i += blockDim.x) {
    float v = 0.f;
    const int part = i / nout, j = i % nout;
    if (j < nfb) {
      if (part == 0) v = (float)(rf[j] * ir);
      else if (part == 1) v = (float)(zf[j] * iz);
      else {
        const int g = nbr[(size_t)f * nnb + part - 2];
        if (g >= 0) v = (float)(z0[(size_t)g * nfb + j] * iz);
      }
    }
    X[(size_t)f * nin + i] = v;
  }
  if (T)
    for (int i = threadIdx.x; i < nout; i += blockDim.x)
      T[(size_t)f * nout + i] = i < nfb ? (float)((e[(size_t)f * nfb + i] - zf[i]) * iz) : 0.f;
}

// z_f += |z0_f| y_f
__global__ void k_face_correct(const float* __restrict__ Y, const double* __restrict__ nrm, double* __restrict__ z,
                               int nfb, int nout, int F) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)F * nfb) return;
  int f = (int)(i / nfb), j = (int)(i % nfb);
  z[i] += nrm[f] * (double)Y[(size_t)f * nout + j];
}

Mlp* M_(mehdg_ctx* ctx) { return static_cast<Mlp*>(ctx->mlp); }

template <class BT, bool TA, bool TB>
int mm(mehdg_ctx* ctx, int M, int N, int K, const float* A, int lda, const BT* B, int ldb, float* C, int ldc,
       const float* bias, int relu, const float* mask, float beta) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_mm<BT, TA, TB><<<grid, 256, 0, ctx->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, mask, beta);
  CKL();
  return MEHDG_OK;
}

// forward of n rows of X (device) into m->H1, H2, Y
int forward(mehdg_ctx* ctx, const float* X, int n) {
  Mlp* m = M_(ctx);
  int rc;
  if ((rc = mm<__nv_bfloat16, false, true>(ctx, n, m->nh, m->nin, X, m->nin, m->Ph + m->oW1, m->nin, m->H1, m->nh,
                                           m->P + m->ob1, 1, nullptr, 0.f)))
    return rc;
  if ((rc = mm<__nv_bfloat16, false, true>(ctx, n, m->nh, m->nh, m->H1, m->nh, m->Ph + m->oW2, m->nh, m->H2, m->nh,
                                           m->P + m->ob2, 1, nullptr, 0.f)))
    return rc;
  return mm<__nv_bfloat16, false, true>(ctx, n, m->nout, m->nh, m->H2, m->nh, m->Ph + m->oW3, m->nh, m->Y, m->nout,
                                        m->P + m->ob3, 0, nullptr, 0.f);
}

// loss and gradient (into m->G) for n rows of X and T; loss returned on the host
int loss_grad(mehdg_ctx* ctx, const float* X, const float* T, int n, double* loss) {
  Mlp* m = M_(ctx);
  int rc;
  if ((rc = forward(ctx, X, n))) return rc;
  CK(cudaMemsetAsync(m->dloss, 0, sizeof(double), ctx->stream));
  long long ny = (long long)n * m->nout;
  k_mse<<<256, 256, 0, ctx->stream>>>(m->Y, T, m->dY, ny, 1.f / (float)ny, m->dloss);
  CKL();
  // W3, b3
  if ((rc = mm<float, true, false>(ctx, m->nout, m->nh, n, m->dY, m->nout, m->H2, m->nh, m->G + m->oW3, m->nh,
                                   nullptr, 0, nullptr, 0.f)))
    return rc;
  k_colsum<<<(m->nout + 127) / 128, 128, 0, ctx->stream>>>(m->dY, n, m->nout, m->G + m->ob3);
  CKL();
  // dH2 = (dY W3) o [H2 > 0]
  if ((rc = mm<__nv_bfloat16, false, false>(ctx, n, m->nh, m->nout, m->dY, m->nout, m->Ph + m->oW3, m->nh, m->dH2,
                                            m->nh, nullptr, 0, m->H2, 0.f)))
    return rc;
  if ((rc = mm<float, true, false>(ctx, m->nh, m->nh, n, m->dH2, m->nh, m->H1, m->nh, m->G + m->oW2, m->nh, nullptr,
                                   0, nullptr, 0.f)))
    return rc;
  k_colsum<<<(m->nh + 127) / 128, 128, 0, ctx->stream>>>(m->dH2, n, m->nh, m->G + m->ob2);
  CKL();
  if ((rc = mm<__nv_bfloat16, false, false>(ctx, n, m->nh, m->nh, m->dH2, m->nh, m->Ph + m->oW2, m->nh, m->dH1,
                                            m->nh, nullptr, 0, m->H1, 0.f)))
    return rc;
  if ((rc = mm<float, true, false>(ctx, m->nh, m->nin, n, m->dH1, m->nh, X, m->nin, m->G + m->oW1, m->nin, nullptr,
                                   0, nullptr, 0.f)))
    return rc;
  k_colsum<<<(m->nh + 127) / 128, 128, 0, ctx->stream>>>(m->dH1, n, m->nh, m->G + m->ob1);
  CKL();
  if (loss) {
    CK(cudaMemcpyAsync(loss, m->dloss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *loss /= (double)ny;
  }
  return MEHDG_OK;
}

// deterministic He-uniform initialisation from a 64-bit LCG
void init_params(std::vector<float>& p, const Mlp& m, unsigned long long seed) {
  unsigned long long s = seed * 6364136223846793005ULL + 1442695040888963407ULL;
  auto uni = [&]() {
    s = s * 6364136223846793005ULL + 1442695040888963407ULL;
    return ((s >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
  };
  std::fill(p.begin(), p.end(), 0.f);
  auto fill = [&](long long off, long long n, int fan_in) {
    double a = std::sqrt(6.0 / fan_in);
    for (long long i = 0; i < n; ++i) p[off + i] = (float)(a * uni());
  };
  fill(m.oW1, (long long)m.nh * m.nin, m.nin);
  fill(m.oW2, (long long)m.nh * m.nh, m.nh);
  fill(m.oW3, (long long)m.nout * m.nh, m.nh);
  // the last layer starts small so that the untrained correction is close to zero
  for (long long i = 0; i < (long long)m.nout * m.nh; ++i) p[m.oW3 + i] *= 0.01f;
}

}  // namespace

int mlp_apply(mehdg_ctx* ctx, const double* r, double* z) {
  Mlp* m = M_(ctx);
  if (!m) return ctx_fail(ctx, MEHDG_ERR_ARG, "preconditioner kind 2 needs mehdg_mlp_setup");
  k_face_samples<<<m->F, 256, 0, ctx->stream>>>(r, nullptr, z, m->Xin, nullptr, m->nrm, m->nfb, m->nin, m->nout,
                                                m->nbr, m->nnb);
  CKL();
  int rc;
  if ((rc = forward(ctx, m->Xin, m->F))) return rc;
  long long tot = (long long)m->F * m->nfb;
  k_face_correct<<<(tot + 255) / 256, 256, 0, ctx->stream>>>(m->Y, m->nrm, z, m->nfb, m->nout, m->F);
  CKL();
  return MEHDG_OK;
}

bool mlp_recording(const mehdg_ctx* ctx) {
  const Mlp* m = static_cast<const Mlp*>(ctx->mlp);
  return m && m->recording && m->count + m->F <= m->cap;
}

// one (residual, error) pair of global trace vectors -> F samples
int mlp_record_pair(mehdg_ctx* ctx, const double* r, const double* e) {
  Mlp* m = M_(ctx);
  if (!m) return ctx_fail(ctx, MEHDG_ERR_ARG, "mehdg_mlp_setup first");
  if (m->count + m->F > m->cap) return MEHDG_OK;   // buffer full: keep the first pairs
  int rc;
  double* z0 = ctx->iw;   // block-Jacobi output of r (scratch of the inner GMRES, idle here)
  if ((rc = precond_impl(ctx, 0, r, z0))) return rc;
  k_face_samples<<<m->F, 256, 0, ctx->stream>>>(r, e, z0, m->X + (size_t)m->count * m->nin,
                                                m->T + (size_t)m->count * m->nout, nullptr, m->nfb, m->nin, m->nout,
                                                m->nbr, m->nnb);
  CKL();
  m->count += m->F;
  return MEHDG_OK;
}

extern "C" int mehdg_mlp_setup(mehdg_ctx* ctx, int hidden, unsigned long long seed, int max_pairs, int neighbors) {
  if (!ctx || hidden < 32 || hidden > 4096 || max_pairs < 1) return MEHDG_ERR_ARG;
  if (ctx->mlp) return ctx_fail(ctx, MEHDG_ERR_ARG, "MLP already set up");
  Mlp* m = new Mlp();
  m->nfb = ctx->nfb;
  m->F = ctx->F;
  m->nout = ((ctx->nfb + 31) / 32) * 32;
  // the other faces of the face's (one or two) owner macro-elements, from the owner and
  // gather maps: owner o of face f is (e, fl), face fl' of e is gather[e][fl' Nfn] / (ns Nfn)
  std::vector<int> nbr;
  if (neighbors) {
    const int nf = ctx->nf;
    m->nnb = 2 * (nf - 1);
    nbr.assign((size_t)ctx->F * m->nnb, -1);
    for (int f = 0; f < ctx->F; ++f) {
      int k = 0;
      for (int o = 0; o < 2; ++o) {
        const int ow = ctx->h_owner[2 * f + o];
        if (ow < 0) { k += nf - 1; continue; }
        const int e = ow / nf, fl = ow % nf;
        for (int g = 0; g < nf; ++g) {
          if (g == fl) continue;
          nbr[(size_t)f * m->nnb + k++] = ctx->h_gather[(size_t)e * ctx->Nt + (size_t)g * ctx->Nfn] / (ctx->ns * ctx->Nfn);
        }
      }
    }
  }
  m->nin = (2 + m->nnb) * m->nout;
  m->nh = hidden;
  m->oW1 = 0;
  m->ob1 = m->oW1 + (long long)m->nh * m->nin;
  m->oW2 = m->ob1 + m->nh;
  m->ob2 = m->oW2 + (long long)m->nh * m->nh;
  m->oW3 = m->ob2 + m->nh;
  m->ob3 = m->oW3 + (long long)m->nout * m->nh;
  m->np = m->ob3 + m->nout;
  m->cap = max_pairs * m->F;
  m->wcap = std::max(m->F, 8192);
  ctx->mlp = m;
  auto al = [&](void** p, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return ctx_fail(ctx, MEHDG_ERR_OOM, "MLP allocation failed");
    ctx->bytes += bytes;
    return 0;
  };
  int rc = 0;
  rc |= al((void**)&m->P, sizeof(float) * m->np);
  rc |= al((void**)&m->G, sizeof(float) * m->np);
  rc |= al((void**)&m->Mm, sizeof(float) * m->np);
  rc |= al((void**)&m->Vv, sizeof(float) * m->np);
  rc |= al((void**)&m->Ph, sizeof(__nv_bfloat16) * m->np);
  rc |= al((void**)&m->X, sizeof(float) * (size_t)m->cap * m->nin);
  rc |= al((void**)&m->T, sizeof(float) * (size_t)m->cap * m->nout);
  rc |= al((void**)&m->H1, sizeof(float) * (size_t)m->wcap * m->nh);
  rc |= al((void**)&m->H2, sizeof(float) * (size_t)m->wcap * m->nh);
  rc |= al((void**)&m->dH1, sizeof(float) * (size_t)m->wcap * m->nh);
  rc |= al((void**)&m->dH2, sizeof(float) * (size_t)m->wcap * m->nh);
  rc |= al((void**)&m->Y, sizeof(float) * (size_t)m->wcap * m->nout);
  rc |= al((void**)&m->dY, sizeof(float) * (size_t)m->wcap * m->nout);
  rc |= al((void**)&m->Xin, sizeof(float) * (size_t)m->F * m->nin);
  rc |= al((void**)&m->nrm, sizeof(double) * m->F);
  rc |= al((void**)&m->dloss, sizeof(double));
  if (m->nnb) rc |= al((void**)&m->nbr, sizeof(int) * nbr.size());
  if (rc) return rc;
  if (m->nnb) CK(cudaMemcpy(m->nbr, nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice));
  std::vector<float> p(m->np);
  init_params(p, *m, seed);
  CK(cudaMemcpy(m->P, p.data(), sizeof(float) * m->np, cudaMemcpyHostToDevice));
  CK(cudaMemset(m->Mm, 0, sizeof(float) * m->np));
  CK(cudaMemset(m->Vv, 0, sizeof(float) * m->np));
  k_to_bf16<<<(m->np + 255) / 256, 256, 0, ctx->stream>>>(m->P, m->Ph, m->np);
  CKL();
  CK(cudaStreamSynchronize(ctx->stream));
  return MEHDG_OK;
}

extern "C" int mehdg_mlp_params(mehdg_ctx* ctx, int set, float* host, long long* count) {
  if (!ctx || !ctx->mlp) return MEHDG_ERR_ARG;
  Mlp* m = M_(ctx);
  if (count) *count = m->np;
  if (!host) return MEHDG_OK;
  if (set) {
    CK(cudaMemcpy(m->P, host, sizeof(float) * m->np, cudaMemcpyHostToDevice));
    k_to_bf16<<<(m->np + 255) / 256, 256, 0, ctx->stream>>>(m->P, m->Ph, m->np);
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(host, m->P, sizeof(float) * m->np, cudaMemcpyDeviceToHost));
  }
  return MEHDG_OK;
}

extern "C" int mehdg_mlp_record(mehdg_ctx* ctx, const double* r, const double* e) {
  if (!ctx || !r || !e) return MEHDG_ERR_ARG;
  return mlp_record_pair(ctx, r, e);
}

extern "C" int mehdg_mlp_set_recording(mehdg_ctx* ctx, int on, int* count) {
  if (!ctx || !ctx->mlp) return MEHDG_ERR_ARG;
  Mlp* m = M_(ctx);
  m->recording = on != 0;
  if (count) *count = m->count;
  return MEHDG_OK;
}

extern "C" int mehdg_mlp_gradient(mehdg_ctx* ctx, const float* X, const float* T, int n, float* grad, double* loss) {
  if (!ctx || !ctx->mlp || !X || !T || n < 1) return MEHDG_ERR_ARG;
  Mlp* m = M_(ctx);
  if (n > m->wcap) return ctx_fail(ctx, MEHDG_ERR_ARG, "too many rows for the MLP work buffers");
  int rc = loss_grad(ctx, X, T, n, loss);
  if (rc) return rc;
  if (grad) {
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(grad, m->G, sizeof(float) * m->np, cudaMemcpyDeviceToHost));
  }
  return MEHDG_OK;
}

extern "C" int mehdg_mlp_train(mehdg_ctx* ctx, int epochs, int batch, double lr, double* losses) {
  if (!ctx || !ctx->mlp || epochs < 1 || batch < 1) return MEHDG_ERR_ARG;
  Mlp* m = M_(ctx);
  if (m->count == 0) return ctx_fail(ctx, MEHDG_ERR_ARG, "no recorded training pairs");
  batch = std::min(batch, m->wcap);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  double first = 0.0, last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    double eloss = 0.0;
    int nb = 0;
    for (int s0 = 0; s0 < m->count; s0 += batch) {
      const int n = std::min(batch, m->count - s0);
      double l;
      int rc = loss_grad(ctx, m->X + (size_t)s0 * m->nin, m->T + (size_t)s0 * m->nout, n, &l);
      if (rc) return rc;
      ++m->step;
      const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
      k_adam<<<(m->np + 255) / 256, 256, 0, ctx->stream>>>(m->P, m->G, m->Mm, m->Vv, m->Ph, m->np, (float)lr, b1, b2,
                                                           eps, c1, c2);
      CKL();
      eloss += l;
      ++nb;
    }
    eloss /= nb;
    if (ep == 0) first = eloss;
    last = eloss;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  m->trained = true;
  if (losses) {
    losses[0] = first;
    losses[1] = last;
  }
  return MEHDG_OK;
}

void mlp_destroy(mehdg_ctx* ctx) {
  Mlp* m = M_(ctx);
  if (!m) return;
  void* ptrs[] = {m->P, m->G, m->Mm, m->Vv, m->Ph, m->X, m->T, m->H1, m->H2, m->dH1, m->dH2, m->Y, m->dY, m->Xin,
                  m->nrm, m->dloss, m->nbr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
  ctx->mlp = nullptr;
}
