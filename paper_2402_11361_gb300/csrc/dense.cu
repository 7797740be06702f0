// a3-a6: second-layer static condensation (eqs. AP12, ASC2), batched dense LU of the
// Schur complements S (Remark, Sec. 3.3) and the condensed right-hand side
// (Algorithm 1, lines 2-5), FP64.
//
//   S = A_uu + shift (I (x) M) - sum_k A_uq_k (I (x) W_k)       W_k  = M^-1 G_k
//   C = -A_uuh + sum_k A_uq_k (I (x) Wh_k)                     Wh_k = M^-1 Gh_k
//   B = A_uhu - sum_k A_uhq_k (I (x) W_k)
//   D = A_uhuh - sum_k A_uhq_k (I (x) Wh_k)
//   g = -R_U + sum_k A_uq_k (I (x) M^-1) R_Q,k,   h = -R_Uh + sum_k A_uhq_k (I (x) M^-1) R_Q,k
//   P S = L U,  b^_i = h - B S^-1 g
// S, C, B, D overwrite A_uu, A_uuh, A_uhu, A_uhuh in place.
#include <algorithm>

#include "internal.cuh"
#include "lu.cuh"

namespace {

// C[b] = alpha A[b] B[b] + beta C[b], row-major, batch b = (i, j), i < n1 (outer), j < n2:
// X[b] = X + i * sX1 + j * sX2.
struct GemmArgs {
  int M, N, K;
  const double* A; int lda; long long sA1, sA2;
  const double* B; int ldb; long long sB1, sB2;
  double* C; int ldc; long long sC1, sC2;
  double alpha, beta;
  int n2;
};

constexpr int TM = 64, TN = 64, TK = 16;
__global__ void __launch_bounds__(256) k_gemm64(GemmArgs a) {
  __shared__ double sA[TK][TM + 1];
  __shared__ double sB[TK][TN + 1];
  const int b = blockIdx.z;
  const int bi = b / a.n2, bj = b % a.n2;
  const double* A = a.A + bi * a.sA1 + bj * a.sA2;
  const double* B = a.B + bi * a.sB1 + bj * a.sB2;
  double* C = a.C + bi * a.sC1 + bj * a.sC2;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < a.K; k0 += TK) {
    for (int i = threadIdx.x; i < TM * TK; i += 256) {
      int r = i / TK, c = i % TK;
      int gr = m0 + r, gc = k0 + c;
      sA[c][r] = (gr < a.M && gc < a.K) ? A[(size_t)gr * a.lda + gc] : 0.0;
    }
    for (int i = threadIdx.x; i < TK * TN; i += 256) {
      int r = i / TN, c = i % TN;
      int gr = k0 + r, gc = n0 + c;
      sB[r][c] = (gr < a.K && gc < a.N) ? B[(size_t)gr * a.ldb + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = sA[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = sB[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
      if (r < a.M && c < a.N) {
        double* p = C + (size_t)r * a.ldc + c;
        *p = a.alpha * acc[i][j] + (a.beta == 0.0 ? 0.0 : a.beta * *p);
      }
    }
}

int gemm(mehdg_ctx* ctx, const GemmArgs& a, int n1) {
  dim3 grid((a.N + TN - 1) / TN, (a.M + TM - 1) / TM, n1 * a.n2);
  k_gemm64<<<grid, 256, 0, ctx->stream>>>(a);
  CKL();
  return MEHDG_OK;
}

// y[b] = alpha A[b] x[b] + beta y[b]; one warp per row
struct GemvArgs {
  int M, N;
  const double* A; int lda; long long sA1, sA2;
  const double* x; long long sx1, sx2;
  double* y; long long sy1, sy2;
  double alpha, beta;
  int n2;
};
__global__ void k_gemv(GemvArgs a) {
  const int b = blockIdx.y;
  const int bi = b / a.n2, bj = b % a.n2;
  const double* A = a.A + bi * a.sA1 + bj * a.sA2;
  const double* x = a.x + bi * a.sx1 + bj * a.sx2;
  double* y = a.y + bi * a.sy1 + bj * a.sy2;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (row >= a.M) return;
  double s = 0.0;
  for (int c = lane; c < a.N; c += 32) s += A[(size_t)row * a.lda + c] * x[c];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = a.alpha * s + (a.beta == 0.0 ? 0.0 : a.beta * y[row]);
}
int gemv(mehdg_ctx* ctx, const GemvArgs& a, int n1) {
  dim3 grid((a.M + 7) / 8, n1 * a.n2);
  k_gemv<<<grid, 256, 0, ctx->stream>>>(a);
  CKL();
  return MEHDG_OK;
}

__global__ void k_scale(double* x, long long n, double a) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) x[i] *= a;
}

// S[(s,a)][(s,b)] += shift M[a][b]
__global__ void k_mass_shift(double* S, const double* M, int Np, int ns, double shift, int E) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)E * ns * Np * Np;
  if (i >= tot) return;
  int b = i % Np;
  int a = (i / Np) % Np;
  int s = (i / ((long long)Np * Np)) % ns;
  int e = (int)(i / ((long long)Np * Np * ns));
  size_t Nu = (size_t)ns * Np;
  S[(size_t)e * Nu * Nu + ((size_t)s * Np + a) * Nu + (size_t)s * Np + b] += shift * M[(size_t)a * Np + b];
}

// MinvRQ[e][k][s] = M^-1 R_Q[e][k][s]
__global__ void k_minv_rq(const double* Minv, const double* RQ, double* out, int Np, long long nvec) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nvec * Np) return;
  int a = i % Np;
  long long v = i / Np;
  const double* r = RQ + v * Np;
  const double* m = Minv + (size_t)a * Np;
  double s = 0.0;
  for (int b = 0; b < Np; ++b) s += m[b] * r[b];
  out[i] = s;
}

// face blocks of A_uhuh: sum of the owners' local blocks (before D overwrites A_uhuh)
__global__ void k_face_blocks(const double* Ahh, const int* owner, double* fblk, int ns, int Nfn, int Nth,
                              int Nt, int d, int F) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int nfb = ns * Nfn;
  if (i >= (long long)F * nfb * nfb) return;
  int c = i % nfb;
  int r = (i / nfb) % nfb;
  int f = (int)(i / ((long long)nfb * nfb));
  int sr = r / Nfn, jr = r % Nfn, sc = c / Nfn, jc = c % Nfn;
  double v = 0.0;
  for (int o = 0; o < 2; ++o) {
    int ow = owner[2 * f + o];
    if (ow < 0) continue;
    int e = ow / (2 * d), fl = ow % (2 * d);
    v += Ahh[(size_t)e * Nt * Nt + ((size_t)sr * Nth + fl * Nfn + jr) * Nt + (size_t)sc * Nth + fl * Nfn + jc];
  }
  fblk[i] = v;
}

// b_loc = h - B S^-1 g, one CTA per macro-element
__global__ void __launch_bounds__(256) k_bhat_local(const double* S, const int* perm, const double* B,
                                                     const double* gvec, const double* hvec, double* bloc, int Nu,
                                                     int Nt) {
  extern __shared__ double sm[];
  double* y = sm;        // Nu
  double* tmp = sm + Nu; // Nu
  const int e = blockIdx.x;
  const double* Se = S + (size_t)e * Nu * Nu;
  const int* pe = perm + (size_t)e * Nu;
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) tmp[i] = gvec[(size_t)e * Nu + i];
  __syncthreads();
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) y[i] = tmp[pe[i]];
  __syncthreads();
  lu_solve_block<double>(Se, Nu, y);
  const double* Be = B + (size_t)e * Nt * Nu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = w; r < Nt; r += nw) {
    double s = 0.0;
    for (int c = lane; c < Nu; c += 32) s += Be[(size_t)r * Nu + c] * y[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) bloc[(size_t)e * Nt + r] = hvec[(size_t)e * Nt + r] - s;
  }
}

}  // namespace

int batched_lu(mehdg_ctx* ctx, double* A, int* perm, int n, int batch, int* flag) {
  size_t smem = lu_smem_bytes<double>(n);
  CK(cudaFuncSetAttribute(k_lu_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_lu_batched<double><<<batch, LU_NT, smem, ctx->stream>>>(A, perm, n, flag);
  CKL();
  return MEHDG_OK;
}

int condense_all(mehdg_ctx* ctx, double shift, double* bhat) {
  cudaStream_t st = ctx->stream;
  const int E = ctx->E, d = ctx->d, ns = ctx->ns, Np = ctx->Np, Nth = ctx->Nth;
  const long long Nu = ctx->Nu, Nt = ctx->Nt;
  int rc;
  // face blocks of A_uhuh for the preconditioner, then their LU
  {
    long long tot = (long long)ctx->F * ctx->nfb * ctx->nfb;
    k_face_blocks<<<(tot + 255) / 256, 256, 0, st>>>(ctx->Ahh, ctx->owner, ctx->fblk, ns, ctx->Nfn, Nth, (int)Nt, d,
                                                     ctx->F);
    CKL();
  }
  phase_begin(ctx, PH_CONDENSE);
  // M^-1 R_Q
  {
    long long nvec = (long long)E * d * ns;
    k_minv_rq<<<(nvec * Np + 255) / 256, 256, 0, st>>>(ctx->Minv, ctx->RQ, ctx->MinvRQ, Np, nvec);
    CKL();
  }
  // g = -R_U + sum_k A_uq_k[:, s] MinvRQ[k][s];  h = -R_Uh + sum_k A_uhq_k[:, s] MinvRQ[k][s]
  CK(cudaMemcpyAsync(ctx->gv, ctx->RU, sizeof(double) * E * Nu, cudaMemcpyDeviceToDevice, st));
  k_scale<<<(E * Nu + 255) / 256, 256, 0, st>>>(ctx->gv, E * Nu, -1.0);
  CK(cudaMemcpyAsync(ctx->hv, ctx->RUh, sizeof(double) * E * Nt, cudaMemcpyDeviceToDevice, st));
  k_scale<<<(E * Nt + 255) / 256, 256, 0, st>>>(ctx->hv, E * Nt, -1.0);
  CKL();
  for (int k = 0; k < d; ++k)
    for (int s = 0; s < ns; ++s) {
      GemvArgs a{};
      a.M = (int)Nu; a.N = Np;
      a.A = ctx->Auq + (size_t)k * Nu * Nu + (size_t)s * Np; a.lda = (int)Nu; a.sA1 = d * Nu * Nu; a.sA2 = 0;
      a.x = ctx->MinvRQ + ((size_t)k * ns + s) * Np; a.sx1 = (long long)d * Nu; a.sx2 = 0;
      a.y = ctx->gv; a.sy1 = Nu; a.sy2 = 0;
      a.alpha = 1.0; a.beta = 1.0; a.n2 = 1;
      if ((rc = gemv(ctx, a, E))) return rc;
      a.M = (int)Nt;
      a.A = ctx->Ahq + (size_t)k * Nt * Nu + (size_t)s * Np; a.sA1 = d * Nt * Nu;
      a.y = ctx->hv; a.sy1 = Nt;
      if ((rc = gemv(ctx, a, E))) return rc;
    }
  // S, C, B, D
  if (shift != 0.0) {
    long long tot = (long long)E * ns * Np * Np;
    k_mass_shift<<<(tot + 255) / 256, 256, 0, st>>>(ctx->Auu, ctx->Mref, Np, ns, shift, E);
    CKL();
  }
  k_scale<<<(E * Nu * Nt + 255) / 256, 256, 0, st>>>(ctx->Auh, E * Nu * Nt, -1.0);
  CKL();
  for (int k = 0; k < d; ++k) {
    GemmArgs a{};
    a.n2 = ns;
    a.alpha = -1.0; a.beta = 1.0;
    // S[:, s blk] -= A_uq_k[:, s blk] W_k
    a.M = (int)Nu; a.N = Np; a.K = Np;
    a.A = ctx->Auq + (size_t)k * Nu * Nu; a.lda = (int)Nu; a.sA1 = d * Nu * Nu; a.sA2 = Np;
    a.B = ctx->Wk + (size_t)k * Np * Np; a.ldb = Np; a.sB1 = 0; a.sB2 = 0;
    a.C = ctx->Auu; a.ldc = (int)Nu; a.sC1 = Nu * Nu; a.sC2 = Np;
    if ((rc = gemm(ctx, a, E))) return rc;
    // C[:, s trace blk] += A_uq_k[:, s blk] Wh_k
    a.alpha = 1.0;
    a.N = Nth;
    a.B = ctx->Whk + (size_t)k * Np * Nth; a.ldb = Nth;
    a.C = ctx->Auh; a.ldc = (int)Nt; a.sC1 = Nu * Nt; a.sC2 = Nth;
    if ((rc = gemm(ctx, a, E))) return rc;
    // B[:, s blk] -= A_uhq_k[:, s blk] W_k
    a.alpha = -1.0;
    a.M = (int)Nt; a.N = Np;
    a.A = ctx->Ahq + (size_t)k * Nt * Nu; a.sA1 = d * Nt * Nu;
    a.B = ctx->Wk + (size_t)k * Np * Np; a.ldb = Np;
    a.C = ctx->Ahu; a.ldc = (int)Nu; a.sC1 = Nt * Nu; a.sC2 = Np;
    if ((rc = gemm(ctx, a, E))) return rc;
    // D[:, s trace blk] -= A_uhq_k[:, s blk] Wh_k
    a.N = Nth;
    a.B = ctx->Whk + (size_t)k * Np * Nth; a.ldb = Nth;
    a.C = ctx->Ahh; a.ldc = (int)Nt; a.sC1 = Nt * Nt; a.sC2 = Nth;
    if ((rc = gemm(ctx, a, E))) return rc;
  }
  phase_end(ctx, PH_CONDENSE);
  // LU of S and of the face blocks
  CK(cudaMemsetAsync(ctx->dflag, 0, sizeof(int) * 16, st));
  phase_begin(ctx, PH_LU);
  if ((rc = batched_lu(ctx, ctx->Auu, ctx->perm, (int)Nu, E, ctx->dflag))) return rc;
  phase_end(ctx, PH_LU);
  phase_begin(ctx, PH_FACE_LU);
  if ((rc = batched_lu(ctx, ctx->fblk, ctx->fperm, ctx->nfb, ctx->F, ctx->dflag + 2))) return rc;
  phase_end(ctx, PH_FACE_LU);
  // b^
  phase_begin(ctx, PH_BHAT);
  {
    size_t smem = sizeof(double) * 2 * Nu;
    CK(cudaFuncSetAttribute(k_bhat_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bhat_local<<<E, 256, smem, st>>>(ctx->Auu, ctx->perm, ctx->Ahu, ctx->gv, ctx->hv, ctx->bloc, (int)Nu, (int)Nt);
    CKL();
  }
  if (bhat) {
    if ((rc = face_reduce(ctx, ctx->bloc, bhat))) return rc;
  }
  phase_end(ctx, PH_BHAT);
  int flags[4];
  CK(cudaMemcpyAsync(flags, ctx->dflag, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->condensed = true;
  if (flags[0]) return ctx_fail(ctx, MEHDG_ERR_SINGULAR, "zero pivot in S of macro-element " + std::to_string(flags[1] - 1));
  if (flags[2]) return ctx_fail(ctx, MEHDG_ERR_SINGULAR, "zero pivot in the A_uhuh block of face " + std::to_string(flags[3] - 1));
  return MEHDG_OK;
}

extern "C" int mehdg_condense_factor(mehdg_ctx* ctx, double shift, double* bhat) {
  if (!ctx) return MEHDG_ERR_ARG;
  return condense_all(ctx, shift, bhat);
}
