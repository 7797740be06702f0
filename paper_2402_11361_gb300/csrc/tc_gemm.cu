// Host side of the tcgen05 TF32 batched GEMM (kernel in tc_gemm.cuh) and its C entry
// point for callers and tests.
#include "internal.cuh"
#include "tc_gemm.cuh"

template <int BN, bool SPLIT>
static cudaError_t launch_bn(const TcArgs& a, int batch, cudaStream_t st) {
  size_t smem = tc_gemm_smem<BN, SPLIT>();
  cudaError_t e =
      cudaFuncSetAttribute(k_tc_gemm_tf32<BN, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.N + BN - 1) / BN, (a.M + 127) / 128, batch);
  k_tc_gemm_tf32<BN, SPLIT><<<grid, 128, smem, st>>>(a);
  return cudaGetLastError();
}

// N tile: 128 for N <= 128, 160 for N in (128, 160] (the trace blocks of p = 2), 256 otherwise.
// split: three TF32 products of the hi/lo parts (about FP32 accuracy).
cudaError_t tc_gemm_launch(const TcArgs& a, int batch, cudaStream_t st, bool split) {
  if (split) {
    if (a.N <= 128) return launch_bn<128, true>(a, batch, st);
    if (a.N <= 160) return launch_bn<160, true>(a, batch, st);
    return launch_bn<256, true>(a, batch, st);
  }
  if (a.N <= 128) return launch_bn<128, false>(a, batch, st);
  if (a.N <= 160) return launch_bn<160, false>(a, batch, st);
  return launch_bn<256, false>(a, batch, st);
}

extern "C" int mehdg_tc_gemm_tf32(int M, int N, int K, const float* A, long long lda, long long sA,
                                  const float* B, long long ldb, long long sB, float* C, long long ldc, long long sC,
                                  float alpha, float beta, int batch, int split, int* err, void* stream) {
  if (M < 1 || N < 1 || K < 1 || batch < 1 || batch > 65535 || !A || !B || !C || !err) return MEHDG_ERR_ARG;
  TcArgs a{};
  a.M = M; a.N = N; a.K = K;
  a.A = A; a.lda = lda; a.sA1 = sA; a.sA2 = 0;
  a.B = B; a.ldb = ldb; a.sB1 = sB; a.sB2 = 0;
  a.C = C; a.ldc = ldc; a.sC1 = sC; a.sC2 = 0;
  a.alpha = alpha; a.beta = beta; a.n2 = 1; a.err = err;
  return tc_gemm_launch(a, batch, static_cast<cudaStream_t>(stream), split != 0) == cudaSuccess ? MEHDG_OK
                                                                                                 : MEHDG_ERR_CUDA;
}

template <int BN>
static cudaError_t launch_nt(const TcNT& a, int batch, cudaStream_t st) {
  const size_t smem = tc_nt_smem<BN>();
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm_nt<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.N + BN - 1) / BN, (a.M + 127) / 128, batch);
  k_tc_gemm_nt<BN><<<grid, TCNT_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

// N tile 128 for N <= 128, else 256 (A^T_i: N = Nt = 750 -> 3 tiles)
cudaError_t tc_gemm_nt_launch(const TcNT& a, int batch, cudaStream_t st) {
  return a.N <= 128 ? launch_nt<128>(a, batch, st) : launch_nt<256>(a, batch, st);
}

extern "C" int mehdg_tc_gemm_nt(int M, int N, int K, const float* A, long long lda, long long sA, const float* Bt,
                                long long ldb, long long sB, float* C, long long ldc, long long sC, float alpha,
                                float beta, int batch, int* err, void* stream) {
  if (M < 1 || N < 1 || K < 1 || batch < 1 || batch > 65535 || !A || !Bt || !C || !err) return MEHDG_ERR_ARG;
  TcNT a{};
  a.M = M; a.N = N; a.K = K;
  a.A = A; a.lda = lda; a.sA = sA;
  a.Bt = Bt; a.ldb = ldb; a.sB = sB;
  a.C = C; a.ldc = ldc; a.sC = sC;
  a.alpha = alpha; a.beta = beta; a.err = err;
  return tc_gemm_nt_launch(a, batch, static_cast<cudaStream_t>(stream)) == cudaSuccess ? MEHDG_OK : MEHDG_ERR_CUDA;
}
