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
#include <cstdio>

#include "internal.cuh"
#include <cuda_bf16.h>

#include "lu.cuh"
#include "lu_panel.cuh"
#include "tc_gemm.cuh"

namespace {

// Second-layer condensation products of one (macro e, species s) pair in one GEMM
// (eq. ASC2a with the lifting factorisation of Sec. 3.2), P = [A_.q_1[:, s] | ... |
// A_.q_d[:, s]] [W_1 | -Wh_1; ...; W_d | -Wh_d]:
//   S_s -= P[:, W part],  C_s -= P[:, Wh part]   (C = -A_uuh + sum A_uq Wh)
//   B_s -= P[:, W part],  D_s += P[:, Wh part]   (D = A_uhuh - sum A_uhq Wh).  K = d*Np concatenates the directions, so
// each output is read and written once; the right factor [W | -Wh] is shared by all
// macros.  Tile 128 x 96 x 16, 8 x 6 outputs per thread, next K tile prefetched into
// registers while the current one is multiplied.
// The same tiles serve the plain batched product D += B X of the explicit local
// operator (one "species" block, no column split).
template <class T>
struct CondArgs {
  const T* A; long long sAe, sAk, sAs; int lda, M, kdiv;   // A(e,s)[r][kk] = A + e sAe + s sAs + (kk/kdiv) sAk + r lda + kk%kdiv
  const T* Bc; long long sBe; int ldb;                      // B(e)[kk][c] = Bc + e sBe + kk ldb + c
  int N, K, ns;
  T* O1; long long sO1e, sO1s; int ldo1, o1_add;            // columns c < nsplit: O1 + e sO1e + s sO1s + r ldo1 + c
  T* O2; long long sO2e, sO2s; int ldo2, o2_add;            // columns c >= nsplit: O2 + ... + (c - nsplit)
  int nsplit;
};
constexpr int CG_BM = 128, CG_BN = 96, CG_BK = 16;
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_cond_gemm(CondArgs<T> a) {
  __shared__ __align__(16) T sA[CG_BK][CG_BM + 4];
  __shared__ __align__(16) T sB[CG_BK][CG_BN];
  const int es = blockIdx.z, e = es / a.ns, s = es % a.ns;
  const int m0 = blockIdx.y * CG_BM, n0 = blockIdx.x * CG_BN;
  const int tid = threadIdx.x, tm = tid / 16, tn = tid % 16;
  const T* Ae = a.A + e * a.sAe + s * a.sAs;
  const T* Be = a.Bc + e * a.sBe;
  constexpr int LA = CG_BM * CG_BK / 256, LB = CG_BK * CG_BN / 256;
  T ra[LA], rb[LB];
  // A moves in 4-row x 8-column patches per warp (lane: row ll / 8, column ll % 8): 32-byte
  // global segments, and one bank per lane in the transposed shared tile (row stride
  // BM + 4 = 4 mod 32 banks); the thread's column is the same for all its rows
  const int lw = tid >> 5, ll = tid & 31;
  const int a_kq = (lw & 1) * 8 + (ll & 7), a_r = (lw >> 1) * 4 + (ll >> 3);
  auto fetch = [&](int k0) {
    const int kk = k0 + a_kq;
    const int kdir = kk / a.kdiv;
    const T* Ak = Ae + kdir * a.sAk + (kk - kdir * a.kdiv);
#pragma unroll
    for (int j = 0; j < LA; ++j) {
      const int gr = m0 + a_r + 16 * j;
      ra[j] = (gr < a.M && kk < a.K) ? Ak[(size_t)gr * a.lda] : T(0);
    }
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      const int i = tid + 256 * j, r = i / CG_BN, c = i % CG_BN;
      const int kk = k0 + r, gc = n0 + c;
      rb[j] = (kk < a.K && gc < a.N) ? Be[(size_t)kk * a.ldb + gc] : T(0);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int j = 0; j < LA; ++j) sA[a_kq][a_r + 16 * j] = ra[j];
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      const int i = tid + 256 * j;
      sB[i / CG_BN][i % CG_BN] = rb[j];
    }
  };
  T acc[8][6];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) acc[i][j] = T(0);
  fetch(0);
  for (int k0 = 0; k0 < a.K; k0 += CG_BK) {
    stash();
    __syncthreads();
    if (k0 + CG_BK < a.K) fetch(k0 + CG_BK);
#pragma unroll
    for (int kk = 0; kk < CG_BK; ++kk) {
      T av[8], bv[6];
      if constexpr (sizeof(T) == 4) {
        // explicit vector loads: 8 consecutive A entries (16-byte aligned), 6 B entries
        // as three 8-byte pairs (the row of sB is 384 B, tn * 24 B is 8-byte aligned)
        const float4 a0 = *reinterpret_cast<const float4*>(&sA[kk][tm * 8]);
        const float4 a1 = *reinterpret_cast<const float4*>(&sA[kk][tm * 8 + 4]);
        av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
        av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
        const float2* b2 = reinterpret_cast<const float2*>(&sB[kk][tn * 6]);
        const float2 b0 = b2[0], b1 = b2[1], bb = b2[2];
        bv[0] = b0.x; bv[1] = b0.y; bv[2] = b1.x; bv[3] = b1.y; bv[4] = bb.x; bv[5] = bb.y;
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] = sA[kk][tm * 8 + i];
#pragma unroll
        for (int j = 0; j < 6; ++j) bv[j] = sB[kk][tn * 6 + j];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + tm * 8 + i;
    if (r >= a.M) continue;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int c = n0 + tn * 6 + j;
      if (c >= a.N) continue;
      if (c < a.nsplit) {
        T* p = a.O1 + e * a.sO1e + s * a.sO1s + (size_t)r * a.ldo1 + c;
        *p = a.o1_add ? *p + acc[i][j] : *p - acc[i][j];
      } else {
        T* p = a.O2 + e * a.sO2e + s * a.sO2s + (size_t)r * a.ldo2 + (c - a.nsplit);
        *p = a.o2_add ? *p + acc[i][j] : *p - acc[i][j];
      }
    }
  }
}

template <class T>
int cond_gemm(mehdg_ctx* ctx, const CondArgs<T>& a, int E) {
  dim3 grid((a.N + CG_BN - 1) / CG_BN, (a.M + CG_BM - 1) / CG_BM, (unsigned)(E * a.ns));
  k_cond_gemm<T><<<grid, 256, 0, ctx->stream>>>(a);
  CKL();
  return MEHDG_OK;
}


// Second-layer condensation on affine box macros (eqs. AP12, ASC2).  There M and G_k are
// Kronecker products of 1D mass and derivative matrices, so the liftings W_k = M^-1 G_k and
// Wh_k = M^-1 Gh_k are sparse: column l of W_k holds n1 = m p + 1 entries, on the axis-k line
// through node l, and column (f, i) of Wh_k holds n1 entries, on the line normal to face f
// through face node i (only the two faces normal to k).  Each output entry of
// A_.q_k (I (x) W_k) is therefore an n1-term sum: 15 multiply-adds per S or B entry and 5 per
// C or D entry for p = 2 (3D), against K = d Np = 375 for the dense product.  The work is then
// bound by streaming the blocks: one CTA takes one row of the stacked [A_uq; A_uhq] at a time
// (all directions, all species, staged in shared memory), writes the matching row of S and C
// (or B and D) in place, and adds the row's term of the right-hand side pieces g and h.  The
// pseudo-time shift (I (x) M) on A_uu and the sign of C = -A_uuh + ... are folded in.
__host__ __device__ constexpr int ipow_k(int b, int e) { return e <= 0 ? 1 : b * ipow_k(b, e - 1); }

template <class T>
struct CondK {
  const T* Auq; const T* Ahq;   // [E][d][Nu][Nu], [E][d][Nt][Nu]
  T* S; T* C; T* B; T* D;       // over A_uu [E][Nu][Nu], A_uuh [E][Nu][Nt], A_uhu [E][Nt][Nu], A_uhuh [E][Nt][Nt]
  const double* klift;          // [d][n1][n1], then [2d][n1]
  const int* fnode;             // [2d][Nfn] macro node of each face node
  const double* M;              // [Np][Np]
  double shift;
  const double* dshift;         // device copy of the shift (read instead of shift when set)
  const T* xq;                  // [E][d][Nu] M^-1 R_Q in the block precision
  const double* RU; const double* RUh;
  double* g; double* h;
  int E, d, n1, Np, Nfn, Nth, Nu, Nt;
};
constexpr int CK_NT = 128;
// D, N1 > 0: compile-time dimension and nodes per macro edge (divisions by constants);
// 0: taken from the arguments
template <class T, int D, int N1>
__global__ void __launch_bounds__(CK_NT) k_cond_kron(CondK<T> a) {
  extern __shared__ __align__(16) unsigned char ck_raw[];
  T* arow = reinterpret_cast<T*>(ck_raw);   // [d][Nu]: one row of A_uq_k (or A_uhq_k) for every k
  __shared__ T w1[3 * 64];
  __shared__ T wf[6 * 8];
  __shared__ double red[CK_NT / 32];
  const double shift = a.dshift ? *a.dshift : a.shift;
  const int tid = threadIdx.x;
  const int d = D ? D : a.d, n1 = N1 ? N1 : a.n1;
  const int Np = D && N1 ? ipow_k(N1, D) : a.Np;
  const int Nfn = D && N1 ? ipow_k(N1, D - 1) : a.Nfn;
  const int Nth = 2 * d * Nfn, Nu = (d + 2) * Np, Nt = (d + 2) * Nth;
  for (int i = tid; i < d * n1 * n1; i += CK_NT) w1[i] = (T)a.klift[i];
  for (int i = tid; i < 2 * d * n1; i += CK_NT) wf[i] = (T)a.klift[d * n1 * n1 + i];
  const int strides[3] = {1, n1, n1 * n1};
  const int rows = Nu + Nt;
  const long long total = (long long)a.E * rows;
  for (long long id = blockIdx.x; id < total; id += gridDim.x) {
    const int e = (int)(id / rows), r = (int)(id - (long long)e * rows);
    const bool top = r < Nu;
    const int rr = top ? r : r - Nu;
    const T* src = top ? a.Auq + (size_t)e * d * Nu * Nu + (size_t)rr * Nu
                       : a.Ahq + (size_t)e * d * Nt * Nu + (size_t)rr * Nu;
    const size_t sk = top ? (size_t)Nu * Nu : (size_t)Nt * Nu;
    __syncthreads();   // the previous row's readers are done
    for (int k = 0; k < d; ++k)
      for (int c = tid; c < Nu; c += CK_NT) arow[k * Nu + c] = src[k * sk + c];
    __syncthreads();
    // right-hand side piece: g_r = -R_U,r + sum_k A_uq_k[r] . xq_k (h from A_uhq and R_Uh);
    // per-thread partial sums in the block precision, reduced in FP64
    {
      const T* xq = a.xq + (size_t)e * d * Nu;
      T part = T(0);
      for (int c = tid; c < d * Nu; c += CK_NT) part += arow[c] * xq[c];
      double pd = (double)part;
      for (int o = 16; o; o >>= 1) pd += __shfl_xor_sync(0xffffffffu, pd, o);
      if ((tid & 31) == 0) red[tid >> 5] = pd;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < CK_NT / 32; ++w) t += red[w];
        if (top) a.g[(size_t)e * Nu + rr] = t - a.RU[(size_t)e * Nu + rr];
        else a.h[(size_t)e * Nt + rr] = t - a.RUh[(size_t)e * Nt + rr];
      }
    }
    // S row (A_uu + shift (I (x) M) - A_uq W) or B row (A_uhu - A_uhq W)
    T* o1 = top ? a.S + (size_t)e * Nu * Nu + (size_t)rr * Nu : a.B + (size_t)e * Nt * Nu + (size_t)rr * Nu;
    const int sr = top ? rr / Np : -1, lr = top ? rr - sr * Np : 0;
    for (int c = tid; c < Nu; c += CK_NT) {
      const int s = c / Np, l = c - s * Np;
      T acc = T(0);
      int rem = l;
#pragma unroll
      for (int k = 0; k < (D ? D : 3); ++k) {
        if (!D && k >= d) break;
        const int lk = rem % n1;
        rem /= n1;
        const T* ak = arow + k * Nu + c - lk * strides[k];
        const T* wk = w1 + k * n1 * n1 + lk;
#pragma unroll
        for (int q = 0; q < (N1 ? N1 : 8); ++q) {
          if (!N1 && q >= n1) break;
          acc += ak[q * strides[k]] * wk[q * n1];
        }
      }
      T v = o1[c] - acc;
      if (s == sr && shift != 0.0) v += (T)(shift * a.M[(size_t)lr * Np + l]);
      o1[c] = v;
    }
    // C row (-A_uuh + A_uq Wh) or D row (A_uhuh - A_uhq Wh): column (species, face, face node)
    T* o2 = top ? a.C + (size_t)e * Nu * Nt + (size_t)rr * Nt : a.D + (size_t)e * Nt * Nt + (size_t)rr * Nt;
    for (int c = tid; c < Nt; c += CK_NT) {
      const int s = c / Nth, rem = c - s * Nth, fl = rem / Nfn, i = rem - fl * Nfn, k = fl >> 1;
      const int l0 = a.fnode[fl * Nfn + i];
      const int lk = (l0 / strides[k]) % n1;
      const T* ak = arow + k * Nu + s * Np + l0 - lk * strides[k];
      const T* wk = wf + fl * n1;
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < (N1 ? N1 : 8); ++q) {
        if (!N1 && q >= n1) break;
        acc += ak[q * strides[k]] * wk[q];
      }
      o2[c] = top ? acc - o2[c] : o2[c] - acc;
    }
  }
}

template <class T, int D, int N1>
int cond_kron_launch(mehdg_ctx* ctx, const CondK<T>& a) {
  const size_t smem = sizeof(T) * (size_t)ctx->d * ctx->Nu;
  CK(cudaFuncSetAttribute(k_cond_kron<T, D, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0, per = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cond_kron<T, D, N1>, CK_NT, smem));
  const long long total = (long long)ctx->E * (ctx->Nu + ctx->Nt);
  const long long grid = std::min<long long>(total, (long long)nsm * std::max(per, 1));
  k_cond_kron<T, D, N1><<<(unsigned)grid, CK_NT, smem, ctx->stream>>>(a);
  CKL();
  return MEHDG_OK;
}

template <class T>
int cond_kron(mehdg_ctx* ctx, double shift, const T* xq) {
  CondK<T> a{};
  a.Auq = reinterpret_cast<const T*>(ctx->Auq);
  a.Ahq = reinterpret_cast<const T*>(ctx->Ahq);
  a.S = reinterpret_cast<T*>(ctx->Auu);
  a.C = reinterpret_cast<T*>(ctx->Auh);
  a.B = reinterpret_cast<T*>(ctx->Ahu);
  a.D = reinterpret_cast<T*>(ctx->Ahh);
  a.klift = ctx->klift; a.fnode = ctx->fnode; a.M = ctx->Mref; a.shift = shift; a.dshift = ctx->dshift; a.xq = xq;
  a.RU = ctx->RU; a.RUh = ctx->RUh; a.g = ctx->gv; a.h = ctx->hv;
  a.E = ctx->E; a.d = ctx->d; a.n1 = ctx->n1; a.Np = ctx->Np; a.Nfn = ctx->Nfn; a.Nth = ctx->Nth;
  a.Nu = ctx->Nu; a.Nt = ctx->Nt;
  const int key = ctx->d * 16 + ctx->n1;
  switch (key) {
    case 2 * 16 + 3: return cond_kron_launch<T, 2, 3>(ctx, a);
    case 2 * 16 + 5: return cond_kron_launch<T, 2, 5>(ctx, a);
    case 2 * 16 + 7: return cond_kron_launch<T, 2, 7>(ctx, a);
    case 3 * 16 + 3: return cond_kron_launch<T, 3, 3>(ctx, a);
    case 3 * 16 + 5: return cond_kron_launch<T, 3, 5>(ctx, a);
    case 3 * 16 + 7: return cond_kron_launch<T, 3, 7>(ctx, a);
    default: return cond_kron_launch<T, 0, 0>(ctx, a);
  }
}

// The same product on the tcgen05 tensor cores (TF32 inputs, FP32 accumulation)
int tc_gemm(mehdg_ctx* ctx, int M, int N, int K, const float* A, long long lda, long long sA1, long long sA2,
            const float* B, long long ldb, long long sB1, long long sB2, float* C, long long ldc, long long sC1,
            long long sC2, float alpha, float beta, int n1, int n2) {
  TcArgs a{};
  a.M = M; a.N = N; a.K = K;
  a.A = A; a.lda = lda; a.sA1 = sA1; a.sA2 = sA2;
  a.B = B; a.ldb = ldb; a.sB1 = sB1; a.sB2 = sB2;
  a.C = C; a.ldc = ldc; a.sC1 = sC1; a.sC2 = sC2;
  a.alpha = alpha; a.beta = beta; a.n2 = n2; a.err = ctx->dtcerr;
  cudaError_t e = tc_gemm_launch(a, n1 * n2, ctx->stream, ctx->tc_split);
  ++ctx->launches;
  if (e != cudaSuccess) return ctx_fail(ctx, MEHDG_ERR_CUDA, std::string("tcgen05 GEMM launch: ") + cudaGetErrorString(e));
  return MEHDG_OK;
}

// y[e][r] = -R[e][r] + sum_k sum_c A_k[e][r][c] x[e][k][c] (one warp per row, FP64 sums):
// the condensed right-hand-side pieces g and h, all directions k in one pass over A_.q
template <class T>
__global__ void __launch_bounds__(256) k_cond_rhs(const T* __restrict__ A, int M, int N, int d, long long sAe,
                                                  long long sAk, const T* __restrict__ x, long long sxe,
                                                  long long sxk, const double* __restrict__ R, double* __restrict__ y) {
  const int e = blockIdx.y, lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= M) return;
  // per-lane partial sums in the block precision (FP32 blocks: FP32, so the product
  // stays off the FP64 pipe), summed across the warp in FP64
  T s0 = T(0), s1 = T(0);
  for (int k = 0; k < d; ++k) {
    const T* a = A + e * sAe + k * sAk + (size_t)r * N;
    const T* xv = x + e * sxe + k * sxk;
    int c = lane;
    for (; c + 32 < N; c += 64) {
      s0 += a[c] * xv[c];
      s1 += a[c + 32] * xv[c + 32];
    }
    for (; c < N; c += 32) s0 += a[c] * xv[c];
  }
  double s = (double)s0 + (double)s1;
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[(size_t)e * M + r] = s - R[(size_t)e * M + r];
}

// BF16 copy (round to nearest even) of row-major [rows x n] blocks for the inner GMRES,
// rows padded to ld entries with zeros
template <class T>
__global__ void k_to_bf16(const T* __restrict__ x, unsigned short* __restrict__ y, long long rows, int n, int ld) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= rows * ld) return;
  const long long r = i / ld;
  const int c = (int)(i - r * ld);
  y[i] = c < n ? __bfloat16_as_ushort(__float2bfloat16_rn((float)x[r * n + c])) : (unsigned short)0;
}

__global__ void k_to_float(const double* x, float* y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

template <class T>
__global__ void k_scale(T* x, long long n, double a) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = (T)(a * (double)x[i]);
}

// S[(s,a)][(s,b)] += shift M[a][b]
template <class T>
__global__ void k_mass_shift(T* S, const double* M, int Np, int ns, double shift, int E, size_t sM,
                             const double* dshift) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (dshift) shift = *dshift;
  long long tot = (long long)E * ns * Np * Np;
  if (i >= tot) return;
  int b = i % Np;
  int a = (i / Np) % Np;
  int s = (i / ((long long)Np * Np)) % ns;
  int e = (int)(i / ((long long)Np * Np * ns));
  size_t Nu = (size_t)ns * Np;
  S[(size_t)e * Nu * Nu + ((size_t)s * Np + a) * Nu + (size_t)s * Np + b] +=
      (T)(shift * M[e * sM + (size_t)a * Np + b]);
}

// MinvRQ[e][k][s] = M^-1 R_Q[e][k][s]  (M^-1 shared, or per macro-element at stride sM; vpe
// vectors per macro-element)
__global__ void k_minv_rq(const double* Minv, const double* RQ, double* out, int Np, long long nvec, long long vpe,
                          size_t sM) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nvec * Np) return;
  int a = i % Np;
  long long v = i / Np;
  const double* r = RQ + v * Np;
  const double* m = Minv + (size_t)(v / vpe) * sM + (size_t)a * Np;
  double s = 0.0;
  for (int b = 0; b < Np; ++b) s += m[b] * r[b];
  out[i] = s;
}

// face blocks of A_uhuh: sum of the owners' local blocks (before D overwrites A_uhuh)
template <class T>
// (ofn: each owner's local face node of every face node, or null when both owners share the order)
__global__ void k_face_blocks(const T* Ahh, const int* owner, const int* ofn, double* fblk, int ns, int Nfn,
                              int Nth, int Nt, int nf, int F) {
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
    int e = ow / nf, fl = ow % nf;
    const int lr = ofn ? ofn[((size_t)2 * f + o) * Nfn + jr] : jr;
    const int lc = ofn ? ofn[((size_t)2 * f + o) * Nfn + jc] : jc;
    v += Ahh[(size_t)e * Nt * Nt + ((size_t)sr * Nth + fl * Nfn + lr) * Nt + (size_t)sc * Nth + fl * Nfn + lc];
  }
  fblk[i] = v;
}

// b_loc = h - B S^-1 g, one CTA per macro-element (FP64 path)
template <class T>
__global__ void __launch_bounds__(256) k_bhat_local(const T* S, const int* perm, const T* B,
                                                     const double* gvec, const double* hvec, double* bloc, int Nu,
                                                     int Nt) {
  extern __shared__ double sm[];
  double* y = sm;             // Nu: solution
  double* tmp = sm + Nu;      // Nu: right-hand side g
  const int e = blockIdx.x;
  const T* Se = S + (size_t)e * Nu * Nu;
  const int* pe = perm + (size_t)e * Nu;
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) tmp[i] = gvec[(size_t)e * Nu + i];
  __syncthreads();
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) y[i] = tmp[pe[i]];
  __syncthreads();
  lu_solve_block<T, double>(Se, Nu, y);
  const T* Be = B + (size_t)e * Nt * Nu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = w; row < Nt; row += nw) {
    double s = 0.0;
    for (int c = lane; c < Nu; c += 32) s += (double)Be[(size_t)row * Nu + c] * y[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) bloc[(size_t)e * Nt + row] = hvec[(size_t)e * Nt + row] - s;
  }
}

// Mixed precision: the same with FP32 substitutions refined in FP64 and the B product
// as FP32 per-lane partial sums added across lanes in FP64
__global__ void __launch_bounds__(256) k_bhat_local_f32(const float* S, const int* perm, const float* B,
                                                        const double* gvec, const double* hvec, double* bloc,
                                                        int Nu, int Nt, const float* S0, int iters) {
  extern __shared__ double sm[];
  double* g = sm;                                // Nu
  double* y = g + Nu;                            // Nu
  double* r = y + Nu;                            // Nu
  double* td = r + Nu;                           // Nu
  float* t = reinterpret_cast<float*>(td + Nu);  // Nu
  float* yf = t + Nu;                            // Nu
  const int e = blockIdx.x;
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) g[i] = gvec[(size_t)e * Nu + i];
  __syncthreads();
  lu_solve_f32_refined(S + (size_t)e * Nu * Nu, perm + (size_t)e * Nu, S0 ? S0 + (size_t)e * Nu * Nu : nullptr, Nu,
                       g, y, r, td, t, iters);
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) yf[i] = (float)y[i];
  __syncthreads();
  const float* Be = B + (size_t)e * Nt * Nu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = w; row < Nt; row += nw) {
    float s = 0.f;
    for (int c = lane; c < Nu; c += 32) s += Be[(size_t)row * Nu + c] * yf[c];
    double sd = s;
    for (int o = 16; o; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
    if (lane == 0) bloc[(size_t)e * Nt + row] = hvec[(size_t)e * Nt + row] - sd;
  }
}

// blocked LU with the panel in shared memory where it fits (227 KB per CTA), else the
// global-memory variant; tc selects the tcgen05 trailing update (FP32 only)
template <class T>
int batched_lu_t(mehdg_ctx* ctx, T* A, int* perm, int n, int batch, int* flag, bool tc = false) {
  if (batch == 0 || n == 0) return MEHDG_OK;
  constexpr size_t kMaxSmem = 227 * 1024 - 1024;
  if constexpr (sizeof(T) == 4) {
    if (tc && lu_panel_smem<T, true>(n) <= kMaxSmem) {
      const size_t smem = lu_panel_smem<T, true>(n);
      CK(cudaFuncSetAttribute(k_lu_panel_smem<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_lu_panel_smem<T, true><<<batch, LP_NT, smem, ctx->stream>>>(A, perm, n, flag, ctx->dtcerr);
      CKL();
      return MEHDG_OK;
    }
  }
  // small matrices (the face blocks) keep the light kernel: more CTAs per SM
  if (n >= 256 && lu_panel_smem<T, false>(n) <= kMaxSmem) {
    const size_t smem = lu_panel_smem<T, false>(n);
    CK(cudaFuncSetAttribute(k_lu_panel_smem<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_lu_panel_smem<T, false><<<batch, LP_NT, smem, ctx->stream>>>(A, perm, n, flag, nullptr);
    CKL();
    return MEHDG_OK;
  }
  size_t smem = lu_smem_bytes<T>(n);
  CK(cudaFuncSetAttribute(k_lu_batched<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_lu_batched<T><<<batch, LU_NT, smem, ctx->stream>>>(A, perm, n, flag);
  CKL();
  return MEHDG_OK;
}

// A^T_i = D + B (S^-1 C) for every macro (apply_mode 1); D is overwritten
template <class T>
int form_local_operator(mehdg_ctx* ctx, T* S, T* B, T* C, T* D) {
  const int E = ctx->E, Nu = ctx->Nu, Nt = ctx->Nt;
  T* X = reinterpret_cast<T*>(ctx->Xbuf);
  // 32 right-hand sides per CTA: the 625 x 32 FP32 block (80 KB) lets two CTAs share an SM
  // (16 per CTA measured slower: more CTAs re-stream the factors)
  constexpr int RC = 32;
  size_t smem = sizeof(T) * (size_t)Nu * RC;
  {
    cudaFuncAttributes fa{};
    int dev = 0, optin = 0;
    CK(cudaFuncGetAttributes(&fa, k_lu_solve_multi<T, RC>));
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem + fa.sharedSizeBytes > (size_t)optin)
      return ctx_fail(ctx, MEHDG_ERR_ARG, "apply_mode 1: S (Nu x 32 right-hand sides) exceeds shared memory; use "
                                          "apply_mode 0 for this degree");
  }
  dim3 grid((Nt + RC - 1) / RC, E);
  if constexpr (sizeof(T) == 4) {
    if (ctx->use_tc_nt) {
      // tcgen05: X^T = (S^-1 C)^T written K-major, then D += B X^T^T on the tensor cores
      CK(cudaFuncSetAttribute(k_lu_solve_multi<T, RC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
      phase_begin(ctx, PH_TRSM);
      k_lu_solve_multi<T, RC, true><<<grid, 256, smem, ctx->stream>>>(S, ctx->perm, C, X, Nu, Nt);
      CKL();
      phase_end(ctx, PH_TRSM);
      TcNT a{};
      a.M = Nt; a.N = Nt; a.K = Nu;
      a.A = B; a.lda = Nu; a.sA = (long long)Nt * Nu;
      a.Bt = X; a.ldb = Nu; a.sB = (long long)Nt * Nu;
      a.C = D; a.ldc = Nt; a.sC = (long long)Nt * Nt;
      a.alpha = 1.f; a.beta = 1.f; a.err = ctx->dtcerr;
      phase_begin(ctx, PH_COND_GEMM);
      cudaError_t e = tc_gemm_nt_launch(a, E, ctx->stream);
      ++ctx->launches;
      phase_end(ctx, PH_COND_GEMM);
      if (e != cudaSuccess) return ctx_fail(ctx, MEHDG_ERR_CUDA, std::string("tcgen05 NT GEMM: ") + cudaGetErrorString(e));
      return MEHDG_OK;
    }
  }
  CK(cudaFuncSetAttribute(k_lu_solve_multi<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  phase_begin(ctx, PH_TRSM);
  k_lu_solve_multi<T, RC><<<grid, 256, smem, ctx->stream>>>(S, ctx->perm, C, X, Nu, Nt);
  CKL();
  phase_end(ctx, PH_TRSM);
  if constexpr (sizeof(T) == 4) {
    if (ctx->use_tc_form)
      return tc_gemm(ctx, Nt, Nt, Nu, B, Nu, (long long)Nt * Nu, 0, X, Nt, (long long)Nu * Nt, 0, D, Nt,
                   (long long)Nt * Nt, 0, 1.f, 1.f, E, 1);
  }
  {
    CondArgs<T> a{};
    a.A = B; a.sAe = (long long)Nt * Nu; a.sAk = 0; a.sAs = 0; a.lda = Nu; a.M = Nt; a.kdiv = Nu;
    a.Bc = X; a.sBe = (long long)Nu * Nt; a.ldb = Nt;
    a.N = Nt; a.K = Nu; a.ns = 1;
    a.O1 = D; a.sO1e = (long long)Nt * Nt; a.sO1s = 0; a.ldo1 = Nt; a.o1_add = 1; a.nsplit = Nt;
    a.O2 = D; a.sO2e = 0; a.sO2s = 0; a.ldo2 = Nt; a.o2_add = 1;
    return cond_gemm(ctx, a, E);
  }
}

}  // namespace

int to_float(mehdg_ctx* ctx, const double* x, float* y, long long n) {
  if (n <= 0) return MEHDG_OK;
  k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(x, y, n);
  CKL();
  return MEHDG_OK;
}

int batched_lu(mehdg_ctx* ctx, double* A, int* perm, int n, int batch, int* flag) {
  return batched_lu_t<double>(ctx, A, perm, n, batch, flag);
}

// part 0: the whole condensation and factorisation; part 1: up to the LU of S (which a batch
// of problems then runs in one work-queue launch); part 2: from the face blocks' LU on, without
// the final status read (condense_status)
template <class T>
int condense_t(mehdg_ctx* ctx, double shift, double* bhat, int part = 0) {
  cudaStream_t st = ctx->stream;
  const int E = ctx->E, d = ctx->d, ns = ctx->ns, Np = ctx->Np, Nth = ctx->Nth;
  const long long Nu = ctx->Nu, Nt = ctx->Nt;
  int rc;
  T* Auu = reinterpret_cast<T*>(ctx->Auu);
  T* Auq = reinterpret_cast<T*>(ctx->Auq);
  T* Auh = reinterpret_cast<T*>(ctx->Auh);
  T* Ahu = reinterpret_cast<T*>(ctx->Ahu);
  T* Ahq = reinterpret_cast<T*>(ctx->Ahq);
  T* Ahh = reinterpret_cast<T*>(ctx->Ahh);
  if (part != 2) {   // ---- condensation up to the LU of S
  // face blocks of A_uhuh for the preconditioner, then their LU
  {
    long long tot = (long long)ctx->F * ctx->nfb * ctx->nfb;
    k_face_blocks<T><<<(tot + 255) / 256, 256, 0, st>>>(Ahh, ctx->owner, ctx->ofn, ctx->fblk, ns, ctx->Nfn, Nth, (int)Nt,
                                                     ctx->nf, ctx->F);
    CKL();
  }
  phase_begin(ctx, PH_CONDENSE);
  // M^-1 R_Q
  {
    long long nvec = (long long)E * d * ns;
    k_minv_rq<<<(nvec * Np + 255) / 256, 256, 0, st>>>(ctx->Minv, ctx->RQ, ctx->MinvRQ, Np, nvec,
                                                        (long long)d * ns, ctx->sM);
    CKL();
  }
  // g = -R_U + sum_k A_uq_k MinvRQ[k];  h = -R_Uh + sum_k A_uhq_k MinvRQ[k]  (eq. ASC2b pieces)
  const bool kron = ctx->klift != nullptr && !(sizeof(T) == 4 && ctx->use_tc_condense);
  if (kron) {
    // Kronecker liftings: S, C, B, D, g and h in one streaming pass (k_cond_kron)
    const T* xq = reinterpret_cast<const T*>(ctx->MinvRQ);
    if constexpr (sizeof(T) == 4) {
      if ((rc = to_float(ctx, ctx->MinvRQ, ctx->q32, (long long)E * d * Nu))) return rc;
      xq = reinterpret_cast<const T*>(ctx->q32);
    }
    phase_begin(ctx, PH_COND_GEMM);
    if ((rc = cond_kron<T>(ctx, shift, xq))) return rc;
    phase_end(ctx, PH_COND_GEMM);
  } else {
    // M^-1 R_Q in the block precision (FP32 path: into the FP32 q scratch of the assembly)
    const T* xq = reinterpret_cast<const T*>(ctx->MinvRQ);
    if constexpr (sizeof(T) == 4) {
      if ((rc = to_float(ctx, ctx->MinvRQ, ctx->q32, (long long)E * d * Nu))) return rc;
      xq = reinterpret_cast<const T*>(ctx->q32);
    }
    dim3 grid((unsigned)((Nu + 7) / 8), (unsigned)E);
    k_cond_rhs<T><<<grid, 256, 0, st>>>(Auq, (int)Nu, (int)Nu, d, (long long)d * Nu * Nu, (long long)Nu * Nu,
                                        xq, (long long)d * Nu, (long long)Nu, ctx->RU, ctx->gv);
    CKL();
    grid.x = (unsigned)((Nt + 7) / 8);
    k_cond_rhs<T><<<grid, 256, 0, st>>>(Ahq, (int)Nt, (int)Nu, d, (long long)d * Nt * Nu, (long long)Nt * Nu,
                                        xq, (long long)d * Nu, (long long)Nu, ctx->RUh, ctx->hv);
    CKL();
  }
  // S, C, B, D
  if (!kron && (shift != 0.0 || ctx->dshift)) {
    long long tot = (long long)E * ns * Np * Np;
    k_mass_shift<T><<<(tot + 255) / 256, 256, 0, st>>>(Auu, ctx->Mref, Np, ns, shift, E, ctx->sM, ctx->dshift);
    CKL();
  }
  if (!kron) {
    k_scale<T><<<(E * Nu * Nt + 255) / 256, 256, 0, st>>>(Auh, E * Nu * Nt, -1.0);
    CKL();
  }
  if (!kron && !(sizeof(T) == 4 && ctx->use_tc_condense)) {
    // [S | C] -= A_uq [W | -Wh],  [B | -D] -= A_uhq [W | -Wh]  (all directions in one K)
    CondArgs<T> a{};
    a.Bc = reinterpret_cast<const T*>(sizeof(T) == 4 ? (const void*)ctx->Bcat32 : (const void*)ctx->Bcat);
    a.sBe = (long long)ctx->sB; a.ldb = Np + Nth;
    a.N = Np + Nth; a.K = d * Np; a.ns = ns; a.kdiv = Np; a.nsplit = Np;
    a.A = Auq; a.sAe = (long long)d * Nu * Nu; a.sAk = (long long)Nu * Nu; a.sAs = Np; a.lda = (int)Nu;
    a.M = (int)Nu;
    a.O1 = Auu; a.sO1e = (long long)Nu * Nu; a.sO1s = Np; a.ldo1 = (int)Nu; a.o1_add = 0;
    a.O2 = Auh; a.sO2e = (long long)Nu * Nt; a.sO2s = Nth; a.ldo2 = (int)Nt; a.o2_add = 0;
    phase_begin(ctx, PH_COND_GEMM);
    if ((rc = cond_gemm(ctx, a, E))) return rc;
    a.A = Ahq; a.sAe = (long long)d * Nt * Nu; a.sAk = (long long)Nt * Nu; a.lda = (int)Nu; a.M = (int)Nt;
    a.O1 = Ahu; a.sO1e = (long long)Nt * Nu; a.ldo1 = (int)Nu;
    a.O2 = Ahh; a.sO2e = (long long)Nt * Nt; a.ldo2 = (int)Nt; a.o2_add = 1;
    if ((rc = cond_gemm(ctx, a, E))) return rc;
    phase_end(ctx, PH_COND_GEMM);
  }
  if (sizeof(T) == 4 && ctx->use_tc_condense) {
    for (int k = 0; k < d; ++k) {
      // S[:, s] -= A_uq_k[:, s] W_k ; C[:, s] += A_uq_k[:, s] Wh_k ; B[:, s] -= A_uhq_k[:, s] W_k ;
      // D[:, s] -= A_uhq_k[:, s] Wh_k   (batch = (macro, species s))
      const float* W32 = ctx->Wk32 + (size_t)k * Np * Np;
      const float* Wh32 = ctx->Whk32 + (size_t)k * Np * Nth;
      const float* Aq = reinterpret_cast<const float*>(Auq) + (size_t)k * Nu * Nu;
      const float* Ahq_k = reinterpret_cast<const float*>(Ahq) + (size_t)k * Nt * Nu;
      float* Auu_f = reinterpret_cast<float*>(Auu);
      float* Auh_f = reinterpret_cast<float*>(Auh);
      float* Ahu_f = reinterpret_cast<float*>(Ahu);
      float* Ahh_f = reinterpret_cast<float*>(Ahh);
      if ((rc = tc_gemm(ctx, (int)Nu, Np, Np, Aq, Nu, d * Nu * Nu, Np, W32, Np, 0, 0, Auu_f, Nu, Nu * Nu, Np, -1.f,
                        1.f, E, ns)))
        return rc;
      if ((rc = tc_gemm(ctx, (int)Nu, Nth, Np, Aq, Nu, d * Nu * Nu, Np, Wh32, Nth, 0, 0, Auh_f, Nt, Nu * Nt, Nth, 1.f,
                        1.f, E, ns)))
        return rc;
      if ((rc = tc_gemm(ctx, (int)Nt, Np, Np, Ahq_k, Nu, d * Nt * Nu, Np, W32, Np, 0, 0, Ahu_f, Nu, Nt * Nu, Np, -1.f,
                        1.f, E, ns)))
        return rc;
      if ((rc = tc_gemm(ctx, (int)Nt, Nth, Np, Ahq_k, Nu, d * Nt * Nu, Np, Wh32, Nth, 0, 0, Ahh_f, Nt, Nt * Nt, Nth,
                        -1.f, 1.f, E, ns)))
        return rc;
    }
  }
  phase_end(ctx, PH_CONDENSE);
  // LU of S and of the face blocks
  CK(cudaMemsetAsync(ctx->dflag, 0, sizeof(int) * 16, st));
  if (sizeof(T) == 4 && ctx->S32)   // unfactored S for the FP64 refinement of the local solves
    CK(cudaMemcpyAsync(ctx->S32, Auu, sizeof(float) * E * Nu * Nu, cudaMemcpyDeviceToDevice, st));
  if (part == 1) return MEHDG_OK;
  phase_begin(ctx, PH_LU);
  if ((rc = batched_lu_t<T>(ctx, Auu, ctx->perm, (int)Nu, E, ctx->dflag, sizeof(T) == 4 && ctx->use_tc_lu)))
    return rc;
  phase_end(ctx, PH_LU);
  }   // ---- from the face blocks' LU on
  phase_begin(ctx, PH_FACE_LU);
  if (ctx->finv32) {
    // mixed path: the block-Jacobi preconditioner only needs A_uhuh,f^-1 to FP32 accuracy, so
    // the face blocks are factored and inverted in FP32 (scratch: the assembly buffer, free
    // until the next assembly) and the inverses land in finv32
    const int nfb = ctx->nfb;
    const long long tot = (long long)ctx->F * nfb * nfb;
    float* f32 = reinterpret_cast<float*>(ctx->Kvol);
    k_to_float<<<(tot + 255) / 256, 256, 0, st>>>(ctx->fblk, f32, tot);
    CKL();
    if ((rc = batched_lu_t<float>(ctx, f32, ctx->fperm, nfb, ctx->F, ctx->dflag + 2))) return rc;
    const size_t smem = sizeof(float) * (size_t)nfb * 64;
    CK(cudaFuncSetAttribute(k_lu_solve_multi<float, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((nfb + 63) / 64, ctx->F);
    k_lu_solve_multi<float, 64><<<grid, 256, smem, st>>>(f32, ctx->fperm, nullptr, ctx->finv32, nfb, nfb);
    CKL();
    if (ctx->finv16) {
      const long long rows = (long long)ctx->F * nfb, tot16 = rows * ctx->ldf16;
      k_to_bf16<float><<<(unsigned)((tot16 + 255) / 256), 256, 0, st>>>(ctx->finv32, ctx->finv16, rows, nfb,
                                                                        ctx->ldf16);
      CKL();
    }
  } else {
    if ((rc = batched_lu(ctx, ctx->fblk, ctx->fperm, ctx->nfb, ctx->F, ctx->dflag + 2))) return rc;
  }
  phase_end(ctx, PH_FACE_LU);
  // b^
  phase_begin(ctx, PH_BHAT);
  if constexpr (sizeof(T) == 4) {
    const size_t smem = sizeof(double) * 4 * Nu + sizeof(float) * 2 * Nu;
    CK(cudaFuncSetAttribute(k_bhat_local_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bhat_local_f32<<<E, 256, smem, st>>>(reinterpret_cast<const float*>(Auu), ctx->perm,
                                           reinterpret_cast<const float*>(Ahu), ctx->gv, ctx->hv, ctx->bloc, (int)Nu,
                                           (int)Nt, ctx->S32, ctx->opt.refine_iters);
    CKL();
  } else {
    size_t smem = sizeof(double) * 2 * Nu;
    CK(cudaFuncSetAttribute(k_bhat_local<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_bhat_local<T><<<E, 256, smem, st>>>(Auu, ctx->perm, Ahu, ctx->gv, ctx->hv, ctx->bloc, (int)Nu, (int)Nt);
    CKL();
  }
  if (bhat) {
    if ((rc = face_reduce(ctx, ctx->bloc, bhat))) return rc;
  }
  phase_end(ctx, PH_BHAT);
  if constexpr (sizeof(T) == 8) {
    if (ctx->opt.apply_mode == 2 && (rc = sparse_pack(ctx))) return rc;
  }
  if (ctx->opt.apply_mode == 1) {
    phase_begin(ctx, PH_FORM);
    if ((rc = form_local_operator<T>(ctx, Auu, Ahu, Auh, Ahh))) return rc;
    if (ctx->Ahat16) {
      const long long rows = (long long)E * Nt, tot = rows * ctx->ld16;
      k_to_bf16<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Ahh, ctx->Ahat16, rows, Nt, ctx->ld16);
      CKL();
    }
    phase_end(ctx, PH_FORM);
  }
  if (part == 2) return MEHDG_OK;
  return condense_status(ctx);
}

// the statuses of the last condensation (synchronises the stream)
int condense_status(mehdg_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  int flags[4], tcerr = 0;
  CK(cudaMemcpyAsync(flags, ctx->dflag, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&tcerr, ctx->dtcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (tcerr) return ctx_fail(ctx, MEHDG_ERR_TIMEOUT, "a tensor-core GEMM wait timed out");
  ctx->condensed = true;
  if (flags[0]) return ctx_fail(ctx, MEHDG_ERR_SINGULAR, "zero pivot in S of macro-element " + std::to_string(flags[1] - 1));
  if (flags[2]) return ctx_fail(ctx, MEHDG_ERR_SINGULAR, "zero pivot in the A_uhuh block of face " + std::to_string(flags[3] - 1));
  return MEHDG_OK;
}

// ---------------------------------------------------------------- one-layer condensation
// Eqs. C46-C47 (Sec. 3.2): the whole local matrix A_local = [A_qq A_qu; A_uq A_uu] of a
// macro-element (size NL = Nq + Nu) is factored, and
//   A^T_i = A_uhuh - [A_uhq A_uhu] A_local^-1 [A_quh; A_uuh],
//   b^T_i = -R_Uh + [A_uhq A_uhu] A_local^-1 [R_Q; R_U],
//   [dQ; dU] = -A_local^-1 ([R_Q; R_U] + [A_quh; A_uuh] dUh).
// The paper's second layer (the default) factors only the Schur complement S (size Nu);
// this form exists to measure that difference (the paper's Table 4).  FP64; A^T_i is stored
// in place of A_uhuh and applied as in apply_mode 1.

namespace {

// A_local and the right-hand sides [A_quh; A_uuh | R] of every macro (eq. C312 blocks;
// A_qq = I (x) M, A_qu = G_k, A_quh = Gh_k as in R_Q = M q + G_k u + Gh_k uh)
__global__ void k_build_local(const double* __restrict__ M, const double* __restrict__ Gk,
                              const double* __restrict__ Ghk, const double* __restrict__ Auq,
                              const double* __restrict__ Auu, const double* __restrict__ Auh,
                              const double* __restrict__ RQ, const double* __restrict__ RU, double shift, int E, int d,
                              int ns, int Np, int Nth, double* __restrict__ Aloc, double* __restrict__ Rhs) {
  const int Nu = ns * Np, Nq = d * Nu, NL = Nq + Nu, Nt = ns * Nth, NR = Nt + 1;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long na = (long long)E * NL * NL, nr = (long long)E * NL * NR;
  if (i < na) {
    const int c = (int)(i % NL), r = (int)((i / NL) % NL);
    const long long e = i / ((long long)NL * NL);
    double v = 0.0;
    if (r < Nq) {
      const int k = r / Nu, s = (r % Nu) / Np, a = r % Np;
      if (c < Nq) {
        if (c / Nu == k && (c % Nu) / Np == s) v = M[(size_t)a * Np + c % Np];
      } else {
        const int cu = c - Nq;
        if (cu / Np == s) v = Gk[((size_t)k * Np + a) * Np + cu % Np];
      }
    } else {
      const int ru = r - Nq;
      if (c < Nq) {
        v = Auq[(((size_t)e * d + c / Nu) * Nu + ru) * Nu + c % Nu];
      } else {
        const int cu = c - Nq;
        v = Auu[((size_t)e * Nu + ru) * Nu + cu];
        if (ru / Np == cu / Np) v += shift * M[(size_t)(ru % Np) * Np + cu % Np];
      }
    }
    Aloc[i] = v;
  }
  if (i < nr) {
    const int j = (int)(i % NR), r = (int)((i / NR) % NL);
    const long long e = i / ((long long)NL * NR);
    double v;
    if (r < Nq) {
      const int k = r / Nu, s = (r % Nu) / Np, a = r % Np;
      if (j == Nt) v = RQ[(size_t)e * Nq + r];
      else v = (j / Nth == s) ? Ghk[((size_t)k * Np + a) * Nth + j % Nth] : 0.0;
    } else {
      const int ru = r - Nq;
      v = (j == Nt) ? RU[(size_t)e * Nu + ru] : Auh[((size_t)e * Nu + ru) * Nt + j];
    }
    Rhs[i] = v;
  }
}

// b_loc[e][r] = -R_Uh[e][r] + [A_uhq A_uhu][r] . y[e], y = A_local^-1 [R_Q; R_U] (last column of X)
__global__ void __launch_bounds__(256) k_onelayer_bhat(const double* __restrict__ Ahq, const double* __restrict__ Ahu,
                                                       const double* __restrict__ X, const double* __restrict__ RUh,
                                                       int d, int Nu, int Nt, double* __restrict__ bloc) {
  const int e = blockIdx.y, lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= Nt) return;
  const int Nq = d * Nu, NL = Nq + Nu, NR = Nt + 1;
  const double* Xe = X + (size_t)e * NL * NR;
  double s = 0.0;
  for (int c = lane; c < Nq; c += 32) s += Ahq[(((size_t)e * d + c / Nu) * Nt + r) * Nu + c % Nu] * Xe[(size_t)c * NR + Nt];
  for (int c = lane; c < Nu; c += 32) s += Ahu[((size_t)e * Nt + r) * Nu + c] * Xe[(size_t)(Nq + c) * NR + Nt];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) bloc[(size_t)e * Nt + r] = s - RUh[(size_t)e * Nt + r];
}

}  // namespace

int condense_one(mehdg_ctx* ctx, double shift, double* bhat) {
  cudaStream_t st = ctx->stream;
  const int E = ctx->E, d = ctx->d, ns = ctx->ns, Np = ctx->Np, Nth = ctx->Nth;
  const long long Nu = ctx->Nu, Nt = ctx->Nt, Nq = (long long)d * Nu, NL = Nq + Nu, NR = Nt + 1;
  int rc;
  {
    long long tot = (long long)ctx->F * ctx->nfb * ctx->nfb;
    k_face_blocks<double><<<(tot + 255) / 256, 256, 0, st>>>(ctx->Ahh, ctx->owner, ctx->ofn, ctx->fblk, ns, ctx->Nfn, Nth,
                                                            (int)Nt, ctx->nf, ctx->F);
    CKL();
  }
  phase_begin(ctx, PH_CONDENSE);
  {
    const long long tot = std::max((long long)E * NL * NL, (long long)E * NL * NR);
    k_build_local<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(ctx->Mref, ctx->Gk, ctx->Ghk, ctx->Auq, ctx->Auu,
                                                                 ctx->Auh, ctx->RQ, ctx->RU, shift, E, d, ns, Np, Nth,
                                                                 ctx->Aloc, ctx->Rloc);
    CKL();
  }
  CK(cudaMemsetAsync(ctx->dflag, 0, sizeof(int) * 16, st));
  phase_begin(ctx, PH_LU);
  if ((rc = batched_lu_t<double>(ctx, ctx->Aloc, ctx->permL, (int)NL, E, ctx->dflag))) return rc;
  phase_end(ctx, PH_LU);
  {
    // X = A_local^-1 [A_quh; A_uuh | R]: 32 right-hand sides per CTA (A_local^-1 applied once per column)
    constexpr int RC = 32;
    const size_t smem = sizeof(double) * (size_t)NL * RC;
    CK(cudaFuncSetAttribute(k_lu_solve_multi<double, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)((NR + RC - 1) / RC), E);
    k_lu_solve_multi<double, RC><<<grid, 256, smem, st>>>(ctx->Aloc, ctx->permL, ctx->Rloc, ctx->Xloc, (int)NL,
                                                           (int)NR);
    CKL();
  }
  {
    // A^T_i = A_uhuh - A_uhq X_q - A_uhu X_u (in place of A_uhuh)
    CondArgs<double> a{};
    a.A = ctx->Ahq; a.sAe = (long long)d * Nt * Nu; a.sAk = (long long)Nt * Nu; a.sAs = 0; a.lda = (int)Nu;
    a.M = (int)Nt; a.kdiv = (int)Nu;
    a.Bc = ctx->Xloc; a.sBe = NL * NR; a.ldb = (int)NR;
    a.N = (int)Nt; a.K = (int)Nq; a.ns = 1;
    a.O1 = ctx->Ahh; a.sO1e = Nt * Nt; a.sO1s = 0; a.ldo1 = (int)Nt; a.o1_add = 0; a.nsplit = (int)Nt;
    a.O2 = ctx->Ahh; a.ldo2 = (int)Nt;
    if ((rc = cond_gemm(ctx, a, E))) return rc;
    a.A = ctx->Ahu; a.sAe = Nt * Nu; a.sAk = 0; a.K = (int)Nu;
    a.Bc = ctx->Xloc + Nq * NR;
    if ((rc = cond_gemm(ctx, a, E))) return rc;
  }
  phase_end(ctx, PH_CONDENSE);
  phase_begin(ctx, PH_FACE_LU);
  if ((rc = batched_lu(ctx, ctx->fblk, ctx->fperm, ctx->nfb, ctx->F, ctx->dflag + 2))) return rc;
  phase_end(ctx, PH_FACE_LU);
  phase_begin(ctx, PH_BHAT);
  {
    dim3 grid((unsigned)((Nt + 7) / 8), E);
    k_onelayer_bhat<<<grid, 256, 0, st>>>(ctx->Ahq, ctx->Ahu, ctx->Xloc, ctx->RUh, d, (int)Nu, (int)Nt, ctx->bloc);
    CKL();
  }
  if (bhat && (rc = face_reduce(ctx, ctx->bloc, bhat))) return rc;
  phase_end(ctx, PH_BHAT);
  int flags[4];
  CK(cudaMemcpyAsync(flags, ctx->dflag, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->condensed = true;
  if (flags[0]) return ctx_fail(ctx, MEHDG_ERR_SINGULAR, "zero pivot in A_local of macro-element " + std::to_string(flags[1] - 1));
  if (flags[2]) return ctx_fail(ctx, MEHDG_ERR_SINGULAR, "zero pivot in the A_uhuh block of face " + std::to_string(flags[3] - 1));
  return MEHDG_OK;
}

namespace {
// [dQ; dU] = -(y + X dUh_loc) for the one-layer form (X, y from condense_one)
__global__ void __launch_bounds__(256) k_recover_one(const double* __restrict__ X, const int* __restrict__ gather,
                                                     const double* __restrict__ duh, int Nq, int Nu, int Nt,
                                                     double* __restrict__ du, double* __restrict__ dq) {
  extern __shared__ double xl[];
  const int e = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int NL = Nq + Nu, NR = Nt + 1;
  for (int i = threadIdx.x; i < Nt; i += blockDim.x) xl[i] = duh[gather[(size_t)e * Nt + i]];
  __syncthreads();
  const double* Xe = X + (size_t)e * NL * NR;
  for (int r = w; r < NL; r += nw) {
    double s = 0.0;
    for (int c = lane; c < Nt; c += 32) s += Xe[(size_t)r * NR + c] * xl[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const double v = -(s + Xe[(size_t)r * NR + Nt]);
      if (r < Nq) dq[(size_t)e * Nq + r] = v;
      else du[(size_t)e * Nu + r - Nq] = v;
    }
  }
}
}  // namespace

int recover_one(mehdg_ctx* ctx, const double* duh, double* du, double* dq) {
  const int Nq = ctx->d * ctx->Nu;
  phase_begin(ctx, PH_RECOVER);
  k_recover_one<<<ctx->E, 256, sizeof(double) * ctx->Nt, ctx->stream>>>(ctx->Xloc, ctx->gather, duh, Nq, ctx->Nu,
                                                                        ctx->Nt, du, dq);
  CKL();
  phase_end(ctx, PH_RECOVER);
  return MEHDG_OK;
}

int condense_all(mehdg_ctx* ctx, double shift, double* bhat) {
  if (ctx->opt.condense_layers == 1) return condense_one(ctx, shift, bhat);
  if (ctx->opt.precision == MEHDG_PREC_MIXED) return condense_t<float>(ctx, shift, bhat);
  return condense_t<double>(ctx, shift, bhat);
}

int condense_part(mehdg_ctx* ctx, double shift, double* bhat, int part) {
  if (ctx->opt.condense_layers == 1) return ctx_fail(ctx, MEHDG_ERR_ARG, "split condensation needs the second layer");
  if (ctx->opt.precision == MEHDG_PREC_MIXED) return condense_t<float>(ctx, shift, bhat, part);
  return condense_t<double>(ctx, shift, bhat, part);
}

extern "C" int mehdg_lu_batched(int n, int batch, void* A, int* perm, int fp32, int* dflag, void* stream) {
  if (n < 1 || batch < 0 || !A || !perm || !dflag) return MEHDG_ERR_ARG;
  mehdg_ctx tmp;
  tmp.stream = static_cast<cudaStream_t>(stream);
  mehdg_ctx* ctx = &tmp;
  CK(cudaMemsetAsync(dflag, 0, sizeof(int) * 2, tmp.stream));
  int rc = fp32 ? batched_lu_t<float>(ctx, static_cast<float*>(A), perm, n, batch, dflag)
                : batched_lu_t<double>(ctx, static_cast<double*>(A), perm, n, batch, dflag);
  if (rc) {
    std::fprintf(stderr, "mehdg_lu_batched: %s\n", tmp.err.c_str());
    return rc;
  }
  int h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, dflag, sizeof(h), cudaMemcpyDeviceToHost, tmp.stream));
  CK(cudaStreamSynchronize(tmp.stream));
  if (h[0]) {
    std::fprintf(stderr, "mehdg_lu_batched: zero pivot in matrix %d\n", h[1] - 1);
    return MEHDG_ERR_SINGULAR;
  }
  return MEHDG_OK;
}

extern "C" int mehdg_condense_factor(mehdg_ctx* ctx, double shift, double* bhat) {
  if (!ctx) return MEHDG_ERR_ARG;
  return condense_all(ctx, shift, bhat);
}
