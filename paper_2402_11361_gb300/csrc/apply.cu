// a7: matrix-free trace operator (Algorithm 2) and a10: local recovery (eq. Csc4),
// FP64 blocks.  One CTA per macro-element: gather x on dT_i, y1 = C x (step 1),
// y2 = S^-1 y1 by substitution with the stored LU factors (step 2), y3 = B y2
// (step 3), y4 = y3 + D x (step 4, local part); the per-macro results go to a slot
// array and a second kernel sums the (at most two) contributions of every
// macro-face (step 4 reduction), in a fixed order.
#include <algorithm>

#include "internal.cuh"
#include "lu.cuh"

namespace {

// Dot product of a global row with a shared-memory vector by one warp: four
// independent partial sums keep four loads per lane in flight.
template <class T, class A>
__device__ __forceinline__ A warp_dot(const T* __restrict__ row, const A* x, int n, int lane) {
  A s0 = A(0), s1 = A(0), s2 = A(0), s3 = A(0);
  int c = lane;
  for (; c + 96 < n; c += 128) {
    s0 += (A)row[c] * x[c];
    s1 += (A)row[c + 32] * x[c + 32];
    s2 += (A)row[c + 64] * x[c + 64];
    s3 += (A)row[c + 96] * x[c + 96];
  }
  for (; c < n; c += 32) s0 += (A)row[c] * x[c];
  A s = (s0 + s1) + (s2 + s3);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// T: block storage type; A: arithmetic type of the local products and solves
// (double for the FP64 path, float for the FP32-block path).
template <class T, class A>
__global__ void __launch_bounds__(512) k_apply(const T* __restrict__ S, const int* __restrict__ perm,
                                               const T* __restrict__ B, const T* __restrict__ C,
                                               const T* __restrict__ D, const int* __restrict__ gather,
                                               const double* __restrict__ x, double* __restrict__ slot, int Nu,
                                               int Nt) {
  extern __shared__ unsigned char sm_raw[];
  A* xg = reinterpret_cast<A*>(sm_raw);  // Nt
  A* y1 = xg + Nt;                        // Nu
  A* y2 = y1 + Nu;                        // Nu
  const int e = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < Nt; i += blockDim.x) xg[i] = (A)x[gather[(size_t)e * Nt + i]];
  __syncthreads();
  const T* Ce = C + (size_t)e * Nu * Nt;
  for (int r = w; r < Nu; r += nw) {
    A s = warp_dot<T, A>(Ce + (size_t)r * Nt, xg, Nt, lane);
    if (lane == 0) y1[r] = s;
  }
  __syncthreads();
  const int* pe = perm + (size_t)e * Nu;
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) y2[i] = y1[pe[i]];
  __syncthreads();
  lu_solve_block<T, A>(S + (size_t)e * Nu * Nu, Nu, y2);
  const T* Be = B + (size_t)e * Nt * Nu;
  const T* De = D + (size_t)e * Nt * Nt;
  for (int r = w; r < Nt; r += nw) {
    A s = warp_dot<T, A>(Be + (size_t)r * Nu, y2, Nu, lane) + warp_dot<T, A>(De + (size_t)r * Nt, xg, Nt, lane);
    if (lane == 0) slot[(size_t)e * Nt + r] = (double)s;
  }
}

// FP32 row . x with 8-byte loads (rows of an even-length FP32 block start 8-byte
// aligned), x read as float2 pairs from shared memory
__device__ __forceinline__ float warp_dot_f2(const float* __restrict__ row, const float* x, int n, int lane) {
  // a whole row (up to 32 x RB float2) is requested at once: RB independent loads per lane
  constexpr int RB = 12;
  const float2* r2 = reinterpret_cast<const float2*>(row);
  const float2* x2 = reinterpret_cast<const float2*>(x);
  const int n2 = n / 2;
  float s0 = 0.f, s1 = 0.f;
  for (int base = 0; base < n2; base += 32 * RB) {
    float2 a[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int j = base + lane + 32 * u;
      a[u] = (j < n2) ? __ldg(r2 + j) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int j = base + lane + 32 * u;
      const float2 xv = (j < n2) ? x2[j] : make_float2(0.f, 0.f);
      if (u & 1) s1 += a[u].x * xv.x + a[u].y * xv.y;
      else s0 += a[u].x * xv.x + a[u].y * xv.y;
    }
  }
  if ((n & 1) && lane == 0) s1 += row[n - 1] * x[n - 1];
  float s = s0 + s1;
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// The same product on the BF16 copy of A^T_i (inner GMRES of the multi-level
// preconditioner), rows padded to ld entries (a multiple of 4, zeros beyond Nt): 8-byte
// loads of four BF16 entries, consecutive across lanes, each matched by one float4 of x
// from shared memory (no bank conflict); entries widened to FP32 by shifts, FP32
// accumulation; the same persistent row-range schedule as the FP32 kernel.  For rows of
// up to 32 x RB loads a warp takes two adjacent rows at a time (3 KB in flight per warp,
// as for one FP32 row; each x chunk serves both rows); the next pair's loads are issued
// as soon as the current pair has been multiplied.
__device__ __forceinline__ float bf16x4_dot(uint2 v, float4 x) {
  return __uint_as_float(v.x << 16) * x.x + __uint_as_float(v.x & 0xFFFF0000u) * x.y +
         __uint_as_float(v.y << 16) * x.z + __uint_as_float(v.y & 0xFFFF0000u) * x.w;
}
__global__ void __launch_bounds__(256, 5) k_apply_explicit_bf16(const unsigned short* __restrict__ Ahat, int ld,
                                                                const int* __restrict__ gather,
                                                                const double* __restrict__ x,
                                                                double* __restrict__ slot, int Nt, int E,
                                                                long long rows_per_cta) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* xg = reinterpret_cast<float*>(sm_raw);   // ld floats, zero beyond Nt
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float4* x4 = reinterpret_cast<const float4*>(xg);
  const long long total = (long long)E * Nt, g0 = (long long)blockIdx.x * rows_per_cta;
  const long long g1 = min(g0 + rows_per_cta, total);
  const int n4 = ld / 4;
  constexpr int RB = 6;
  const bool pair = n4 <= 32 * RB;
  for (long long gs = g0; gs < g1;) {
    const int e = (int)(gs / Nt);
    const long long ge = min(g1, (long long)(e + 1) * Nt);
    uint2 va[RB], vb[RB];
    auto load_pair = [&](long long gr) {
      const uint2* pa = reinterpret_cast<const uint2*>(Ahat) + (size_t)gr * n4 + lane;
      const int na = gr < ge ? n4 - lane : 0, nb = gr + 1 < ge ? n4 - lane : 0;   // live entries from lane
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        va[u] = (32 * u < na) ? __ldg(pa + 32 * u) : make_uint2(0u, 0u);
        vb[u] = (32 * u < nb) ? __ldg(pa + n4 + 32 * u) : make_uint2(0u, 0u);
      }
    };
    __syncthreads();
    for (int i = threadIdx.x; i < ld; i += blockDim.x) xg[i] = i < Nt ? (float)x[gather[(size_t)e * Nt + i]] : 0.f;
    __syncthreads();
    if (pair) {
      load_pair(gs + 2 * w);
      for (long long gr = gs + 2 * w; gr < ge; gr += 2 * nw) {
        float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          const int j = lane + 32 * u;
          const float4 xv = (j < n4) ? x4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float ta = bf16x4_dot(va[u], xv), tb = bf16x4_dot(vb[u], xv);
          if (u & 1) { a1 += ta; b1 += tb; }
          else { a0 += ta; b0 += tb; }
        }
        float sa = a0 + a1, sb = b0 + b1;
        for (int o = 16; o; o >>= 1) {
          sa += __shfl_xor_sync(0xffffffffu, sa, o);
          sb += __shfl_xor_sync(0xffffffffu, sb, o);
        }
        if (lane == 0) {
          slot[gr] = (double)sa;
          if (gr + 1 < ge) slot[gr + 1] = (double)sb;
        }
        load_pair(gr + 2 * nw);
      }
    } else {
      for (long long gr = gs + w; gr < ge; gr += nw) {
        const uint2* w4 = reinterpret_cast<const uint2*>(Ahat + (size_t)gr * ld);
        float s0 = 0.f, s1 = 0.f;
        for (int base = 0; base < n4; base += 32 * RB) {
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            const int j = base + lane + 32 * u;
            va[u] = (j < n4) ? __ldg(w4 + j) : make_uint2(0u, 0u);
          }
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            const int j = base + lane + 32 * u;
            const float4 xv = (j < n4) ? x4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float t = bf16x4_dot(va[u], xv);
            if (u & 1) s1 += t;
            else s0 += t;
          }
        }
        float s = s0 + s1;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) slot[gr] = (double)s;
      }
    }
    gs = ge;
  }
}

// apply_mode 1: y4 = A^T_i x on dT_i with the stored local operator; grid (macro, row block)
template <class T, class A>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 4) k_apply_explicit(const T* __restrict__ Ahat, const int* __restrict__ gather,
                                                        const double* __restrict__ x, double* __restrict__ slot,
                                                        int Nt, int E, long long rows_per_cta) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  A* xg = reinterpret_cast<A*>(sm_raw);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // FP32 blocks with an even row length: 8-byte row loads
  const bool F2 = sizeof(T) == 4 && sizeof(A) == 4 && (Nt % 2) == 0;
  // persistent CTA: a contiguous range of the E * Nt rows, x regathered per macro-element
  const long long total = (long long)E * Nt, g0 = (long long)blockIdx.x * rows_per_cta;
  const long long g1 = min(g0 + rows_per_cta, total);
  for (long long gs = g0; gs < g1;) {
    const int e = (int)(gs / Nt);
    const long long ge = min(g1, (long long)(e + 1) * Nt);
    __syncthreads();
    for (int i = threadIdx.x; i < Nt; i += blockDim.x) xg[i] = (A)x[gather[(size_t)e * Nt + i]];
    __syncthreads();
    for (long long gr = gs + w; gr < ge; gr += nw) {
      A s;
      if (F2)
        s = (A)warp_dot_f2(reinterpret_cast<const float*>(Ahat) + (size_t)gr * Nt,
                           reinterpret_cast<const float*>(xg), Nt, lane);
      else
        s = warp_dot<T, A>(Ahat + (size_t)gr * Nt, xg, Nt, lane);
      if (lane == 0) slot[gr] = (double)s;
    }
    gs = ge;
  }
}

// y[f][s][j] = sum over the owners (e, fl) of slot[e][s][fl, l], l = j or, when the owners order
// the face nodes differently (curved meshes), l = ofn[f][o][j]
__global__ void k_face_reduce(const double* __restrict__ slot, const int* __restrict__ owner,
                              double* __restrict__ y, int ns, int Nfn, int Nth, int Nt, int nf, long long ntr,
                              const int* __restrict__ ofn = nullptr) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= ntr) return;
  int j = i % Nfn;
  int s = (i / Nfn) % ns;
  int f = (int)(i / ((long long)Nfn * ns));
  double v = 0.0;
  for (int o = 0; o < 2; ++o) {
    int ow = owner[2 * f + o];
    if (ow < 0) continue;
    int e = ow / nf, fl = ow % nf;
    const int l = ofn ? ofn[((size_t)2 * f + o) * Nfn + j] : j;
    v += slot[(size_t)e * Nt + (size_t)s * Nth + fl * Nfn + l];
  }
  y[i] = v;
}

// du = S^-1 (g + C duh_i);  dq[k][s] = -M^-1 R_Q[k][s] - W_k du_s - Wh_k duh_i,s
template <class T>
__global__ void __launch_bounds__(256) k_recover(const T* __restrict__ S, const int* __restrict__ perm,
                                                 const T* __restrict__ C, const double* __restrict__ gvec,
                                                 const double* __restrict__ MinvRQ, const double* __restrict__ Wk,
                                                 const double* __restrict__ Whk, const int* __restrict__ gather,
                                                 const double* __restrict__ duh, double* __restrict__ du,
                                                 double* __restrict__ dq, int Nu, int Nt, int Np, int Nth, int ns,
                                                 int d, size_t sG, size_t sGh) {
  extern __shared__ double sm[];
  double* xg = sm;        // Nt
  double* y1 = xg + Nt;   // Nu
  double* y2 = y1 + Nu;   // Nu
  const int e = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < Nt; i += blockDim.x) xg[i] = duh[gather[(size_t)e * Nt + i]];
  __syncthreads();
  const T* Ce = C + (size_t)e * Nu * Nt;
  for (int r = w; r < Nu; r += nw) {
    double s = 0.0;
    for (int c = lane; c < Nt; c += 32) s += (double)Ce[(size_t)r * Nt + c] * xg[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y1[r] = s + gvec[(size_t)e * Nu + r];
  }
  __syncthreads();
  const int* pe = perm + (size_t)e * Nu;
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) y2[i] = y1[pe[i]];
  __syncthreads();
  lu_solve_block<T, double>(S + (size_t)e * Nu * Nu, Nu, y2);
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) du[(size_t)e * Nu + i] = y2[i];
  const int nq = d * ns * Np;
  for (int i = threadIdx.x; i < nq; i += blockDim.x) {
    int a = i % Np, s = (i / Np) % ns, k = i / (Np * ns);
    const double* W = Wk + e * sG + ((size_t)k * Np + a) * Np;
    const double* Wh = Whk + e * sGh + ((size_t)k * Np + a) * Nth;
    double acc = MinvRQ[(size_t)e * nq + i];
    for (int b = 0; b < Np; ++b) acc += W[b] * y2[s * Np + b];
    for (int c = 0; c < Nth; ++c) acc += Wh[c] * xg[s * Nth + c];
    dq[(size_t)e * nq + i] = -acc;
  }
}

// Mixed-precision recovery: the same equations with FP32 products (per-lane FP32 partial
// sums, FP64 across lanes), FP32 substitutions with FP64-refined local solve, and the
// lifting products W_k, Wh_k in FP32.
__global__ void __launch_bounds__(256) k_recover_f32(const float* __restrict__ S, const int* __restrict__ perm,
                                                     const float* __restrict__ C, const double* __restrict__ gvec,
                                                     const double* __restrict__ MinvRQ, const float* __restrict__ Wk,
                                                     const float* __restrict__ Whk, const int* __restrict__ gather,
                                                     const double* __restrict__ duh, double* __restrict__ du,
                                                     double* __restrict__ dq, int Nu, int Nt, int Np, int Nth, int ns,
                                                     int d, const float* __restrict__ S0, int iters, size_t sG,
                                                     size_t sGh) {
  extern __shared__ double sm[];
  double* y1 = sm;                                 // Nu: right-hand side
  double* y2 = y1 + Nu;                            // Nu: solution
  double* r = y2 + Nu;                             // Nu: refinement residual
  double* td = r + Nu;                             // Nu: refinement correction
  float* xf = reinterpret_cast<float*>(td + Nu);   // Nt: gathered duh
  float* t = xf + ((Nt + 1) & ~1);                 // Nu: FP32 solve vector (first Nt doubles: gathered duh)
  float* yf = t + (Nu > 2 * Nt ? Nu : 2 * Nt);     // Nu: FP32 copy of the solution
  const int e = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* xg = reinterpret_cast<double*>(t);   // the FP32 scratch is not in use yet: gathered duh in FP64
  for (int i = threadIdx.x; i < Nt; i += blockDim.x) {
    const double v = duh[gather[(size_t)e * Nt + i]];
    xf[i] = (float)v;
    xg[i] = v;
  }
  __syncthreads();
  // right-hand side of the local solve, g + C duh, accumulated in FP64 (the refined solve
  // is then accurate to the FP64 level for this right-hand side)
  const float* Ce = C + (size_t)e * Nu * Nt;
  for (int row = w; row < Nu; row += nw) {
    double s = 0.0;
    for (int c = lane; c < Nt; c += 32) s += (double)Ce[(size_t)row * Nt + c] * xg[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y1[row] = s + gvec[(size_t)e * Nu + row];
  }
  __syncthreads();
  const int* pe = perm + (size_t)e * Nu;
  lu_solve_f32_refined(S + (size_t)e * Nu * Nu, pe, S0 ? S0 + (size_t)e * Nu * Nu : nullptr, Nu, y1, y2, r, td, t,
                       iters);
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) {
    du[(size_t)e * Nu + i] = y2[i];
    yf[i] = (float)y2[i];
  }
  __syncthreads();
  const int nq = d * ns * Np;
  for (int i = threadIdx.x; i < nq; i += blockDim.x) {
    int a = i % Np, s = (i / Np) % ns, k = i / (Np * ns);
    const float* W = Wk + e * sG + ((size_t)k * Np + a) * Np;
    const float* Wh = Whk + e * sGh + ((size_t)k * Np + a) * Nth;
    float acc = 0.f;
    for (int b = 0; b < Np; ++b) acc += W[b] * yf[s * Np + b];
    for (int c = 0; c < Nth; ++c) acc += Wh[c] * xf[s * Nth + c];
    dq[(size_t)e * nq + i] = -(MinvRQ[(size_t)e * nq + i] + (double)acc);
  }
}

}  // namespace

int face_reduce(mehdg_ctx* ctx, const double* slot, double* y) {
  k_face_reduce<<<(ctx->ntr + 255) / 256, 256, 0, ctx->stream>>>(slot, ctx->owner, y, ctx->ns, ctx->Nfn, ctx->Nth,
                                                                 ctx->Nt, ctx->nf, ctx->ntr, ctx->ofn);
  CKL();
  return MEHDG_OK;
}

template <class T, class A>
static int apply_t(mehdg_ctx* ctx, const double* x, double* y) {
  if (ctx->opt.apply_mode == 1) {
    // persistent grid: (resident CTAs per SM) x (SM count), each CTA a contiguous
    // share of the rows, so no partial last wave
    const bool lowp = ctx->lowp_apply && ctx->Ahat16;
    int& grid = lowp ? ctx->apply_grid16 : ctx->apply_grid;
    if (grid <= 0) {
      int dev = 0, sms = 0, per = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      if (lowp)
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_apply_explicit_bf16, 256, sizeof(float) * ctx->ld16));
      else
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_apply_explicit<T, A>, 256, sizeof(A) * ctx->Nt));
      grid = std::max(1, sms * std::max(1, per));
    }
    const long long total = (long long)ctx->E * ctx->Nt;
    const long long rows = (total + grid - 1) / grid;
    if (lowp) {
      phase_begin(ctx, PH_APPLY_BF16);
      k_apply_explicit_bf16<<<grid, 256, sizeof(float) * ctx->ld16, ctx->stream>>>(
          ctx->Ahat16, ctx->ld16, ctx->gather, x, ctx->slot, ctx->Nt, ctx->E, rows);
      CKL();
      phase_end(ctx, PH_APPLY_BF16);
      return y ? face_reduce(ctx, ctx->slot, y) : MEHDG_OK;
    }
    phase_begin(ctx, PH_APPLY);
    k_apply_explicit<T, A><<<grid, 256, sizeof(A) * ctx->Nt, ctx->stream>>>(
        reinterpret_cast<const T*>(ctx->Ahh), ctx->gather, x, ctx->slot, ctx->Nt, ctx->E, rows);
    CKL();
    phase_end(ctx, PH_APPLY);
    return face_reduce(ctx, ctx->slot, y);
  }
  size_t smem = sizeof(A) * (ctx->Nt + 2 * (size_t)ctx->Nu);
  CK(cudaFuncSetAttribute(k_apply<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  phase_begin(ctx, PH_APPLY);
  k_apply<T, A><<<ctx->E, 512, smem, ctx->stream>>>(
      reinterpret_cast<const T*>(ctx->Auu), ctx->perm, reinterpret_cast<const T*>(ctx->Ahu),
      reinterpret_cast<const T*>(ctx->Auh), reinterpret_cast<const T*>(ctx->Ahh), ctx->gather, x, ctx->slot, ctx->Nu,
      ctx->Nt);
  CKL();
  phase_end(ctx, PH_APPLY);
  return face_reduce(ctx, ctx->slot, y);
}

// The BF16 apply of the inner GMRES into the per-macro slots only (the face reduction is
// left to the consumer); true when the context has that path.
bool apply_bf16_slots_available(const mehdg_ctx* ctx) {
  // (the fused face sum inside the BF16 block-Jacobi product assumes both owners of a face
  // order its nodes alike: box meshes)
  return ctx->opt.precision == MEHDG_PREC_MIXED && ctx->opt.apply_mode == 1 && ctx->Ahat16 && ctx->finv16 &&
         !ctx->ofn;
}
int apply_bf16_slots(mehdg_ctx* ctx, const double* x) {
  if (!apply_bf16_slots_available(ctx)) return ctx_fail(ctx, MEHDG_ERR_ARG, "no BF16 operator copy");
  const bool keep = ctx->lowp_apply;
  ctx->lowp_apply = true;
  const int rc = apply_t<float, float>(ctx, x, nullptr);
  ctx->lowp_apply = keep;
  return rc;
}

int apply_trace_impl(mehdg_ctx* ctx, const double* x, double* y) {
  if (!ctx->condensed) return ctx_fail(ctx, MEHDG_ERR_ARG, "apply before mehdg_condense_factor");
  if (ctx->opt.precision == MEHDG_PREC_MIXED) return apply_t<float, float>(ctx, x, y);
  if (ctx->opt.apply_mode == 2) return apply_sparse(ctx, x, y);
  return apply_t<double, double>(ctx, x, y);
}

int recover_impl(mehdg_ctx* ctx, const double* duh, double* du, double* dq) {
  if (!ctx->condensed) return ctx_fail(ctx, MEHDG_ERR_ARG, "recover before mehdg_condense_factor");
  if (ctx->opt.condense_layers == 1) return recover_one(ctx, duh, du, dq);
  size_t smem = sizeof(double) * (ctx->Nt + 2 * (size_t)ctx->Nu);
  phase_begin(ctx, PH_RECOVER);
  if (ctx->opt.precision == MEHDG_PREC_MIXED) {
    const size_t Nu = ctx->Nu, Nt = ctx->Nt;
    const size_t smem32 = sizeof(double) * 4 * Nu + sizeof(float) * (((Nt + 1) & ~(size_t)1) + (Nu > 2 * Nt ? Nu : 2 * Nt) + Nu);
    CK(cudaFuncSetAttribute(k_recover_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32));
    k_recover_f32<<<ctx->E, 256, smem32, ctx->stream>>>(
        reinterpret_cast<const float*>(ctx->Auu), ctx->perm, reinterpret_cast<const float*>(ctx->Auh), ctx->gv,
        ctx->MinvRQ, ctx->Wk32, ctx->Whk32, ctx->gather, duh, du, dq, ctx->Nu, ctx->Nt, ctx->Np, ctx->Nth, ctx->ns,
        ctx->d, ctx->S32, ctx->opt.refine_iters, ctx->sG, ctx->sGh);
    CKL();
    phase_end(ctx, PH_RECOVER);
    return MEHDG_OK;
  }
  CK(cudaFuncSetAttribute(k_recover<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_recover<double><<<ctx->E, 256, smem, ctx->stream>>>(ctx->Auu, ctx->perm, ctx->Auh, ctx->gv, ctx->MinvRQ, ctx->Wk,
                                                ctx->Whk, ctx->gather, duh, du, dq, ctx->Nu, ctx->Nt, ctx->Np,
                                                ctx->Nth, ctx->ns, ctx->d, ctx->sG, ctx->sGh);
  CKL();
  phase_end(ctx, PH_RECOVER);
  return MEHDG_OK;
}

extern "C" int mehdg_apply_trace(mehdg_ctx* ctx, const double* x, double* y) {
  if (!ctx || !x || !y || x == y) return MEHDG_ERR_ARG;
  return apply_trace_impl(ctx, x, y);
}

extern "C" int mehdg_recover(mehdg_ctx* ctx, const double* duh, double* du, double* dq) {
  if (!ctx || !duh || !du || !dq) return MEHDG_ERR_ARG;
  return recover_impl(ctx, duh, du, dq);
}

// ---------------------------------------------------------------- allocation-free trace apply
// Same kernels as mehdg_apply_trace, but every array is the caller's and the per-macro
// slot scratch lives in a file-scope device array instead of context memory.
#include <cstdio>
#include <mutex>

static constexpr long long kNoallocSlotMax = 1LL << 22;   // doubles (32 MiB)
static __device__ __align__(256) double g_noalloc_slot[kNoallocSlotMax];

namespace {
std::mutex g_noalloc_mtx;
double* g_noalloc_ptr[128] = {};

int noalloc_slot(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) {
    fprintf(stderr, "mehdg_apply_trace_noalloc: no usable current device (%s)\n", cudaGetErrorString(e));
    return MEHDG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mtx);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_slot);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "mehdg_apply_trace_noalloc: cudaGetSymbolAddress failed (%s)\n", cudaGetErrorString(e));
      return MEHDG_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return MEHDG_OK;
}
}  // namespace

extern "C" int mehdg_apply_trace_noalloc(int dim, int n_macro, int n_face, int Nu, int Nfn, const double* S_lu,
                                         const int* perm, const double* B, const double* C, const double* D,
                                         const int* gather, const int* owner, const double* x, double* y,
                                         void* stream) {
  if (dim < 2 || dim > 3 || n_macro < 1 || n_face < 1 || Nu < 1 || Nfn < 1 || !S_lu || !perm || !B || !C || !D ||
      !gather || !owner || !x || !y || x == y)
    return MEHDG_ERR_ARG;
  const int ns = dim + 2;
  const int Nth = 2 * dim * Nfn;
  const int Nt = ns * Nth;
  const long long need = (long long)n_macro * Nt;
  if (need > kNoallocSlotMax) {
    fprintf(stderr,
            "mehdg_apply_trace_noalloc: n_macro * Nt = %lld doubles exceeds the static scratch of %lld doubles\n",
            need, kNoallocSlotMax);
    return MEHDG_ERR_TOO_LARGE;
  }
  const size_t smem = sizeof(double) * (Nt + 2 * (size_t)Nu);
  double* slot = nullptr;
  int rc = noalloc_slot(&slot);
  if (rc) return rc;
  {
    // the kernel's own static shared memory (the substitution's diagonal block) counts
    // against the same per-block limit as the dynamic part
    cudaFuncAttributes fa{};
    int dev = 0, optin = 0;
    if (cudaFuncGetAttributes(&fa, k_apply<double, double>) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return MEHDG_ERR_CUDA;
    if (smem + fa.sharedSizeBytes > (size_t)optin) {
      fprintf(stderr, "mehdg_apply_trace_noalloc: Nt + 2 Nu = %lld doubles of shared memory exceed the %d bytes "
              "a block may use next to the kernel's %zu static bytes\n", (long long)(Nt + 2 * (size_t)Nu), optin,
              (size_t)fa.sharedSizeBytes);
      return MEHDG_ERR_ARG;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaFuncSetAttribute(k_apply<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return MEHDG_ERR_CUDA;
  k_apply<double, double><<<n_macro, 512, smem, st>>>(S_lu, perm, B, C, D, gather, x, slot, Nu, Nt);
  const long long ntr = (long long)n_face * ns * Nfn;
  k_face_reduce<<<(ntr + 255) / 256, 256, 0, st>>>(slot, owner, y, ns, Nfn, Nth, Nt, 2 * dim, ntr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "mehdg_apply_trace_noalloc: launch failed (%s)\n", cudaGetErrorString(e));
    return MEHDG_ERR_CUDA;
  }
  return MEHDG_OK;
}
