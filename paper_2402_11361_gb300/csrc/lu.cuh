// Batched dense LU with partial pivoting (P A = L U, first maximal |.| row wins ties)
// and the matching forward/back substitution for one CTA.  The paper stores a
// factorisation of each Schur complement S and applies S^-1 by substitution
// (Remark, Sec. 3.3); here one CTA factors one matrix held in global memory:
// unblocked panel of width LU_NB with row swaps over whole rows, triangular solve
// for the block row of U, then a tiled rank-LU_NB update of the trailing matrix
// (FP32 SIMT or FP64 DFMA; for FP32 matrices optionally split-TF32 tcgen05 MMAs with the
// accumulator in tensor memory).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "tc_gemm.cuh"

constexpr int LU_NT = 256;
constexpr int LU_NB = 32;
constexpr int LU_TM = 64;

template <class T>
inline size_t lu_smem_bytes(int n) {
  (void)n;
  return sizeof(T) * ((size_t)LU_TM * (LU_NB + 1) + (size_t)LU_NB * (LU_TM + 1));
}

template <class T>
__global__ void __launch_bounds__(LU_NT) k_lu_batched(T* __restrict__ Aall, int* __restrict__ permall, int n,
                                                     int* __restrict__ flag) {
  extern __shared__ unsigned char lu_smem_raw[];
  T* sL = reinterpret_cast<T*>(lu_smem_raw);          // [LU_TM][LU_NB+1]
  T* sU = sL + LU_TM * (LU_NB + 1);                   // [LU_NB][LU_TM+1]
  __shared__ double rv[LU_NT / 32];
  __shared__ int ri[LU_NT / 32];
  __shared__ int spiv;
  __shared__ T spval;
  T* A = Aall + (size_t)blockIdx.x * n * n;
  int* perm = permall + (size_t)blockIdx.x * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += LU_NT) perm[i] = i;
  __syncthreads();
  for (int j0 = 0; j0 < n; j0 += LU_NB) {
    const int jb = min(LU_NB, n - j0);
    for (int j = j0; j < j0 + jb; ++j) {
      // pivot search in column j
      double bv = -1.0;
      int bi = n;
      for (int i = j + tid; i < n; i += LU_NT) {
        double v = fabs((double)A[(size_t)i * n + j]);
        if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
      }
      for (int o = 16; o; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) { rv[warp] = bv; ri[warp] = bi; }
      __syncthreads();
      if (tid == 0) {
        double b = rv[0];
        int ib = ri[0];
        for (int w = 1; w < LU_NT / 32; ++w)
          if (rv[w] > b || (rv[w] == b && ri[w] < ib)) { b = rv[w]; ib = ri[w]; }
        spiv = ib;
        if (b == 0.0) {
          if (atomicCAS(flag, 0, 1) == 0) flag[1] = blockIdx.x + 1;
        }
      }
      __syncthreads();
      const int r = spiv;
      if (r != j && r < n) {
        for (int c = tid; c < n; c += LU_NT) {
          T t = A[(size_t)j * n + c];
          A[(size_t)j * n + c] = A[(size_t)r * n + c];
          A[(size_t)r * n + c] = t;
        }
        if (tid == 0) {
          int t = perm[j];
          perm[j] = perm[r];
          perm[r] = t;
        }
      }
      __syncthreads();
      if (tid == 0) spval = A[(size_t)j * n + j];
      __syncthreads();
      const T piv = spval;
      const T inv = (piv != T(0)) ? T(1) / piv : T(0);
      for (int i = j + 1 + tid; i < n; i += LU_NT) {
        T l = A[(size_t)i * n + j] * inv;
        A[(size_t)i * n + j] = l;
        for (int c = j + 1; c < j0 + jb; ++c) A[(size_t)i * n + c] -= l * A[(size_t)j * n + c];
      }
      __syncthreads();
    }
    const int c0 = j0 + jb;
    if (c0 >= n) break;
    // U12 = L11^-1 A12, one thread per column
    for (int c = c0 + tid; c < n; c += LU_NT) {
      for (int r = 1; r < jb; ++r) {
        T s = A[(size_t)(j0 + r) * n + c];
        for (int q = 0; q < r; ++q) s -= A[(size_t)(j0 + r) * n + j0 + q] * A[(size_t)(j0 + q) * n + c];
        A[(size_t)(j0 + r) * n + c] = s;
      }
    }
    __syncthreads();
    // A22 -= L21 U12, 64 x 64 tiles, 16 outputs per thread
    const int m2 = n - c0;
    const int tx = tid % 16, ty = tid / 16;
    for (int ti = 0; ti < m2; ti += LU_TM) {
      for (int i = tid; i < LU_TM * jb; i += LU_NT) {
        int rr = i / jb, cc = i % jb;
        int gr = c0 + ti + rr;
        sL[rr * (LU_NB + 1) + cc] = (gr < n) ? A[(size_t)gr * n + j0 + cc] : T(0);
      }
      for (int tj = 0; tj < m2; tj += LU_TM) {
        for (int i = tid; i < jb * LU_TM; i += LU_NT) {
          int rr = i / LU_TM, cc = i % LU_TM;
          int gc = c0 + tj + cc;
          sU[rr * (LU_TM + 1) + cc] = (gc < n) ? A[(size_t)(j0 + rr) * n + gc] : T(0);
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
        for (int kk = 0; kk < jb; ++kk) {
          T lv[4], uv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) lv[a] = sL[(ty + 16 * a) * (LU_NB + 1) + kk];
#pragma unroll
          for (int b = 0; b < 4; ++b) uv[b] = sU[kk * (LU_TM + 1) + tx + 16 * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += lv[a] * uv[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            int gr = c0 + ti + ty + 16 * a, gc = c0 + tj + tx + 16 * b;
            if (gr < n && gc < n) A[(size_t)gr * n + gc] -= acc[a][b];
          }
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

// y <- U^-1 L^-1 y for factors LU (row-major, unit L), y already permuted (P y).
// Called by all threads of the CTA; y in shared memory; arithmetic in Acc.
// Blocked by 32 rows: the warps first subtract the already-solved part from the block's
// rows (one warp per row, dot products over the solved prefix or suffix) while the
// 32 x 32 diagonal block is staged in shared memory (transposed, row stride 33: lane r
// reads its row without bank conflicts); then warp 0 solves the block column by column:
// lane l holds y_l, and once y_l is final it is broadcast by one shuffle and every lane
// r below (above) it subtracts L[r][l] y_l (U[r][l] y_l).  The block's dependent chain
// is one shuffle and one FMA per column, with no global-memory load inside it.
template <class T, class Acc = double>
__device__ void lu_solve_block(const T* __restrict__ LU, int n, Acc* y) {
  __shared__ Acc dblk[32][33];   // dblk[l][r] = factor entry (row i0 + r, column i0 + l)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto stage = [&](int i0, int ib) {
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
      const int r = idx >> 5, l = idx & 31;
      dblk[l][r] = (r < ib && l < ib) ? (Acc)LU[(size_t)(i0 + r) * n + i0 + l] : Acc(0);
    }
  };
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int ib = min(32, n - i0);
    stage(i0, ib);
    for (int r = warp; r < ib; r += nw) {
      const T* row = LU + (size_t)(i0 + r) * n;
      Acc s0 = Acc(0), s1 = Acc(0), s2 = Acc(0), s3 = Acc(0);
      int c = lane;
      for (; c + 96 < i0; c += 128) {
        s0 += (Acc)row[c] * y[c];
        s1 += (Acc)row[c + 32] * y[c + 32];
        s2 += (Acc)row[c + 64] * y[c + 64];
        s3 += (Acc)row[c + 96] * y[c + 96];
      }
      for (; c < i0; c += 32) s0 += (Acc)row[c] * y[c];
      Acc s = (s0 + s1) + (s2 + s3);
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) y[i0 + r] -= s;
    }
    __syncthreads();
    if (warp == 0) {
      Acc yl = (lane < ib) ? y[i0 + lane] : Acc(0);
      for (int l = 0; l < ib - 1; ++l) {
        const Acc yb = __shfl_sync(0xffffffffu, yl, l);
        if (lane > l) yl -= dblk[l][lane] * yb;
      }
      if (lane < ib) y[i0 + lane] = yl;
    }
    __syncthreads();
  }
  for (int i0 = ((n - 1) / 32) * 32; i0 >= 0; i0 -= 32) {
    const int ib = min(32, n - i0);
    stage(i0, ib);
    for (int r = warp; r < ib; r += nw) {
      const T* row = LU + (size_t)(i0 + r) * n;
      Acc s0 = Acc(0), s1 = Acc(0), s2 = Acc(0), s3 = Acc(0);
      int c = i0 + ib + lane;
      for (; c + 96 < n; c += 128) {
        s0 += (Acc)row[c] * y[c];
        s1 += (Acc)row[c + 32] * y[c + 32];
        s2 += (Acc)row[c + 64] * y[c + 64];
        s3 += (Acc)row[c + 96] * y[c + 96];
      }
      for (; c < n; c += 32) s0 += (Acc)row[c] * y[c];
      Acc s = (s0 + s1) + (s2 + s3);
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) y[i0 + r] -= s;
    }
    __syncthreads();
    if (warp == 0) {
      Acc yl = (lane < ib) ? y[i0 + lane] : Acc(0);
      for (int l = ib - 1; l >= 0; --l) {
        if (lane == l) yl = yl / dblk[l][l];
        const Acc yb = __shfl_sync(0xffffffffu, yl, l);
        if (lane < l) yl -= dblk[l][lane] * yb;
      }
      if (lane < ib) y[i0 + lane] = yl;
    }
    __syncthreads();
  }
}

// FP32-factor solve with FP64 refinement (mixed precision): x = S^-1 rhs by FP32
// substitutions, then `iters` sweeps of r = rhs - S0 x accumulated in FP64 (S0 the FP32
// matrix before factorisation, or none) and x += S^-1 r, the correction by substitutions
// in FP64 arithmetic on the FP32 factors.  rhs, x, r, td: FP64 shared vectors of length
// n; t: FP32 shared scratch of length n.
__device__ inline void lu_solve_f32_refined(const float* __restrict__ LU, const int* __restrict__ perm,
                                            const float* __restrict__ S0, int n, const double* rhs, double* x,
                                            double* r, double* td, float* t, int iters) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t[i] = (float)rhs[perm[i]];
  __syncthreads();
  lu_solve_block<float, float>(LU, n, t);
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = t[i];
  __syncthreads();
  for (int it = 0; S0 && it < iters; ++it) {
    for (int row = w; row < n; row += nw) {
      const float* sr = S0 + (size_t)row * n;
      double s = 0.0;
      for (int c = lane; c < n; c += 32) s += (double)sr[c] * x[c];
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) r[row] = rhs[row] - s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) td[i] = r[perm[i]];
    __syncthreads();
    lu_solve_block<float, double>(LU, n, td);
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] += td[i];
    __syncthreads();
  }
}

// X = S^-1 B for a block of RC right-hand-side columns of one macro-element
// (grid: column block x macro), from the LU factors and row permutation of S.
// B and X are row-major [n][nrhs]; the RC columns of P B live in shared memory.
// Right-looking blocked substitution: for each 32-row block, the diagonal block of
// L (or U) is staged in shared memory and the block's rows are solved in registers
// (256 / RC threads per right-hand side); then every row below (forward) or above
// (backward) is updated, x_r -= L[r, blk] x_blk, in chunks of 128 rows: the chunk of
// L is staged in shared memory transposed (prefetched into registers while the previous
// chunk computes) and each thread keeps an 8-row x CPT-column tile of the update in
// registers.  B == nullptr solves for the identity (columns of S^-1).
// XT: write X transposed, [nrhs][n] (the K-major right operand of a tcgen05 product)
template <class T, int RC, bool XT = false>
__global__ void __launch_bounds__(256, (RC * sizeof(T) <= 64) ? 3 : ((RC * sizeof(T) <= 128) ? 2 : 1))
    k_lu_solve_multi(const T* __restrict__ LUall, const int* __restrict__ permall,
                                                       const T* __restrict__ Ball, T* __restrict__ Xall, int n,
                                                       int nrhs) {
  constexpr int CH = 128;                 // rows per update chunk
  constexpr int CPT = RC / 16;            // columns per thread in the update
  constexpr int PF = CH * 32 / 256;       // chunk elements per thread
  static_assert(RC % 16 == 0 && (CPT * sizeof(T) == 16 || CPT * sizeof(T) == 8 || CPT * sizeof(T) == 4), "RC");
  using V16 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  using V8 = typename std::conditional<sizeof(T) == 4, float2, double>::type;
  using V = typename std::conditional<CPT * sizeof(T) == 16, V16,
                                      typename std::conditional<CPT * sizeof(T) == 8, V8, float>::type>::type;
  extern __shared__ __align__(16) unsigned char lum_raw[];
  T* x = reinterpret_cast<T*>(lum_raw);   // [n][RC]
  __shared__ T lt[32][33];                // diagonal block
  __shared__ __align__(16) T ls[32][CH + 4];   // update chunk of L or U, stored transposed [k][row]
  // grid (column block, matrix): the column-block CTAs of one matrix are adjacent in
  // launch order, so they run together and share its factors through L2
  const int e = blockIdx.y, c0 = blockIdx.x * RC;
  const int rc = min(RC, nrhs - c0);
  const T* LU = LUall + (size_t)e * n * n;
  const int* perm = permall + (size_t)e * n;
  const T* Bm = Ball ? Ball + (size_t)e * n * nrhs : nullptr;
  T* X = Xall + (size_t)e * n * nrhs;
  const int tid = threadIdx.x;
  for (int i = tid; i < n * RC; i += blockDim.x) {
    int r = i / RC, c = i % RC;
    if (Bm) x[i] = (c < rc) ? Bm[(size_t)perm[r] * nrhs + c0 + c] : T(0);
    else x[i] = (c < rc && perm[r] == c0 + c) ? T(1) : T(0);   // B = I: columns of S^-1
  }
  const int tr = tid / 16, tcol = (tid % 16) * CPT;   // update tile: rows tr*8.., columns tcol..
  T pf[PF];
  // chunk rows [r0, r1) x block columns [i0, i0 + ib) into registers (zero outside)
  // a warp moves 4-row x 8-column patches of the chunk: 32-byte segments of 4 rows from
  // global memory, and into the transposed shared layout (row stride CH + 4 = 4 mod 32
  // banks) one bank per lane
  const int lw = tid >> 5, ll = tid & 31;
  auto fetch = [&](int r0, int r1, int i0, int ib) {
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      const int t = lw + 8 * j, rr = (t >> 2) * 4 + (ll >> 3), kk = (t & 3) * 8 + (ll & 7);
      pf[j] = (r0 + rr < r1 && kk < ib) ? LU[(size_t)(r0 + rr) * n + i0 + kk] : T(0);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      const int t = lw + 8 * j, rr = (t >> 2) * 4 + (ll >> 3), kk = (t & 3) * 8 + (ll & 7);
      ls[kk][rr] = pf[j];
    }
  };
  // x[r0 + rr] -= ls[rr] . x[i0 .. i0 + ib) for the rows of the chunk
  auto update = [&](int r0, int r1, int i0, int ib) {
    T acc[8][CPT];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int o = 0; o < CPT; ++o) acc[a][o] = T(0);
#pragma unroll 4
    for (int q = 0; q < ib; ++q) {
      const V xv = *reinterpret_cast<const V*>(x + (size_t)(i0 + q) * RC + tcol);
      const T* xs = reinterpret_cast<const T*>(&xv);
      // the thread's 8 rows of column q of the chunk: contiguous, 16-byte aligned
      T lv[8];
      if constexpr (sizeof(T) == 4) {
        const float4 l0 = *reinterpret_cast<const float4*>(&ls[q][tr * 8]);
        const float4 l1 = *reinterpret_cast<const float4*>(&ls[q][tr * 8 + 4]);
        lv[0] = l0.x; lv[1] = l0.y; lv[2] = l0.z; lv[3] = l0.w;
        lv[4] = l1.x; lv[5] = l1.y; lv[6] = l1.z; lv[7] = l1.w;
      } else {
#pragma unroll
        for (int a = 0; a < 8; ++a) lv[a] = ls[q][tr * 8 + a];
      }
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int o = 0; o < CPT; ++o) acc[a][o] += lv[a] * xs[o];
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int r = r0 + tr * 8 + a;
      if (r < r1) {
        T* xo = x + (size_t)r * RC + tcol;
#pragma unroll
        for (int o = 0; o < CPT; ++o) xo[o] -= acc[a][o];
      }
    }
  };
  // 32 x 32 diagonal-block solves: TPC threads per right-hand side (adjacent lanes), each
  // holding the block rows q = dsub + TPC u in registers; column by column, the owner of
  // the finished row l broadcasts it within its lane group by one shuffle and every thread
  // subtracts L[q][l] (U[q][l]) times it from its rows below (above) l, so the dependent
  // chain is one shuffle and one FMA per column
  constexpr int TPC = 256 / RC, QPT = 32 / TPC;
  static_assert(TPC * RC == 256 && TPC <= 32 && 32 % TPC == 0, "threads per right-hand side");
  const int dcol = tid / TPC, dsub = tid % TPC, gbase = (tid & 31) & ~(TPC - 1);
  auto diag_fwd = [&](int i0, int ib) {
    T v[QPT];
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
      const int q = dsub + TPC * u;
      v[u] = (q < ib) ? x[(size_t)(i0 + q) * RC + dcol] : T(0);
    }
#pragma unroll
    for (int l = 0; l < 31; ++l) {
      if (l >= ib - 1) break;
      const T vb = __shfl_sync(0xffffffffu, v[l / TPC], gbase + l % TPC);
#pragma unroll
      for (int u = 0; u < QPT; ++u) {
        const int q = dsub + TPC * u;
        if (q > l) v[u] -= lt[q][l] * vb;
      }
    }
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
      const int q = dsub + TPC * u;
      if (q < ib) x[(size_t)(i0 + q) * RC + dcol] = v[u];
    }
  };
  auto diag_bwd = [&](int i0, int ib) {
    T v[QPT];
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
      const int q = dsub + TPC * u;
      v[u] = (q < ib) ? x[(size_t)(i0 + q) * RC + dcol] : T(0);
    }
#pragma unroll
    for (int l = 31; l >= 0; --l) {
      if (l < ib) {
        if (dsub == l % TPC) v[l / TPC] = v[l / TPC] / lt[l][l];
        const T vb = __shfl_sync(0xffffffffu, v[l / TPC], gbase + l % TPC);
#pragma unroll
        for (int u = 0; u < QPT; ++u) {
          const int q = dsub + TPC * u;
          if (q < l) v[u] -= lt[q][l] * vb;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
      const int q = dsub + TPC * u;
      if (q < ib) x[(size_t)(i0 + q) * RC + dcol] = v[u];
    }
  };
  __syncthreads();
  // the next 32 x 32 diagonal block is prefetched into registers while the current block
  // is processed (4 entries per thread), so only the first one of each sweep waits
  T dg[4];
  auto fetch_diag = [&](int i0, int ib) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = tid + 256 * u, a = i / 32, b = i % 32;
      dg[u] = (a < ib && b < ib) ? LU[(size_t)(i0 + a) * n + i0 + b] : T(0);
    }
  };
  auto stash_diag = [&]() {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = tid + 256 * u;
      lt[i / 32][i % 32] = dg[u];
    }
  };
  // ---- forward: L y = P b (unit diagonal)
  fetch_diag(0, min(32, n));
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int ib = min(32, n - i0);
    stash_diag();
    if (i0 + 32 < n) fetch_diag(i0 + 32, min(32, n - i0 - 32));
    int r0 = i0 + ib;
    if (r0 < n) fetch(r0, n, i0, ib);
    __syncthreads();
    diag_fwd(i0, ib);
    for (; r0 < n; r0 += CH) {
      stash();
      __syncthreads();
      if (r0 + CH < n) fetch(r0 + CH, n, i0, ib);
      update(r0, min(r0 + CH, n), i0, ib);
      __syncthreads();
    }
    __syncthreads();
  }
  // ---- backward: U x = y
  {
    const int il = ((n - 1) / 32) * 32;
    fetch_diag(il, n - il);
  }
  for (int i0 = ((n - 1) / 32) * 32; i0 >= 0; i0 -= 32) {
    const int ib = min(32, n - i0);
    stash_diag();
    if (i0 > 0) fetch_diag(i0 - 32, 32);
    if (i0 > 0) fetch(0, i0, i0, ib);
    __syncthreads();
    diag_bwd(i0, ib);
    for (int r0 = 0; r0 < i0; r0 += CH) {
      stash();
      __syncthreads();
      if (r0 + CH < i0) fetch(r0 + CH, i0, i0, ib);
      update(r0, min(r0 + CH, i0), i0, ib);
      __syncthreads();
    }
    __syncthreads();
  }
  if constexpr (XT) {
    for (int i = tid; i < n * RC; i += blockDim.x) {
      const int c = i / n, r = i % n;
      if (c < rc) X[(size_t)(c0 + c) * n + r] = x[(size_t)r * RC + c];
    }
  } else {
    for (int i = tid; i < n * RC; i += blockDim.x) {
      int r = i / RC, c = i % RC;
      if (c < rc) X[(size_t)r * nrhs + c0 + c] = x[i];
    }
  }
}
