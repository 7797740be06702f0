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

#include "tc_gemm.cuh"

constexpr int LU_NT = 256;
constexpr int LU_NB = 32;
constexpr int LU_TM = 64;

template <class T>
inline size_t lu_smem_bytes(int n) {
  (void)n;
  return sizeof(T) * ((size_t)LU_TM * (LU_NB + 1) + (size_t)LU_NB * (LU_TM + 1));
}

// tensor-core trailing update (FP32 matrices): staging for a 128 x 32 tile of L21 and a
// 256 x 32 tile of U12^T in the canonical K-major layout (2 x hi/lo), then a 128 x 257
// result tile for the coalesced epilogue
constexpr int LUTC_BM = 128, LUTC_BN = 256;
constexpr size_t LUTC_STAGE = 2 * (size_t)(LUTC_BM + LUTC_BN) * 32 * 4;   // hi and lo parts
constexpr size_t LUTC_TILE = (size_t)LUTC_BM * (LUTC_BN + 1) * 4;
inline size_t lu_tc_smem_bytes() { return LUTC_STAGE + LUTC_TILE + 1024; }

// A22[0:m2, 0:m2] -= L21 U12 with split TF32 (hi*hi + hi*lo + lo*hi) on tcgen05, called by
// all threads of the CTA; L21 = A + (c0)*n + j0, U12 = A + j0*n + c0, A22 = A + c0*n + c0.
__device__ __forceinline__ bool lu_tc_update(float* A, int n, int j0, int jb, int c0, unsigned char* smem,
                                             uint32_t tmem, uint64_t* bar, uint32_t& phase) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m2 = n - c0;
  unsigned char* sAh = smem;
  unsigned char* sAl = sAh + LUTC_BM * 32 * 4;
  unsigned char* sBh = sAl + LUTC_BM * 32 * 4;
  unsigned char* sBl = sBh + LUTC_BN * 32 * 4;
  float* tile = reinterpret_cast<float*>(smem + LUTC_STAGE);
  bool ok = true;
  for (int ti = 0; ti < m2; ti += LUTC_BM) {
    // L21 tile: rows c0+ti.., columns j0..j0+jb (zero beyond)
    for (int i = tid; i < LUTC_BM * 32; i += blockDim.x) {
      int r = i >> 5, k = i & 31;
      float v = (ti + r < m2 && k < jb) ? A[(size_t)(c0 + ti + r) * n + j0 + k] : 0.f;
      float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
      uint32_t off = tc::canon_off(r, k);
      *reinterpret_cast<float*>(sAh + off) = hi;
      *reinterpret_cast<float*>(sAl + off) = v - hi;
    }
    for (int tj = 0; tj < m2; tj += LUTC_BN) {
      for (int i = tid; i < LUTC_BN * 32; i += blockDim.x) {
        int k = i / LUTC_BN, c = i % LUTC_BN;
        float v = (tj + c < m2 && k < jb) ? A[(size_t)(j0 + k) * n + c0 + tj + c] : 0.f;
        float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        uint32_t off = tc::canon_off(c, k);
        *reinterpret_cast<float*>(sBh + off) = hi;
        *reinterpret_cast<float*>(sBl + off) = v - hi;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = tc::smem_u32(sAh), al = tc::smem_u32(sAl), bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            uint64_t ad = tc::desc_kmajor((t == 2 ? al : ah) + kk * 256, 128, 1024);
            uint64_t bd = tc::desc_kmajor((t == 1 ? bl : bh) + kk * 256, 128, 1024);
            uint32_t accum = (kk > 0 || t > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(tc::idesc_tf32(LUTC_BM, LUTC_BN)), "r"(accum)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tc::smem_u32(bar))
                     : "memory");
      }
      if (!tc::mbar_wait(bar, phase)) ok = false;
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // TMEM -> tile: warp w reads lanes 32 (w % 4).., columns (w / 4) * 128 ..
      {
        const int lrow = (warp & 3) * 32 + lane;
        const int cbase = (warp >> 2) * (LUTC_BN / 2);
#pragma unroll 1
        for (int cc = 0; cc < LUTC_BN / 2; cc += 16) {
          uint32_t r[16];
          const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(cbase + cc);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j) tile[lrow * (LUTC_BN + 1) + cbase + cc + j] = __uint_as_float(r[j]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      const int rows = min(LUTC_BM, m2 - ti), cols = min(LUTC_BN, m2 - tj);
      for (int i = tid; i < rows * LUTC_BN; i += blockDim.x) {
        int rr = i / LUTC_BN, cc = i % LUTC_BN;
        if (cc < cols) A[(size_t)(c0 + ti + rr) * n + c0 + tj + cc] -= tile[rr * (LUTC_BN + 1) + cc];
      }
      __syncthreads();
    }
  }
  return ok;
}

template <class T, bool TC = false>
__global__ void __launch_bounds__(LU_NT) k_lu_batched(T* __restrict__ Aall, int* __restrict__ permall, int n,
                                                     int* __restrict__ flag, int* __restrict__ tcerr = nullptr) {
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
  __shared__ __align__(8) uint64_t tc_bar;
  __shared__ uint32_t tc_slot;
  uint32_t tc_phase = 0;
  bool tc_ok = true;
  if (TC) {
    if (tid == 0) {
      tc::mbar_init(&tc_bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tc_slot)),
                   "r"(256u)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  for (int i = tid; i < n; i += LU_NT) perm[i] = i;
  __syncthreads();
  if (TC) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
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
    if constexpr (TC) {
      if (!lu_tc_update(reinterpret_cast<float*>(A), n, j0, jb, c0, lu_smem_raw, tc_slot, &tc_bar, tc_phase))
        tc_ok = false;
      continue;
    }
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
  if (TC) {
    if (!tc_ok && tid == 0) atomicExch(tcerr, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc_slot), "r"(256u) : "memory");
  }
}

// y <- U^-1 L^-1 y for factors LU (row-major, unit L), y already permuted (P y).
// Called by all threads of the CTA; y in shared memory; arithmetic in Acc.
template <class T, class Acc = double>
__device__ void lu_solve_block(const T* __restrict__ LU, int n, Acc* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int ib = min(32, n - i0);
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
      for (int r = 1; r < ib; ++r) {
        Acc v = (lane < r) ? (Acc)LU[(size_t)(i0 + r) * n + i0 + lane] * y[i0 + lane] : Acc(0);
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) y[i0 + r] -= v;
        __syncwarp();
      }
    }
    __syncthreads();
  }
  for (int i0 = ((n - 1) / 32) * 32; i0 >= 0; i0 -= 32) {
    const int ib = min(32, n - i0);
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
      for (int r = ib - 1; r >= 0; --r) {
        Acc v = (lane > r && lane < ib) ? (Acc)LU[(size_t)(i0 + r) * n + i0 + lane] * y[i0 + lane] : Acc(0);
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) y[i0 + r] = (y[i0 + r] - v) / (Acc)LU[(size_t)(i0 + r) * n + i0 + r];
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

// X = S^-1 B for a block of RC right-hand-side columns of one macro-element
// (grid: macro x column block), from the LU factors and row permutation of S.
// B and X are row-major [n][nrhs]; the RC columns live in shared memory.  Blocked
// substitution: for each 32-row block the update from the solved rows is a small
// GEMM (32 x done) x (done x RC) with 32 x 32 tiles of L or U staged in shared
// memory and 8 outputs per thread in registers; then the 32 x 32 diagonal block is
// solved column by column (one thread per right-hand side).
// B == nullptr solves for the identity (columns of S^-1).
template <class T, int RC>
__global__ void __launch_bounds__(256) k_lu_solve_multi(const T* __restrict__ LUall, const int* __restrict__ permall,
                                                       const T* __restrict__ Ball, T* __restrict__ Xall, int n,
                                                       int nrhs) {
  static_assert(RC % 8 == 0 && RC <= 256, "RC");
  constexpr int OPT = 32 * RC / 256;   // outputs per thread in a 32-row block
  extern __shared__ unsigned char lum_raw[];
  T* x = reinterpret_cast<T*>(lum_raw);   // [n][RC]
  __shared__ T lt[32][33];
  const int e = blockIdx.x, c0 = blockIdx.y * RC;
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
  __syncthreads();
  // thread layout of the block update: row rr = tid / (256/32) ... 32 rows x RC columns
  constexpr int TPR = 256 / 32;          // threads per row
  const int rr = tid / TPR, cq = tid % TPR;
  auto block_update = [&](int i0, int ib, int j_begin, int j_end) {
    T acc[OPT];
#pragma unroll
    for (int o = 0; o < OPT; ++o) acc[o] = T(0);
    for (int jb = j_begin; jb < j_end; jb += 32) {
      const int jl = min(32, j_end - jb);
      for (int i = tid; i < 32 * 32; i += blockDim.x) {
        int a = i / 32, b = i % 32;
        lt[a][b] = (a < ib && b < jl) ? LU[(size_t)(i0 + a) * n + jb + b] : T(0);
      }
      __syncthreads();
      for (int q = 0; q < jl; ++q) {
        const T l = lt[rr][q];
        const T* xr = x + (size_t)(jb + q) * RC;
#pragma unroll
        for (int o = 0; o < OPT; ++o) acc[o] += l * xr[cq + TPR * o];
      }
      __syncthreads();
    }
    if (rr < ib) {
      T* xo = x + (size_t)(i0 + rr) * RC;
#pragma unroll
      for (int o = 0; o < OPT; ++o) xo[cq + TPR * o] -= acc[o];
    }
    __syncthreads();
  };
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int ib = min(32, n - i0);
    if (i0 > 0) block_update(i0, ib, 0, i0);
    for (int cc = tid; cc < RC; cc += blockDim.x)
      for (int r = 1; r < ib; ++r) {
        const T* row = LU + (size_t)(i0 + r) * n + i0;
        T s = T(0);
        for (int q = 0; q < r; ++q) s += row[q] * x[(i0 + q) * RC + cc];
        x[(i0 + r) * RC + cc] -= s;
      }
    __syncthreads();
  }
  for (int i0 = ((n - 1) / 32) * 32; i0 >= 0; i0 -= 32) {
    const int ib = min(32, n - i0);
    if (i0 + ib < n) block_update(i0, ib, i0 + ib, n);
    for (int cc = tid; cc < RC; cc += blockDim.x)
      for (int r = ib - 1; r >= 0; --r) {
        const T* row = LU + (size_t)(i0 + r) * n;
        T s = T(0);
        for (int q = r + 1; q < ib; ++q) s += row[i0 + q] * x[(i0 + q) * RC + cc];
        x[(i0 + r) * RC + cc] = (x[(i0 + r) * RC + cc] - s) / row[i0 + r];
      }
    __syncthreads();
  }
  for (int i = tid; i < n * RC; i += blockDim.x) {
    int r = i / RC, c = i % RC;
    if (c < rc) X[(size_t)r * nrhs + c0 + c] = x[i];
  }
}

