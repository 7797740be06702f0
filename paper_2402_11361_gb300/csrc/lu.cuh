// Batched dense LU with partial pivoting (P A = L U, first maximal |.| row wins ties)
// and the matching forward/back substitution for one CTA.  The paper stores a
// factorisation of each Schur complement S and applies S^-1 by substitution
// (Remark, Sec. 3.3); here one CTA factors one matrix held in global memory:
// unblocked panel of width LU_NB with row swaps over whole rows, triangular solve
// for the block row of U, then a tiled rank-LU_NB update of the trailing matrix.
#pragma once
#include <cuda_runtime.h>

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
// Called by all threads of the CTA; y in shared memory; arithmetic in double.
template <class T>
__device__ void lu_solve_block(const T* __restrict__ LU, int n, double* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int ib = min(32, n - i0);
    for (int r = warp; r < ib; r += nw) {
      const T* row = LU + (size_t)(i0 + r) * n;
      double s = 0.0;
      for (int c = lane; c < i0; c += 32) s += (double)row[c] * y[c];
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) y[i0 + r] -= s;
    }
    __syncthreads();
    if (warp == 0) {
      for (int r = 1; r < ib; ++r) {
        double v = (lane < r) ? (double)LU[(size_t)(i0 + r) * n + i0 + lane] * y[i0 + lane] : 0.0;
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
      double s = 0.0;
      for (int c = i0 + ib + lane; c < n; c += 32) s += (double)row[c] * y[c];
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) y[i0 + r] -= s;
    }
    __syncthreads();
    if (warp == 0) {
      for (int r = ib - 1; r >= 0; --r) {
        double v = (lane > r && lane < ib) ? (double)LU[(size_t)(i0 + r) * n + i0 + lane] * y[i0 + lane] : 0.0;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) y[i0 + r] = (y[i0 + r] - v) / (double)LU[(size_t)(i0 + r) * n + i0 + r];
        __syncwarp();
      }
    }
    __syncthreads();
  }
}
