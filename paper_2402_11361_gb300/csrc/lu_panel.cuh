// Batched dense LU with partial pivoting, P A = L U (first maximal |.| row wins ties),
// the factorisation of each Schur complement S that the trace apply and recovery use
// through substitution (Remark, Sec. 3.3).  One CTA factors one matrix (row-major, in
// place; perm[i] = original row now at position i, rows swapped over their full length).
//
// Right-looking blocked form with panel width 32:
//  1. the panel (rows j0..n-1, columns j0..j0+31) is copied to shared memory and
//     factored there: per column one look-ahead pivot search fused into the previous
//     column's elimination, so two barriers per column and no global-memory chains;
//  2. the panel's row swaps are composed into one net permutation of at most 64 rows
//     (warp 0, shuffles), applied to the perm vector and, one thread per column, to
//     every column outside the panel: all loads of a column are issued before its
//     stores, so the swaps cost one round trip instead of 32 dependent ones;
//  3. in the same pass the thread of a trailing column solves its 32 entries of the
//     block row U12 = L11^-1 (P A12) in registers (L11 read from shared memory);
//  4. trailing update A22 -= L21 U12, L21 read from the shared-memory panel: either
//     SIMT 64 x 64 tiles (FP32 or FP64), or, for FP32 matrices, tcgen05 MMAs
//     (kind::tf32, 128 x 256 tiles, operands split hi + lo so that hi*hi + hi*lo +
//     lo*hi keeps FP32 accuracy) with the accumulator in tensor memory, read back by
//     tcgen05.ld and subtracted from A22 in place.
// Every mbarrier wait is bounded; on timeout the kernel records an error word and
// still releases its tensor memory.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "tc_gemm.cuh"

constexpr int LP_NT = 256;            // threads per CTA
constexpr int LP_NB = 32;             // panel width
constexpr int LP_LDP = LP_NB + 1;     // panel row stride in shared memory
constexpr int LP_TM = 64;             // SIMT update tile
constexpr int LPTC_BM = 128, LPTC_BN = 256;

template <class T, bool TC, int NB = LP_NB>
inline size_t lu_panel_smem(int n) {
  size_t p = (sizeof(T) * (size_t)n * (NB + 1) + 127) / 128 * 128;
  if (TC) return p + (size_t)2 * (LPTC_BM + LPTC_BN) * 32 * 4;
  return p + sizeof(T) * (size_t)NB * (LP_TM + 1);
}

template <class T>
__device__ __forceinline__ void lp_warp_argmax(T& bv, int& bi) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
}

// A22 -= L21 U12 on tcgen05 for one panel step (FP32 matrix); all threads of the CTA.
// L21 = rows jb.. of the shared-memory panel, U12 = rows j0..j0+31 of A (already solved).
__device__ __forceinline__ bool lp_tc_update(float* A, int n, int j0, int c0, const float* sP, unsigned char* sX,
                                             uint32_t tmem, uint64_t* bar, uint32_t& phase) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m2 = n - c0, jb = LP_NB;
  unsigned char* sAh = sX;
  unsigned char* sAl = sAh + LPTC_BM * 32 * 4;
  unsigned char* sBh = sAl + LPTC_BM * 32 * 4;
  unsigned char* sBl = sBh + LPTC_BN * 32 * 4;
  for (int ti = 0; ti < m2; ti += LPTC_BM) {
    // L21 tile [128 x 32] from the panel; lanes cover an 8-row x 4-column core-matrix patch
    for (int i = tid; i < LPTC_BM * 32; i += LP_NT) {
      const int kq = i & 3, rl = (i >> 2) & 7, kh = (i >> 5) & 7, rh = i >> 8;
      const int r = rh * 8 + rl, k = kh * 4 + kq;
      const float v = (ti + r < m2) ? sP[(jb + ti + r) * LP_LDP + k] : 0.f;
      const float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
      const uint32_t off = (uint32_t)(rh * 1024 + kh * 128 + rl * 16 + kq * 4);
      *reinterpret_cast<float*>(sAh + off) = hi;
      *reinterpret_cast<float*>(sAl + off) = v - hi;
    }
    for (int tj = 0; tj < m2; tj += LPTC_BN) {
      // U12^T tile [256 x 32] (K-major): lanes read 8 consecutive columns of 4 rows
      for (int i = tid; i < LPTC_BN * 32; i += LP_NT) {
        const int kq = i & 3, cl = (i >> 2) & 7, kh = (i >> 5) & 7, ch = i >> 8;
        const int c = ch * 8 + cl, k = kh * 4 + kq;
        const float v = (tj + c < m2) ? A[(size_t)(j0 + k) * n + c0 + tj + c] : 0.f;
        const float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        const uint32_t off = (uint32_t)(ch * 1024 + kh * 128 + cl * 16 + kq * 4);
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
            const uint64_t ad = tc::desc_kmajor((t == 2 ? al : ah) + kk * 256, 128, 1024);
            const uint64_t bd = tc::desc_kmajor((t == 1 ? bl : bh) + kk * 256, 128, 1024);
            const uint32_t accum = (kk > 0 || t > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(tc::idesc_tf32(LPTC_BM, LPTC_BN)), "r"(accum)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tc::smem_u32(bar))
                     : "memory");
      }
      if (!__syncthreads_and(tc::mbar_wait(bar, phase))) {
        // a wait ran out: issue nothing more, wait once more (bounded) for the MMAs of this
        // commit to finish with TMEM and shared memory, and report the failure; the caller
        // abandons the factorisation and releases TMEM
        tc::mbar_wait(bar, phase);
        phase ^= 1;
        return false;
      }
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // warp w reads TMEM lanes 32 (w % 4).. (rows) and accumulator columns (w / 4) * 128 ..
      const int row = ti + (warp & 3) * 32 + lane;
      const int cbase = (warp >> 2) * (LPTC_BN / 2);
      float* Arow = A + (size_t)(c0 + min(row, m2 - 1)) * n + c0 + tj;
#pragma unroll 1
      for (int cc = 0; cc < LPTC_BN / 2; cc += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(cbase + cc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < m2) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = cbase + cc + j;
            if (tj + col < m2) Arow[col] -= __uint_as_float(r[j]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  return true;
}

// One CTA factors the n x n matrix A in place with panel width NB (8, 16 or 32; the
// tcgen05 update needs 32).  A zero pivot sets flag[0] and flag[1] = tag.  The panel is
// staged in the dynamic shared memory lp_raw (lu_panel_smem<T, TC, NB>(n) bytes).
template <class T, bool TC, int NB>
__device__ __forceinline__ void lp_factor(T* __restrict__ A, int* __restrict__ perm, int n, int* __restrict__ flag,
                                          int* __restrict__ tcerr, int tag, unsigned char* lp_raw) {
  static_assert(NB == 8 || NB == 16 || NB == 32, "panel width");
  static_assert(!TC || NB == 32, "the tcgen05 update takes 32-wide panels");
  constexpr int LP_LDP = NB + 1;
  T* sP = reinterpret_cast<T*>(lp_raw);   // [n][NB + 1], rows j0.. of the current panel
  unsigned char* sX = lp_raw + (sizeof(T) * (size_t)n * LP_LDP + 127) / 128 * 128;
  __shared__ T rv[LP_NT / 32];   // pivot candidates, compared in the matrix's own precision
  __shared__ int ri[LP_NT / 32];
  __shared__ int spiv[NB];
  __shared__ int topsrc[NB], xsrc[NB], xdst[NB];
  __shared__ int nxs;
  __shared__ __align__(8) uint64_t tc_bar;
  __shared__ uint32_t tc_slot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t tc_phase = 0;
  bool tc_ok = true;
  if constexpr (TC) {
    if (tid == 0) {
      tc::mbar_init(&tc_bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tc_slot)),
                   "r"((uint32_t)LPTC_BN)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  for (int i = tid; i < n; i += LP_NT) perm[i] = i;
  __syncthreads();
  if constexpr (TC) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  for (int j0 = 0; j0 < n; j0 += NB) {
    const int jb = min(NB, n - j0), m = n - j0, c0 = j0 + jb;
    // ---- 1. panel to shared memory, factor it there
    for (int idx = tid; idx < m * NB; idx += LP_NT) {
      const int r = idx / NB, c = idx % NB;
      sP[r * LP_LDP + c] = (c < jb) ? A[(size_t)(j0 + r) * n + j0 + c] : T(0);
    }
    __syncthreads();
    {
      T bv = T(-1);
      int bi = m;
      for (int i = tid; i < m; i += LP_NT) {
        const T v = fabs(sP[i * LP_LDP]);
        if (v > bv) { bv = v; bi = i; }
      }
      lp_warp_argmax(bv, bi);
      if (lane == 0) { rv[warp] = bv; ri[warp] = bi; }
    }
    __syncthreads();
    for (int j = 0; j < jb; ++j) {
      T b = rv[0];
      int r = ri[0];
#pragma unroll
      for (int w = 1; w < LP_NT / 32; ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < r)) { b = rv[w]; r = ri[w]; }
      if (r >= m) r = j;   // no finite candidate (NaN column): keep the row
      if (tid == 0) {
        spiv[j] = r;
        if (b == T(0) && atomicCAS(flag, 0, 1) == 0) flag[1] = tag;
      }
      if (r != j && tid < NB) {
        const T t = sP[j * LP_LDP + tid];
        sP[j * LP_LDP + tid] = sP[r * LP_LDP + tid];
        sP[r * LP_LDP + tid] = t;
      }
      __syncthreads();
      const T piv = sP[j * LP_LDP + j];
      const T inv = (piv != T(0)) ? T(1) / piv : T(0);
      T bv = T(-1);
      int bi = m;
      for (int i = j + 1 + tid; i < m; i += LP_NT) {
        T* row = sP + i * LP_LDP;
        const T l = row[j] * inv;
        row[j] = l;
        for (int c = j + 1; c < jb; ++c) row[c] -= l * sP[j * LP_LDP + c];
        if (j + 1 < jb) {
          const T v = fabs(row[j + 1]);
          if (v > bv) { bv = v; bi = i; }
        }
      }
      lp_warp_argmax(bv, bi);
      if (lane == 0) { rv[warp] = bv; ri[warp] = bi; }
      __syncthreads();
    }
    // ---- 2. net permutation of the panel's swaps: slot k < jb is row j0 + k; rows below
    // the panel that a swap touched get extra slots (keyed by row)
    if (warp == 0) {
      int content = lane, xkey = -1, xcontent = -1, nx = 0;
      for (int j = 0; j < jb; ++j) {
        const int r = spiv[j];
        if (r == j) continue;
        const int cj = __shfl_sync(0xffffffffu, content, j);
        int cr;
        if (r < NB) {
          cr = __shfl_sync(0xffffffffu, content, r);
          if (lane == r) content = cj;
        } else {
          const unsigned hit = __ballot_sync(0xffffffffu, xkey == r);
          if (hit) {
            const int src = __ffs(hit) - 1;
            cr = __shfl_sync(0xffffffffu, xcontent, src);
            if (lane == src) xcontent = cj;
          } else {
            cr = r;
            if (lane == nx) { xkey = r; xcontent = cj; }
            ++nx;
          }
        }
        if (lane == j) content = cr;
      }
      if (lane < jb) topsrc[lane] = content;
      if (lane < nx) { xdst[lane] = xkey; xsrc[lane] = xcontent; }
      if (lane == 0) nxs = nx;
    }
    __syncthreads();
    const int nx = nxs;
    if (warp == 0) {
      const int pv = lane < jb ? perm[j0 + topsrc[lane]] : 0;
      const int px = lane < nx ? perm[j0 + xsrc[lane]] : 0;
      __syncwarp();
      if (lane < jb) perm[j0 + lane] = pv;
      if (lane < nx) perm[j0 + xdst[lane]] = px;
    }
    // panel back to global memory
    for (int idx = tid; idx < m * NB; idx += LP_NT) {
      const int r = idx / NB, c = idx % NB;
      if (c < jb) A[(size_t)(j0 + r) * n + j0 + c] = sP[r * LP_LDP + c];
    }
    // ---- 3. swaps outside the panel, and U12 = L11^-1 (P A12) for trailing columns
    for (int cidx = tid; cidx < n - jb; cidx += LP_NT) {
      const int col = (cidx < j0) ? cidx : cidx + jb;
      T* Ac = A + col;
      T u[NB], x[NB];
#pragma unroll
      for (int k = 0; k < NB; ++k) u[k] = (k < jb) ? Ac[(size_t)(j0 + topsrc[k]) * n] : T(0);
#pragma unroll
      for (int k = 0; k < NB; ++k) x[k] = (k < nx) ? Ac[(size_t)(j0 + xsrc[k]) * n] : T(0);
      const bool trailing = col >= c0;
      if (trailing) {   // here jb == NB
#pragma unroll
        for (int r = 1; r < NB; ++r) {
          T s = u[r];
#pragma unroll
          for (int q = 0; q < r; ++q) s -= sP[r * LP_LDP + q] * u[q];
          u[r] = s;
        }
      }
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (k < jb && (trailing || topsrc[k] != k)) Ac[(size_t)(j0 + k) * n] = u[k];
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (k < nx) Ac[(size_t)(j0 + xdst[k]) * n] = x[k];
    }
    __syncthreads();
    if (c0 >= n) break;
    // ---- 4. trailing update A22 -= L21 U12
    if constexpr (TC) {
      if (!lp_tc_update(reinterpret_cast<float*>(A), n, j0, c0, reinterpret_cast<const float*>(sP), sX, tc_slot,
                        &tc_bar, tc_phase)) {
        tc_ok = false;   // uniform across the CTA: stop here, the factors are discarded by the host
        break;
      }
    } else {
      T* sU = reinterpret_cast<T*>(sX);   // [NB][LP_TM + 1]
      const int m2 = n - c0;
      const int tx = tid % 16, ty = tid / 16;
      const int nt = (m2 + LP_TM - 1) / LP_TM, ntiles = nt * nt;
      constexpr int RU = NB * LP_TM / LP_NT;
      T ru[RU];
      // U12 tile (32 x 64) of column block tj into registers
      auto fetch_u = [&](int tj) {
#pragma unroll
        for (int j = 0; j < RU; ++j) {
          const int i = tid + LP_NT * j, rr = i / LP_TM, cc = i % LP_TM;
          const int gc = c0 + tj + cc;
          ru[j] = (gc < n) ? A[(size_t)(j0 + rr) * n + gc] : T(0);
        }
      };
      fetch_u(0);
      for (int t = 0; t < ntiles; ++t) {
        const int ti = (t / nt) * LP_TM, tj = (t % nt) * LP_TM;
        // the 4 x 4 entries of A22 this thread updates, loaded before the product
        T a22[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int gr = c0 + ti + ty + 16 * a, gc = c0 + tj + tx + 16 * b;
            a22[a][b] = (gr < n && gc < n) ? A[(size_t)gr * n + gc] : T(0);
          }
#pragma unroll
        for (int j = 0; j < RU; ++j) {
          const int i = tid + LP_NT * j;
          sU[(i / LP_TM) * (LP_TM + 1) + i % LP_TM] = ru[j];
        }
        __syncthreads();
        if (t + 1 < ntiles) fetch_u(((t + 1) % nt) * LP_TM);
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
        int prow[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) prow[a] = min(jb + ti + ty + 16 * a, m - 1) * LP_LDP;
#pragma unroll 8
        for (int kk = 0; kk < NB; ++kk) {
          T lv[4], uv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) lv[a] = sP[prow[a] + kk];
#pragma unroll
          for (int b = 0; b < 4; ++b) uv[b] = sU[kk * (LP_TM + 1) + tx + 16 * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += lv[a] * uv[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int gr = c0 + ti + ty + 16 * a, gc = c0 + tj + tx + 16 * b;
            if (gr < n && gc < n) A[(size_t)gr * n + gc] = a22[a][b] - acc[a][b];
          }
        __syncthreads();
      }
    }
  }
  if constexpr (TC) {
    if (!tc_ok && tid == 0 && tcerr) atomicExch(tcerr, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc_slot), "r"((uint32_t)LPTC_BN)
                   : "memory");
  }
}

template <class T, bool TC>
__global__ void __launch_bounds__(LP_NT, (sizeof(T) == 4 && !TC) ? 2 : 1)
    k_lu_panel_smem(T* __restrict__ Aall, int* __restrict__ permall, int n, int* __restrict__ flag,
                    int* __restrict__ tcerr) {
  extern __shared__ __align__(128) unsigned char lp_raw[];
  lp_factor<T, TC, LP_NB>(Aall + (size_t)blockIdx.x * n * n, permall + (size_t)blockIdx.x * n, n, flag, tcerr,
                          blockIdx.x + 1, lp_raw);
}

// Work queue of matrices of uneven size (the batching of independent problems): item i is
// the n_i x n_i matrix A_i with pivot vector perm_i, factored with panel width nb_i (chosen
// per size by the batch's autotuner); a zero pivot sets flag_i[0] and flag_i[1] = tag_i.
struct LuItem {
  void* A;
  int* perm;
  int* flag;
  int n, nb, tag, pad;
};

// Persistent: the grid is sized to the GPU (SMs x resident CTAs), each CTA takes the next item
// from the counter (items sorted largest first) until the queue is empty.  No waiting: the
// counter only grows, so every CTA leaves after at most nitems + 1 fetches.
// (FP32: two CTAs per SM, as k_lu_panel_smem<float>, when the largest panel leaves room)
template <class T>
__global__ void __launch_bounds__(LP_NT, sizeof(T) == 4 ? 2 : 1)
    k_lu_queue(const LuItem* __restrict__ items, int nitems, int* __restrict__ counter) {
  extern __shared__ __align__(128) unsigned char lq_raw[];
  __shared__ int it;
  for (;;) {
    if (threadIdx.x == 0) it = atomicAdd(counter, 1);
    __syncthreads();
    const int i = it;
    __syncthreads();
    if (i >= nitems) break;
    const LuItem w = items[i];
    T* A = static_cast<T*>(w.A);
    if (w.nb == 8) lp_factor<T, false, 8>(A, w.perm, w.n, w.flag, nullptr, w.tag, lq_raw);
    else if (w.nb == 16) lp_factor<T, false, 16>(A, w.perm, w.n, w.flag, nullptr, w.tag, lq_raw);
    else lp_factor<T, false, 32>(A, w.perm, w.n, w.flag, nullptr, w.tag, lq_raw);
    __syncthreads();
  }
}
