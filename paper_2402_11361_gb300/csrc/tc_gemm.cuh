// Batched GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32), for the
// dense local products of the mixed-precision path:
//   C[b] = alpha * A[b] * B[b] + beta * C[b],  A [M x K], B [K x N], C [M x N] row-major FP32,
// any leading dimensions and batch strides (b = (i, j), X[b] = X + i*sX1 + j*sX2).
//
// One CTA (4 warps) computes a 128 x BN tile.  Each K block of 32 is staged by the
// threads into shared memory in the canonical K-major, non-swizzled tcgen05 layout
// (8-row x 16-byte core matrices: LBO = 128 B between core matrices along K,
// SBO = 1024 B between 8-row groups), so operands need no alignment and B is
// transposed for free while staging.  Thread 0 issues four 128 x BN x 8 MMAs per
// K block into a TMEM accumulator and commits them to the stage's mbarrier; the
// next K block is staged meanwhile (two stages).  The epilogue reads TMEM with
// tcgen05.ld (warp w owns lanes 32w..32w+31 = rows) and writes alpha*acc + beta*C.
// Every mbarrier wait is bounded; on timeout the CTA stops issuing MMAs, waits once more
// (bounded) on a commit covering all MMAs it issued, records an error word, skips the
// epilogue and releases its TMEM.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

struct TcArgs {
  int M, N, K;
  const float* A; long long lda, sA1, sA2;
  const float* B; long long ldb, sB1, sB2;
  float* C; long long ldc, sC1, sC2;
  float alpha, beta;
  int n2;
  int* err;   // device error word (set to 1 on a timed-out wait)
};

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: false after `limit` unsuccessful polls (each poll may suspend briefly)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = 4000000) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of tcgen05; base offset 0, no swizzle
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, shape M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) of a [rows x 32] FP32 tile in the canonical layout
__device__ __forceinline__ uint32_t canon_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

}  // namespace tc

template <int BN, bool SPLIT>
__global__ void __launch_bounds__(128) k_tc_gemm_tf32(TcArgs a) {
  constexpr int BM = 128, BK = 32;
  constexpr int A_BYTES = BM * BK * 4;   // 16 KB
  constexpr int B_BYTES = BN * BK * 4;
  constexpr int NP = SPLIT ? 2 : 1;      // hi (and lo) parts per operand
  constexpr int STAGE = NP * (A_BYTES + B_BYTES);
  constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[3];
  __shared__ uint32_t tmem_slot;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.z;
  const int bi = b / a.n2, bj = b % a.n2;
  const float* A = a.A + bi * a.sA1 + bj * a.sA2;
  const float* B = a.B + bi * a.sB1 + bj * a.sB2;
  float* C = a.C + bi * a.sC1 + bj * a.sC2;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_init(&bar[2], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  const int nkb = (a.K + BK - 1) / BK;
  bool ok = true;
  uint32_t phase[2] = {0, 0};
  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb & 1;
    unsigned char* sA = smem + s * STAGE;           // [hi, lo] parts of A, then of B
    unsigned char* sB = sA + NP * A_BYTES;
    if (kb >= 2) {   // the MMAs of K block kb-2 read this stage
      if (!tc::mbar_wait(&bar[s], phase[s])) ok = false;
      phase[s] ^= 1;
    }
    const int k0 = kb * BK;
#pragma unroll 4
    for (int i = 0; i < (BM * BK) / 128; ++i) {
      int idx = i * 128 + tid;
      int r = idx >> 5, k = idx & 31;
      int gr = m0 + r, gk = k0 + k;
      float v = (gr < a.M && gk < a.K) ? A[(size_t)gr * a.lda + gk] : 0.f;
      const uint32_t off = tc::canon_off(r, k);
      if (SPLIT) {
        float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        *reinterpret_cast<float*>(sA + off) = hi;
        *reinterpret_cast<float*>(sA + A_BYTES + off) = v - hi;
      } else {
        *reinterpret_cast<float*>(sA + off) = v;
      }
    }
#pragma unroll 4
    for (int i = 0; i < (BN * BK) / 128; ++i) {
      int idx = i * 128 + tid;
      int k = idx / BN, n = idx % BN;
      int gk = k0 + k, gn = n0 + n;
      float v = (gk < a.K && gn < a.N) ? B[(size_t)gk * a.ldb + gn] : 0.f;
      const uint32_t off = tc::canon_off(n, k);
      if (SPLIT) {
        float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        *reinterpret_cast<float*>(sB + off) = hi;
        *reinterpret_cast<float*>(sB + B_BYTES + off) = v - hi;
      } else {
        *reinterpret_cast<float*>(sB + off) = v;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // a timed-out wait stops the K loop for the whole CTA: no further MMAs are issued
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ahi = tc::smem_u32(sA), bhi = tc::smem_u32(sB);
      const uint32_t alo = ahi + A_BYTES, blo = bhi + B_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        const uint32_t ko = kk * 256;
        uint32_t accum = (kb > 0 || kk > 0) ? 1u : 0u;
        const int nterms = SPLIT ? 3 : 1;
#pragma unroll
        for (int t = 0; t < nterms; ++t) {
          const uint32_t aa = (t == 2 ? alo : ahi) + ko, bb = (t == 1 ? blo : bhi) + ko;
          uint64_t ad = tc::desc_kmajor(aa, 128, 1024);
          uint64_t bd = tc::desc_kmajor(bb, 128, 1024);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(tc::idesc_tf32(BM, BN)), "r"(t > 0 ? 1u : accum)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc::smem_u32(&bar[s]))
                   : "memory");
    }
  }
  // this commit tracks every MMA the CTA issued, also after an early stop: its bounded
  // wait is the wait for the work still in flight before TMEM is released
  if (tid == 0) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc::smem_u32(&bar[2]))
                 : "memory");
  }
  if (!tc::mbar_wait(&bar[2], 0)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = __syncthreads_and(ok) != 0;   // uniform decision for the warp-collective loads
  if (ok) {
    // TMEM -> shared tile [128][BN+1] (all MMAs are done, the staging buffers are free)
    float* tile = reinterpret_cast<float*>(smem);
    const int trow = warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) tile[trow * (BN + 1) + c0 + j] = __uint_as_float(r[j]);
    }
    __syncthreads();
    // coalesced read-modify-write of C: consecutive threads along a row
    const int rows = min(BM, a.M - m0), cols = min(BN, a.N - n0);
    for (int i = tid; i < rows * BN; i += 128) {
      const int rr = i / BN, cc = i % BN;
      if (cc < cols) {
        float* p = C + (size_t)(m0 + rr) * a.ldc + n0 + cc;
        const float v = a.alpha * tile[rr * (BN + 1) + cc];
        *p = (a.beta == 0.f) ? v : v + a.beta * *p;
      }
    }
  } else if (tid == 0) {
    atomicExch(a.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <int BN, bool SPLIT>
inline size_t tc_gemm_smem() {
  size_t stages = 2 * (size_t)(SPLIT ? 2 : 1) * (128 * 32 * 4 + BN * 32 * 4);
  size_t tile = (size_t)128 * (BN + 1) * 4;
  size_t need = (stages > tile ? stages : tile) + 1024;
  // at most two CTAs per SM so that their TMEM allocations always fit (512 columns)
  return need < 100 * 1024 ? 100 * 1024 : need;
}

// ---------------------------------------------------------------------------------------
// C_b = alpha A_b Bt_b^T + beta C_b on tcgen05 (kind::tf32, split into hi + lo TF32 parts, three
// products per term: about FP32 accuracy), A [M x K] and Bt [N x K] both row-major (K-major
// operands: the product of a block with the transpose of another, e.g. B (S^-1 C) with
// (S^-1 C) stored transposed), any leading dimension and batch stride (4-byte alignment only).
//
// Tiles of 128 x BN x 32: each operand row of 32 FP32 (128 bytes) goes to one row of the
// 128-byte-swizzled K-major layout (16-byte chunk c of row r at chunk c ^ (r mod 8); tile bases
// 1024-byte aligned), so a warp reading 32 consecutive K values of one row (one coalesced
// 128-byte load) writes 32 distinct banks.  The four warps stage the next K block (two stages)
// while thread 0 issues the 12 MMAs of the current one (4 K steps of 8, advancing the descriptor
// start by 32 bytes inside the swizzle row) into a TMEM accumulator and commits them to the
// stage's mbarrier.  Epilogue: TMEM -> shared tile -> coalesced read-modify-write of C.  Waits
// are bounded as in k_tc_gemm_tf32.
struct TcNT {
  int M, N, K;
  const float* A; long long lda, sA;
  const float* Bt; long long ldb, sB;
  float* C; long long ldc, sC;
  float alpha, beta;
  int* err;
};

namespace tc {
// K-major, 128-byte swizzle: LBO unused (1), SBO = 8 rows x 128 B, descriptor version 1,
// layout type 2 (128-byte swizzle) in bits 61..63
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__device__ __forceinline__ uint32_t sw128_off(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 2) ^ row) & 7) << 4) + (k & 3) * 4);
}
}  // namespace tc

template <int BN>
constexpr size_t tc_nt_smem() {
  return (size_t)2 * 2 * (128 + BN) * 128 + 1024;   // two stages of hi/lo A and Bt tiles, + alignment
}

constexpr int TCNT_THREADS = 256;   // eight warps stage a whole K block at once

template <int BN>
__global__ void __launch_bounds__(TCNT_THREADS, 1) k_tc_gemm_nt(TcNT a) {
  constexpr int BM = 128, BK = 32, NW = TCNT_THREADS / 32;
  constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128;
  constexpr int STAGE = 2 * (A_BYTES + B_BYTES);
  constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  extern __shared__ unsigned char nt_raw[];
  unsigned char* smem = nt_raw + ((1024 - (tc::smem_u32(nt_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar[3];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long b = blockIdx.z;
  const float* A = a.A + b * a.sA;
  const float* Bt = a.Bt + b * a.sB;
  float* C = a.C + b * a.sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_init(&bar[2], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // operand tiles: warp w takes rows w, w + 8, ... of the A (BM rows) and Bt (BN rows) tiles,
  // lane = K index.  The loads of K block kb + 1 are issued into registers right after K block
  // kb is stored, so they are in flight during the barrier, the MMA issue and the next wait.
  constexpr int PA = BM / NW, PB = BN / NW;
  float va[PA], vb[PB];
  auto load_regs = [&](int k0) {
    const int k = k0 + lane;
    const bool kin = k < a.K;
#pragma unroll
    for (int u = 0; u < PA; ++u) {
      const int gr = m0 + warp + NW * u;
      va[u] = (gr < a.M && kin) ? A[(size_t)gr * a.lda + k] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const int gr = n0 + warp + NW * u;
      vb[u] = (gr < a.N && kin) ? Bt[(size_t)gr * a.ldb + k] : 0.f;
    }
  };
  auto store_regs = [&](unsigned char* ahi, unsigned char* alo, unsigned char* bhi, unsigned char* blo) {
#pragma unroll
    for (int u = 0; u < PA; ++u) {
      const uint32_t off = tc::sw128_off(warp + NW * u, lane);
      const float h = __uint_as_float(__float_as_uint(va[u]) & 0xFFFFE000u);
      *reinterpret_cast<float*>(ahi + off) = h;
      *reinterpret_cast<float*>(alo + off) = va[u] - h;
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const uint32_t off = tc::sw128_off(warp + NW * u, lane);
      const float h = __uint_as_float(__float_as_uint(vb[u]) & 0xFFFFE000u);
      *reinterpret_cast<float*>(bhi + off) = h;
      *reinterpret_cast<float*>(blo + off) = vb[u] - h;
    }
  };

  const int nkb = (a.K + BK - 1) / BK;
  bool ok = true;
  uint32_t phase[2] = {0, 0};
  load_regs(0);
  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb & 1;
    unsigned char* sAh = smem + s * STAGE;
    unsigned char* sAl = sAh + A_BYTES;
    unsigned char* sBh = sAl + A_BYTES;
    unsigned char* sBl = sBh + B_BYTES;
    if (kb >= 2) {   // the MMAs of K block kb - 2 read this stage
      if (!tc::mbar_wait(&bar[s], phase[s])) ok = false;
      phase[s] ^= 1;
    }
    store_regs(sAh, sAl, sBh, sBl);
    if (kb + 1 < nkb) load_regs((kb + 1) * BK);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = tc::smem_u32(sAh), al = tc::smem_u32(sAl), bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const uint64_t ad = tc::desc_sw128((t == 2 ? al : ah) + kk * 32);
          const uint64_t bd = tc::desc_sw128((t == 1 ? bl : bh) + kk * 32);
          const uint32_t accum = (kb > 0 || kk > 0 || t > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(tc::idesc_tf32(BM, BN)), "r"(accum)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc::smem_u32(&bar[s]))
                   : "memory");
    }
  }
  // this commit tracks every MMA the CTA issued (also after an early stop)
  if (tid == 0)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc::smem_u32(&bar[2]))
                 : "memory");
  if (!tc::mbar_wait(&bar[2], 0)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = __syncthreads_and(ok) != 0;
  if (ok) {
    // warp w reads TMEM lane quarter w % 4 (rows) and column half w / 4
    float* tile = reinterpret_cast<float*>(smem);   // [128][BN + 1]; the stage buffers are free
    const int trow = (warp & 3) * 32 + lane, cbase = (warp >> 2) * (BN / 2);
#pragma unroll 1
    for (int c0 = 0; c0 < BN / 2; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(cbase + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) tile[trow * (BN + 1) + cbase + c0 + j] = __uint_as_float(r[j]);
    }
    __syncthreads();
    const int rows = min(BM, a.M - m0), cols = min(BN, a.N - n0);
    for (int i = tid; i < rows * BN; i += TCNT_THREADS) {
      const int rr = i / BN, cc = i % BN;
      if (cc < cols) {
        float* p = C + (size_t)(m0 + rr) * a.ldc + n0 + cc;
        const float v = a.alpha * tile[rr * (BN + 1) + cc];
        *p = (a.beta == 0.f) ? v : v + a.beta * *p;
      }
    }
  } else if (tid == 0) {
    atomicExch(a.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}
