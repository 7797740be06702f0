// Row-compressed condensed operators for the FP64 Algorithm-2 apply (apply_mode 2).
//
// On GB300 the FP64 pipe, not HBM, bounds the FP64 trace apply (Algorithm 2 moves 8 bytes
// per multiply-add and the FP64 rate is below the HBM byte rate / 4).  B, C and D of a
// macro-element are mostly structural zeros (3D, p = 2: 25 %, 46 % and 14 % of their
// entries are nonzero): B = A_uhu - A_uhq W and D = A_uhuh - A_uhq Wh only reach the
// nodes near a face and the lifting lines through them, C = -A_uuh + A_uq Wh only the
// nodes whose sub-elements meet such a line.  The pattern depends on the mesh and the
// degree, not on the state, and is the same for every macro-element of a box mesh up to
// its boundary faces.  It is found once, at context creation, as the union over all
// macro-elements and all species pairs of the nonzero entries of B, C, D assembled and
// condensed at a generic (seeded random) state; a coincidental zero at that state would
// need an exact cancellation in every macro-element at once.  Each condensation then
// packs the values of B, C, D into [macro][nonzero] arrays in that pattern (row-major,
// species-expanded), and the apply runs Algorithm 2 with these sparse rows.
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "lu.cuh"

namespace {

__device__ __forceinline__ double unit_hash(unsigned long long i, unsigned long long seed) {
  unsigned long long z = i * 0x9E3779B97F4A7C15ull + seed;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// generic state: u and uhat = (1, 0.1, -0.05, 0.08, 2) (d momenta) + U(-0.05, 0.05), q = U(-0.2, 0.2)
__global__ void k_generic_state(double* u, double* q, double* uh, long long nu, long long nq, long long nh, int Np,
                                int Nfn, int ns) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const double base[5] = {1.0, 0.1, -0.05, 0.08, 2.0};
  if (i < nu) {
    const int s = (int)((i / Np) % ns);
    u[i] = (s == ns - 1 ? base[4] : base[s]) + 0.1 * (unit_hash(i, 11) - 0.5);
  }
  if (i < nq) q[i] = 0.4 * (unit_hash(i, 23) - 0.5);
  if (i < nh) {
    const int s = (int)((i / Nfn) % ns);
    uh[i] = (s == ns - 1 ? base[4] : base[s]) + 0.1 * (unit_hash(i, 37) - 0.5);
  }
}

// flag[rn][cn] |= (X[e][t * RN + rn][s * CN + cn] != 0) over all e, t, s (node-level pattern)
__global__ void k_node_pattern(const double* X, int E, int ns, int RN, int CN, unsigned char* flag) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)RN * CN) return;
  const int rn = (int)(i / CN), cn = (int)(i % CN);
  const size_t rows = (size_t)ns * RN, cols = (size_t)ns * CN;
  unsigned char f = 0;
  for (int e = 0; e < E && !f; ++e)
    for (int t = 0; t < ns && !f; ++t)
      for (int s = 0; s < ns; ++s)
        if (X[(size_t)e * rows * cols + ((size_t)t * RN + rn) * cols + (size_t)s * CN + cn] != 0.0) {
          f = 1;
          break;
        }
  flag[i] = f;
}

// packed[e][k] = X[e][row[k]][col[k]]
__global__ void k_pack(const double* X, size_t rows, size_t cols, const int* prow, const int* pcol, long long nnz,
                       int E, double* packed) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nnz * E) return;
  const long long e = i / nnz, k = i - e * nnz;
  packed[i] = X[(size_t)e * rows * cols + (size_t)prow[k] * cols + pcol[k]];
}

__device__ __forceinline__ double sp_row_dot(const double* __restrict__ v, const int* __restrict__ col, int k0, int k1,
                                             const double* x, int lane) {
  double s0 = 0.0, s1 = 0.0;
  int k = k0 + lane;
  for (; k + 32 < k1; k += 64) {
    s0 += v[k] * x[col[k]];
    s1 += v[k + 32] * x[col[k + 32]];
  }
  if (k < k1) s0 += v[k] * x[col[k]];
  double s = s0 + s1;
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Algorithm 2 for one macro-element per CTA with the row-compressed C, B, D: gather x on dT_i,
// y1 = C x, y2 = S^-1 y1 (LU factors, dense), slot = B y2 + D x
constexpr int SP_NT = 256;   // four CTAs (macro-elements) resident per SM hide the solves' latency
__global__ void __launch_bounds__(SP_NT, 4) k_apply_sparse(const double* __restrict__ S, const int* __restrict__ perm,
                                                      SpOp B, SpOp C, SpOp D, const int* __restrict__ gather,
                                                      const double* __restrict__ x, double* __restrict__ slot, int Nu,
                                                      int Nt) {
  extern __shared__ unsigned char sm_raw[];
  double* xg = reinterpret_cast<double*>(sm_raw);   // Nt
  double* y1 = xg + Nt;                              // Nu
  double* y2 = y1 + Nu;                              // Nu
  const int e = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < Nt; i += blockDim.x) xg[i] = x[gather[(size_t)e * Nt + i]];
  __syncthreads();
  const double* Cv = C.val + (size_t)e * C.nnz;
  for (int r = w; r < Nu; r += nw) {
    const double s = sp_row_dot(Cv, C.col, C.off[r], C.off[r + 1], xg, lane);
    if (lane == 0) y1[r] = s;
  }
  __syncthreads();
  const int* pe = perm + (size_t)e * Nu;
  for (int i = threadIdx.x; i < Nu; i += blockDim.x) y2[i] = y1[pe[i]];
  __syncthreads();
  lu_solve_block<double, double>(S + (size_t)e * Nu * Nu, Nu, y2);
  const double* Bv = B.val + (size_t)e * B.nnz;
  const double* Dv = D.val + (size_t)e * D.nnz;
  for (int r = w; r < Nt; r += nw) {
    const double s = sp_row_dot(Bv, B.col, B.off[r], B.off[r + 1], y2, lane) +
                     sp_row_dot(Dv, D.col, D.off[r], D.off[r + 1], xg, lane);
    if (lane == 0) slot[(size_t)e * Nt + r] = s;
  }
}

// host: species-expanded CSR of a node-level pattern [RN][CN]; rows t * RN + rn, columns s * CN + cn
int build_csr(mehdg_ctx* ctx, const std::vector<unsigned char>& flag, int RN, int CN, SpOp& op, int** prow) {
  const int ns = ctx->ns;
  std::vector<int> off((size_t)ns * RN + 1, 0), col, row;
  for (int t = 0; t < ns; ++t)
    for (int rn = 0; rn < RN; ++rn) {
      const int r = t * RN + rn;
      for (int s = 0; s < ns; ++s)
        for (int cn = 0; cn < CN; ++cn)
          if (flag[(size_t)rn * CN + cn]) {
            col.push_back(s * CN + cn);
            row.push_back(r);
          }
      off[r + 1] = (int)col.size();
    }
  op.nnz = (long long)col.size();
  int *doff = nullptr, *dcol = nullptr, *drow = nullptr;
  double* dval = nullptr;
  CK(cudaMalloc(&doff, sizeof(int) * off.size()));
  CK(cudaMalloc(&dcol, sizeof(int) * std::max<size_t>(1, col.size())));
  CK(cudaMalloc(&drow, sizeof(int) * std::max<size_t>(1, row.size())));
  CK(cudaMalloc(&dval, sizeof(double) * std::max<long long>(1, op.nnz * ctx->E)));
  ctx->bytes += sizeof(int) * (off.size() + 2 * col.size()) + sizeof(double) * op.nnz * ctx->E;
  CK(cudaMemcpy(doff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
  if (!col.empty()) {
    CK(cudaMemcpy(dcol, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(drow, row.data(), sizeof(int) * row.size(), cudaMemcpyHostToDevice));
  }
  op.off = doff;
  op.col = dcol;
  op.val = dval;
  *prow = drow;
  return MEHDG_OK;
}

}  // namespace

int sparse_setup(mehdg_ctx* ctx) {
  if (ctx->opt.precision != MEHDG_PREC_FP64)
    return ctx_fail(ctx, MEHDG_ERR_ARG, "apply_mode 2 (row-compressed Algorithm 2) is an FP64 form");
  const int E = ctx->E, ns = ctx->ns, Np = ctx->Np, Nth = ctx->Nth;
  const long long nu = (long long)E * ctx->Nu, nq = nu * ctx->d, nh = ctx->ntr;
  const long long nmax = std::max(std::max(nu, nq), nh);
  k_generic_state<<<(unsigned)((nmax + 255) / 256), 256, 0, ctx->stream>>>(ctx->du, ctx->dq, ctx->duh, nu, nq, nh,
                                                                            Np, ctx->Nfn, ns);
  CKL();
  int rc;
  if ((rc = assemble_all(ctx, ctx->du, ctx->dq, ctx->duh, nullptr, nullptr))) return rc;
  ctx->sp_pending = true;   // condensation without packing (the pattern does not exist yet)
  rc = condense_all(ctx, 1.0, nullptr);
  ctx->sp_pending = false;
  if (rc) return rc;
  ctx->condensed = false;
  unsigned char* dflag = nullptr;
  const size_t nflag = (size_t)Nth * Np + (size_t)Np * Nth + (size_t)Nth * Nth;
  CK(cudaMalloc(&dflag, nflag));
  unsigned char *fB = dflag, *fC = fB + (size_t)Nth * Np, *fD = fC + (size_t)Np * Nth;
  k_node_pattern<<<(unsigned)(((size_t)Nth * Np + 255) / 256), 256, 0, ctx->stream>>>(ctx->Ahu, E, ns, Nth, Np, fB);
  k_node_pattern<<<(unsigned)(((size_t)Np * Nth + 255) / 256), 256, 0, ctx->stream>>>(ctx->Auh, E, ns, Np, Nth, fC);
  k_node_pattern<<<(unsigned)(((size_t)Nth * Nth + 255) / 256), 256, 0, ctx->stream>>>(ctx->Ahh, E, ns, Nth, Nth, fD);
  ctx->launches += 3;
  std::vector<unsigned char> h(nflag);
  cudaError_t ce = cudaMemcpyAsync(h.data(), dflag, nflag, cudaMemcpyDeviceToHost, ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  cudaFree(dflag);
  if (ce != cudaSuccess) return ctx_fail(ctx, MEHDG_ERR_CUDA, std::string("sparse pattern: ") + cudaGetErrorString(ce));
  std::vector<unsigned char> hB(h.begin(), h.begin() + (size_t)Nth * Np);
  std::vector<unsigned char> hC(h.begin() + (size_t)Nth * Np, h.begin() + (size_t)Nth * Np + (size_t)Np * Nth);
  std::vector<unsigned char> hD(h.begin() + (size_t)Nth * Np + (size_t)Np * Nth, h.end());
  if ((rc = build_csr(ctx, hB, Nth, Np, ctx->spB, &ctx->spB_row))) return rc;
  if ((rc = build_csr(ctx, hC, Np, Nth, ctx->spC, &ctx->spC_row))) return rc;
  if ((rc = build_csr(ctx, hD, Nth, Nth, ctx->spD, &ctx->spD_row))) return rc;
  return MEHDG_OK;
}

int sparse_pack(mehdg_ctx* ctx) {
  if (ctx->sp_pending || !ctx->spB.val) return MEHDG_OK;
  const int E = ctx->E;
  const size_t Nu = ctx->Nu, Nt = ctx->Nt;
  struct { const double* X; size_t r, c; SpOp* op; const int* row; } jobs[3] = {
      {ctx->Ahu, Nt, Nu, &ctx->spB, ctx->spB_row}, {ctx->Auh, Nu, Nt, &ctx->spC, ctx->spC_row},
      {ctx->Ahh, Nt, Nt, &ctx->spD, ctx->spD_row}};
  for (auto& j : jobs) {
    const long long tot = j.op->nnz * E;
    if (tot == 0) continue;
    k_pack<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(j.X, j.r, j.c, j.row, j.op->col, j.op->nnz, E,
                                                                    j.op->val);
    CKL();
  }
  return MEHDG_OK;
}

int apply_sparse(mehdg_ctx* ctx, const double* x, double* y) {
  const size_t smem = sizeof(double) * (ctx->Nt + 2 * (size_t)ctx->Nu);
  CK(cudaFuncSetAttribute(k_apply_sparse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  phase_begin(ctx, PH_APPLY);
  k_apply_sparse<<<ctx->E, SP_NT, smem, ctx->stream>>>(ctx->Auu, ctx->perm, ctx->spB, ctx->spC, ctx->spD, ctx->gather,
                                                     x, ctx->slot, ctx->Nu, ctx->Nt);
  CKL();
  int rc = face_reduce(ctx, ctx->slot, y);
  phase_end(ctx, PH_APPLY);
  return rc;
}

void sparse_destroy(mehdg_ctx* ctx) {
  SpOp* ops[3] = {&ctx->spB, &ctx->spC, &ctx->spD};
  for (SpOp* o : ops) {
    if (o->off) cudaFree((void*)o->off);
    if (o->col) cudaFree((void*)o->col);
    if (o->val) cudaFree((void*)o->val);
  }
  int* rows[3] = {ctx->spB_row, ctx->spC_row, ctx->spD_row};
  for (int* r : rows)
    if (r) cudaFree(r);
}
