// a0: macro-element mesh, DOF maps, reference operators, closed-form data, state
// initialisation and the context lifecycle (mehdg_mesh / query / init_state /
// get_block / destroy).
//
// Spaces (Sec. 2.2): u and q are C0 tensor-product Lagrange polynomials of degree
// p on the m^d sub-boxes of each macro-element (GLL nodes), the trace lives on
// each macro-face in the C0 degree-p space of its m^(d-1) sub-faces.  Quadrature:
// p+2 Gauss-Legendre points per direction on every sub-box / sub-face.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"
#include "physics.cuh"

int ctx_fail(mehdg_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

// Inside a stream capture the events become event-record nodes of the graph
// (cudaEventRecordExternal), so phases inside the captured inner GMRES are timed at
// each replay too.
void phase_begin(mehdg_ctx* ctx, int p) {
  if (ctx->no_phase) return;
  if (ctx->capturing) {
    if (!ctx->ev[2 * p]) {
      cudaEventCreate(&ctx->ev[2 * p]);
      cudaEventCreate(&ctx->ev[2 * p + 1]);
    }
    cudaEventRecordWithFlags(ctx->ev[2 * p], ctx->stream, cudaEventRecordExternal);
    ++ctx->ph_graph[p];
    return;
  }
  std::vector<cudaEvent_t>&b = ctx->ring_b[p], &e = ctx->ring_e[p];
  if (ctx->ring_n[p] == (int)b.size()) {
    if (b.size() < 1024) {
      cudaEvent_t x = nullptr, y = nullptr;
      cudaEventCreate(&x);
      cudaEventCreate(&y);
      b.push_back(x);
      e.push_back(y);
    } else {   // pool full: wait for its last pair and fold the pool into the sums
      cudaEventSynchronize(e[ctx->ring_n[p] - 1]);
      phase_harvest(ctx);
    }
  }
  cudaEventRecord(b[ctx->ring_n[p]], ctx->stream);
}
void phase_end(mehdg_ctx* ctx, int p) {
  if (ctx->no_phase) return;
  if (ctx->capturing) {
    cudaEventRecordWithFlags(ctx->ev[2 * p + 1], ctx->stream, cudaEventRecordExternal);
    ctx->ev_rec[p] = true;
    return;
  }
  cudaEventRecord(ctx->ring_e[p][ctx->ring_n[p]], ctx->stream);
  ++ctx->ring_n[p];
}
void phase_harvest(mehdg_ctx* ctx) {
  for (int p = 0; p < PH_COUNT; ++p) {
    for (int i = 0; i < ctx->ring_n[p]; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ctx->ring_b[p][i], ctx->ring_e[p][i]) == cudaSuccess) {
        ctx->ph_sum[p] += t;
        ++ctx->ph_cnt[p];
        ctx->ph_last[p] = t;
      }
    }
    ctx->ring_n[p] = 0;
    if (ctx->ph_graph[p] && ctx->ev_rec[p] && ctx->ig_replays > 0) {
      // graph phases: the pair holds the last execution of the last replay; every execution
      // of the replays since the last harvest is counted at that duration
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ctx->ev[2 * p], ctx->ev[2 * p + 1]) == cudaSuccess) {
        const long long n = ctx->ig_replays * ctx->ph_graph[p];
        ctx->ph_sum[p] += (double)t * n;
        ctx->ph_cnt[p] += n;
        ctx->ph_last[p] = t;
      }
    }
  }
  cudaGetLastError();
  ctx->ig_replays = 0;
}

extern "C" int mehdg_graph_replays(const mehdg_ctx* ctx, long long* count) {
  if (!ctx || !count) return MEHDG_ERR_ARG;
  *count = ctx->ig_total;
  return MEHDG_OK;
}

extern "C" int mehdg_launch_count(const mehdg_ctx* ctx, long long* count) {
  if (!ctx || !count) return MEHDG_ERR_ARG;
  *count = ctx->launches;
  return MEHDG_OK;
}

extern "C" int mehdg_phase_times(mehdg_ctx* ctx, double* ms, int n) {
  if (!ctx || !ms || n < 0 || n > PH_COUNT) return MEHDG_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  phase_harvest(ctx);
  for (int p = 0; p < n; ++p) ms[p] = ctx->ph_cnt[p] > 0 ? ctx->ph_last[p] : -1.0;
  return MEHDG_OK;
}

extern "C" int mehdg_phase_stats(mehdg_ctx* ctx, double* sum_ms, long long* count, int n, int reset) {
  if (!ctx || n < 0 || n > PH_COUNT) return MEHDG_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  phase_harvest(ctx);
  for (int p = 0; p < n; ++p) {
    if (sum_ms) sum_ms[p] = ctx->ph_sum[p];
    if (count) count[p] = ctx->ph_cnt[p];
  }
  if (reset)
    for (int p = 0; p < PH_COUNT; ++p) {
      ctx->ph_sum[p] = 0.0;
      ctx->ph_cnt[p] = 0;
    }
  return MEHDG_OK;
}

Geo make_geo(const mehdg_ctx* c) {
  Geo g;
  g.d = c->d; g.ns = c->ns; g.m = c->m; g.p = c->p; g.n1 = c->n1; g.Np = c->Np; g.Nfn = c->Nfn;
  g.Nth = c->Nth; g.Nu = c->Nu; g.Nt = c->Nt; g.nel = c->nel; g.nloc = c->nloc; g.ng1 = c->ng1;
  g.Ng = c->Ng; g.nsf = c->nsf; g.nfs = c->nfs; g.nfp = c->nfp;
  g.nf = c->nf;
  for (int k = 0; k < 3; ++k) g.he[k] = c->he[k];
  return g;
}

// ---------------------------------------------------------------- 1D rules
static void legendre(int n, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = -cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, z, P, dP);
      double dz = P / dP;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double P, dP;
    legendre(n, z, P, dP);
    x[i] = z;
    w[i] = 2.0 / ((1 - z * z) * dP * dP);
  }
}

static std::vector<double> gll_nodes(int p) {
  std::vector<double> x(p + 1);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double z = -cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, z, P, dP);
      double d2P = (2 * z * dP - p * (p + 1) * P) / (1 - z * z);
      double dz = dP / d2P;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  return x;
}

static void lagrange_at(const std::vector<double>& xn, double x, double* L, double* dL) {
  int n = (int)xn.size();
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) v *= (x - xn[k]) / (xn[j] - xn[k]);
    L[j] = v;
    double dv = 0.0;
    for (int l = 0; l < n; ++l) {
      if (l == j) continue;
      double t = 1.0 / (xn[j] - xn[l]);
      for (int k = 0; k < n; ++k)
        if (k != j && k != l) t *= (x - xn[k]) / (xn[j] - xn[k]);
      dv += t;
    }
    dL[j] = dv;
  }
}

// small dense inverse (Gauss-Jordan with partial pivoting)
void invert(std::vector<double>& A, int n) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int r = c;
    for (int i = c + 1; i < n; ++i)
      if (fabs(A[i * n + c]) > fabs(A[r * n + c])) r = i;
    for (int j = 0; j < n; ++j) {
      std::swap(A[c * n + j], A[r * n + j]);
      std::swap(I[c * n + j], I[r * n + j]);
    }
    double piv = A[c * n + c];
    for (int j = 0; j < n; ++j) { A[c * n + j] /= piv; I[c * n + j] /= piv; }
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      double f = A[i * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) { A[i * n + j] -= f * A[c * n + j]; I[i * n + j] -= f * I[c * n + j]; }
    }
  }
  A = I;
}

// Kronecker product over axes (axis 0 fastest) of n1 x n1 (or n1 x 1) factors
static void kron_dense(int d, int n1, const std::vector<const double*>& f, std::vector<int> cols,
                       std::vector<double>& out, int& R, int& C) {
  R = 1; C = 1;
  for (int k = 0; k < d; ++k) { R *= n1; C *= cols[k]; }
  out.assign((size_t)R * C, 0.0);
  for (int a = 0; a < R; ++a)
    for (int b = 0; b < C; ++b) {
      int aa = a, bb = b;
      double v = 1.0;
      for (int k = 0; k < d; ++k) {
        int ak = aa % n1, bk = bb % cols[k];
        aa /= n1; bb /= cols[k];
        v *= f[k][ak * cols[k] + bk];
      }
      out[(size_t)a * C + b] = v;
    }
}

// ---------------------------------------------------------------- device kernels for data
template <int D>
__global__ void k_source(Geo g, const double* tab, mehdg_problem pr, double* src) {
  constexpr int NS = D + 2;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)pr.nmac[0] * (D > 1 ? pr.nmac[1] : 1) * (D > 2 ? pr.nmac[2] : 1) * g.nel * g.Ng;
  if (tid >= tot) return;
  int gq = tid % g.Ng;
  int el = (tid / g.Ng) % g.nel;
  int e = (int)(tid / ((long long)g.Ng * g.nel));
  // table layout: b1, db1, Gauss weights, Gauss points, macro node coordinates
  const double* gx = tab + 2 * g.ng1 * (g.p + 1) + g.ng1;
  double x[D];
  int ee = e, ll = el, gg = gq;
  for (int k = 0; k < D; ++k) {
    int ek = ee % pr.nmac[k]; ee /= pr.nmac[k];
    int lk = ll % g.m; ll /= g.m;
    int gk = gg % g.ng1; gg /= g.ng1;
    double hm = (pr.hi[k] - pr.lo[k]) / pr.nmac[k];
    x[k] = pr.lo[k] + ek * hm + (lk + 0.5 * (gx[gk] + 1.0)) * g.he[k];
  }
  closed_form_source<D>(pr.field == MEHDG_FIELD_COUETTE3D, pr.field_par, pr.gamma, pr.Re, pr.Pr, x, src + tid * NS);
}

// closed-form state at a physical point
template <int D>
__device__ void field_at(const mehdg_problem& pr, const double* x, double* u) {
  static_assert(MEHDG_FIELD_MMS == 1 && MEHDG_FIELD_TGV == 3 && MEHDG_FIELD_COUETTE3D == 5, "field kinds");
  closed_form_state<D>(pr.field, pr.field_par, pr.gamma, x, u);
}

template <int D>
__global__ void k_dirichlet(Geo g, const double* tab, mehdg_problem pr, const int* bkind, double* uD) {
  constexpr int NS = D + 2;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int E = pr.nmac[0] * (D > 1 ? pr.nmac[1] : 1) * (D > 2 ? pr.nmac[2] : 1);
  long long tot = (long long)E * 2 * D * g.nsf * g.nfp;
  if (tid >= tot) return;
  int fp = tid % g.nfp;
  int sf = (tid / g.nfp) % g.nsf;
  int fl = (tid / ((long long)g.nfp * g.nsf)) % (2 * D);
  int e = (int)(tid / ((long long)g.nfp * g.nsf * 2 * D));
  double* out = uD + tid * NS;
  if (bkind[e * 2 * D + fl] == MEHDG_BC_FARFIELD) {   // the free stream u_inf of field_par
    field_uniform<D>(pr.field_par, pr.gamma, out);
    return;
  }
  if (bkind[e * 2 * D + fl] != MEHDG_BC_DIRICHLET) {
    for (int s = 0; s < NS; ++s) out[s] = 0.0;
    return;
  }
  const double* gx = tab + 2 * g.ng1 * (g.p + 1) + g.ng1;
  int k = fl / 2, side = fl % 2;
  int eidx[3], ee = e;
  for (int kk = 0; kk < D; ++kk) { eidx[kk] = ee % pr.nmac[kk]; ee /= pr.nmac[kk]; }
  double x[D];
  int ss = sf, pp = fp;
  for (int kk = 0; kk < D; ++kk) {
    double hm = (pr.hi[kk] - pr.lo[kk]) / pr.nmac[kk];
    double x0 = pr.lo[kk] + eidx[kk] * hm;
    if (kk == k) {
      x[kk] = side ? x0 + hm : x0;
    } else {
      int sk = ss % g.m; ss /= g.m;
      int gk = pp % g.ng1; pp /= g.ng1;
      x[kk] = x0 + (sk + 0.5 * (gx[gk] + 1.0)) * g.he[kk];
    }
  }
  double u[NS];
  field_at<D>(pr, x, u);
  for (int s = 0; s < NS; ++s) out[s] = u[s];
}

template <int D>
__global__ void k_init_state(Geo g, mehdg_problem pr, const double* xnode1, const double* du,
                             double* u) {
  constexpr int NS = D + 2;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int E = pr.nmac[0] * (D > 1 ? pr.nmac[1] : 1) * (D > 2 ? pr.nmac[2] : 1);
  if (tid >= (long long)E * g.Np) return;
  int a = tid % g.Np;
  int e = (int)(tid / g.Np);
  double x[D];
  int ee = e, aa = a;
  for (int k = 0; k < D; ++k) {
    int ek = ee % pr.nmac[k]; ee /= pr.nmac[k];
    int ak = aa % g.n1; aa /= g.n1;
    double hm = (pr.hi[k] - pr.lo[k]) / pr.nmac[k];
    x[k] = pr.lo[k] + ek * hm + xnode1[k * g.n1 + ak];
  }
  double uu[NS];
  field_at<D>(pr, x, uu);
  for (int s = 0; s < NS; ++s) {
    long long o = ((long long)e * NS + s) * g.Np + a;
    u[o] = uu[s] + (du ? du[o] : 0.0);
  }
}

__global__ void k_init_trace(Geo g, const int* owner, const int* fnode, const double* u,
                             const double* duh, double* uh, int F) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)F * g.ns * g.Nfn) return;
  int j = tid % g.Nfn;
  int f = (int)(tid / ((long long)g.ns * g.Nfn));
  int s = (tid / g.Nfn) % g.ns;
  int o = owner[2 * f];
  if (o < 0) o = owner[2 * f + 1];
  int e = o / g.nf, fl = o % g.nf;
  int a = fnode[fl * g.Nfn + j];
  uh[tid] = u[((long long)e * g.ns + s) * g.Np + a] + (duh ? duh[tid] : 0.0);
}

// q = -M^-1 (G_k u + Gh_k uh_loc): the gradient that makes R_Q vanish
__global__ void k_lift(Geo g, const double* Wk, const double* Whk, const int* gather,
                       const double* u, const double* uh, double* q, int E, size_t sG, size_t sGh) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)E * g.d * g.ns * g.Np;
  if (tid >= tot) return;
  int a = tid % g.Np;
  int s = (tid / g.Np) % g.ns;
  int k = (tid / ((long long)g.Np * g.ns)) % g.d;
  int e = (int)(tid / ((long long)g.Np * g.ns * g.d));
  const double* W = Wk + e * sG + (size_t)k * g.Np * g.Np + (size_t)a * g.Np;
  const double* Wh = Whk + e * sGh + (size_t)k * g.Np * g.Nth + (size_t)a * g.Nth;
  const double* ue = u + ((size_t)e * g.ns + s) * g.Np;
  const int* ge = gather + (size_t)e * g.Nt + (size_t)s * g.Nth;
  double acc = 0.0;
  for (int b = 0; b < g.Np; ++b) acc += W[b] * ue[b];
  for (int i = 0; i < g.Nth; ++i) acc += Wh[i] * uh[ge[i]];
  q[tid] = -acc;
}

// ---------------------------------------------------------------- context
static int alloc(mehdg_ctx* ctx, void** p, size_t bytes) {
  if (bytes == 0) { *p = nullptr; return 0; }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess)
    return ctx_fail(ctx, MEHDG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  ctx->bytes += bytes;
  return 0;
}
#define ALLOC(ptr, count)                                                        \
  do {                                                                           \
    int r_ = alloc(ctx, (void**)&(ptr), sizeof(*(ptr)) * (size_t)(count));       \
    if (r_) return r_;                                                           \
  } while (0)

static void default_options(mehdg_options* o) {
  memset(o, 0, sizeof(*o));
  o->precision = MEHDG_PREC_FP64;
  o->precond = 0;
  o->restart = 30;
  o->max_iters = 2000;
  o->lin_rtol = 1e-6;
  o->lin_atol = 0.0;
  o->inner_iters = 5;
  o->newton_rtol = 1e-8;
  o->newton_atol = 1e-14;
  o->max_newton = 100;
  o->tau_init = 1.0;
  o->tau_max = 1e8;
  o->refine_iters = 2;
  o->apply_mode = 0;
  o->tc_mode = 0;
  o->precond_bf16 = 0;
  o->solver = 0;
  o->condense_layers = 2;
}

// allocations common to every mesh kind: blocks, pointwise scratch, face blocks, reduction
// scratch, Krylov and state vectors (tab, Wk, Whk: host tables for the FP32 copies of box meshes)
static int setup_common(mehdg_ctx* ctx, const std::vector<double>& tab, const std::vector<double>& Wk,
                        const std::vector<double>& Whk) {
  const int d = ctx->d, E = ctx->E, F = ctx->F, ns = ctx->ns, Np = ctx->Np, Nfn = ctx->Nfn;
  const size_t Nu = ctx->Nu, Nt = ctx->Nt;
  cudaStream_t st = ctx->stream;

  // blocks are FP32 in the mixed-precision path: allocate half the doubles
  const size_t bsz = ctx->opt.precision == MEHDG_PREC_MIXED ? 2 : 1;
  ALLOC(ctx->Auu, (size_t)E * Nu * Nu / bsz + 1);
  ALLOC(ctx->Auq, (size_t)E * d * Nu * Nu / bsz + 1);
  ALLOC(ctx->Auh, (size_t)E * Nu * Nt / bsz + 1);
  ALLOC(ctx->Ahu, (size_t)E * Nt * Nu / bsz + 1);
  ALLOC(ctx->Ahq, (size_t)E * d * Nt * Nu / bsz + 1);
  ALLOC(ctx->Ahh, (size_t)E * Nt * Nt / bsz + 1);
  ALLOC(ctx->perm, (size_t)E * Nu);
  ALLOC(ctx->RQ, (size_t)E * d * Nu);
  ALLOC(ctx->RU, (size_t)E * Nu);
  ALLOC(ctx->RUh, (size_t)E * Nt);
  ALLOC(ctx->gv, (size_t)E * Nu);
  ALLOC(ctx->hv, (size_t)E * Nt);
  ALLOC(ctx->MinvRQ, (size_t)E * d * Nu);
  ALLOC(ctx->bloc, (size_t)E * Nt);
  ALLOC(ctx->slot, (size_t)E * Nt);
  {
    size_t nk = (size_t)E * (d + 1) * ns * ctx->nel * ctx->Ng * (d + 1) * ns * (d + 1) / bsz + 1;
    // the same scratch holds the face-block inverses of the mixed block-Jacobi (FP64, F nfb^2)
    nk = std::max(nk, (size_t)ctx->F * ns * Nfn * ns * Nfn);
    ALLOC(ctx->Kvol, nk);
  }
  ALLOC(ctx->rvol, (size_t)E * ctx->nel * ctx->Ng * ns * (d + 1));
  ALLOC(ctx->Kface, (size_t)E * ctx->nf * ctx->nsf * ctx->nfp * ctx->ndir_f * 2 * ns);
  ALLOC(ctx->rface, (size_t)E * ctx->nf * ctx->nsf * ctx->nfp * 2 * ns);
  ctx->nfb = ns * Nfn;
  ALLOC(ctx->fblk, (size_t)F * ctx->nfb * ctx->nfb);
  ALLOC(ctx->fperm, (size_t)F * ctx->nfb);
  if (!ctx->dflag) ALLOC(ctx->dflag, 16);
  ALLOC(ctx->dred, 1 << 17);
  ALLOC(ctx->ddiag, (size_t)E * 3 + 4);
  CK(cudaMemsetAsync(ctx->dred, 0, sizeof(double) << 17, st));   // reduction tickets start at zero
  CK(cudaMallocHost((void**)&ctx->hred, sizeof(double) * 256));
  ALLOC(ctx->dtcerr, 4);
  CK(cudaMemsetAsync(ctx->dtcerr, 0, sizeof(int) * 4, st));
  if (ctx->opt.precision == MEHDG_PREC_MIXED) {
    ALLOC(ctx->finv32, (size_t)F * ctx->nfb * ctx->nfb);
    if (ctx->mapped) {
      // FP32 copies of the per-macro liftings and condensation factor
      const long long nw = (long long)E * ctx->sG, nwh = (long long)E * ctx->sGh, nb = (long long)E * ctx->sB;
      ALLOC(ctx->Wk32, nw);
      ALLOC(ctx->Whk32, nwh);
      ALLOC(ctx->Bcat32, nb);
      int r_;
      if ((r_ = to_float(ctx, ctx->Wk, ctx->Wk32, nw))) return r_;
      if ((r_ = to_float(ctx, ctx->Whk, ctx->Whk32, nwh))) return r_;
      if ((r_ = to_float(ctx, ctx->Bcat, ctx->Bcat32, nb))) return r_;
    } else {
      std::vector<float> w32(Wk.begin(), Wk.end()), wh32(Whk.begin(), Whk.end());
      ALLOC(ctx->Wk32, w32.size());
      ALLOC(ctx->Whk32, wh32.size());
      CK(cudaMemcpy(ctx->Wk32, w32.data(), sizeof(float) * w32.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(ctx->Whk32, wh32.data(), sizeof(float) * wh32.size(), cudaMemcpyHostToDevice));
    }
    if (ctx->opt.refine_iters > 0) ALLOC(ctx->S32, (size_t)E * Nu * Nu);
    ALLOC(ctx->u32, (size_t)E * ns * Np);
    ALLOC(ctx->h32, (size_t)E * ns * Np);
    ALLOC(ctx->q32, (size_t)E * d * ns * Np);
    std::vector<float> t32(tab.begin(), tab.end());
    ALLOC(ctx->tab32, t32.size());
    CK(cudaMemcpy(ctx->tab32, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice));
  }
  if (ctx->opt.apply_mode == 1) {
    size_t esz = ctx->opt.precision == MEHDG_PREC_MIXED ? sizeof(float) : sizeof(double);
    {
      // forming A^T_i keeps a Nu x 32 block of right-hand sides in shared memory
      int dev = 0, optin = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      if (esz * Nu * 32 + 48 * 1024 > (size_t)optin)
        return ctx_fail(ctx, MEHDG_ERR_ARG, "apply_mode 1 needs Nu x 32 entries in shared memory; use apply_mode 0");
    }
    ALLOC(ctx->Xbuf, (size_t)E * Nu * Nt * esz / sizeof(double) + 1);
    if (ctx->opt.precond_bf16) {
      ctx->ld16 = (Nt + 3) & ~3;
      ALLOC(ctx->Ahat16, (size_t)E * Nt * ctx->ld16);
    }
    if (ctx->opt.precond_bf16 && ctx->opt.precision == MEHDG_PREC_MIXED) {
      ctx->ldf16 = (ctx->nfb + 31) & ~31;
      ALLOC(ctx->finv16, (size_t)F * ctx->nfb * ctx->ldf16);
    }
  }
  ctx->restart = std::min(120, std::max(2, ctx->opt.restart));
  const long long n = ctx->ntr;
  ALLOC(ctx->V, (size_t)(ctx->restart + 1) * n);
  ALLOC(ctx->Zk, (size_t)ctx->restart * n);
  ALLOC(ctx->wv, n);
  ALLOC(ctx->tv, n);
  ALLOC(ctx->tv2, n);
  ALLOC(ctx->rv, n);
  int nin = std::min(120, std::max(1, ctx->opt.inner_iters));
  ALLOC(ctx->iV, (size_t)(nin + 1) * n);
  ALLOC(ctx->iw, n);
  ALLOC(ctx->xstart, n);
  ALLOC(ctx->dHo, (size_t)(ctx->restart + 1) * ctx->restart + 3 * (size_t)ctx->restart + 1);
  ALLOC(ctx->dHi, (size_t)(nin + 1) * nin + 3 * (size_t)nin + 1);
  ALLOC(ctx->gin, n);
  ALLOC(ctx->gout, n);
  ALLOC(ctx->un, (size_t)E * Nu);
  ALLOC(ctx->ustage, (size_t)3 * E * Nu);
  ALLOC(ctx->hist, (size_t)E * Nu);
  ALLOC(ctx->du, (size_t)E * Nu);
  ALLOC(ctx->dq, (size_t)E * d * Nu);
  ALLOC(ctx->duh, n);
  ALLOC(ctx->bhat, n);

  return MEHDG_OK;
}

// simplicial macro-elements: sizes, maps and per-macro geometry from csrc/simplex.cu, uploaded
// as for curved macros (per-macro M, G_k, Gh_k, liftings and condensation factor), then the
// common allocations and the closed-form data at the volume and face points.  FP64 only.
static int setup_simplex(mehdg_ctx* ctx) {
  const mehdg_problem& pr = ctx->prob;
  const int d = pr.dim;
  ctx->d = d;
  ctx->ns = d + 2;
  ctx->m = pr.m;
  ctx->p = pr.p;
  ctx->n1 = pr.m * pr.p + 1;
  ctx->ng1 = pr.p + 3;
  ctx->mapped = false;
  ctx->simplex = 1;
  ctx->ndir_v = ctx->ns * (1 + d);
  ctx->ndir_f = ctx->ns * (d + 2);
  SxRef R;
  SxHost H;
  if (int r_ = sx_maps(ctx, R, H)) return r_;
  const int E = ctx->E, F = ctx->F, Np = ctx->Np, Nfn = ctx->Nfn, Nth = ctx->Nth, Nt = ctx->Nt, nf = ctx->nf;
  const int ns = ctx->ns;
  ctx->sM = (size_t)Np * Np;
  ctx->sG = (size_t)d * Np * Np;
  ctx->sGh = (size_t)d * Np * Nth;
  ctx->sB = (size_t)d * Np * (Np + Nth);
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  ALLOC(ctx->gather, (size_t)E * Nt);
  ALLOC(ctx->owner, 2 * (size_t)F);
  ALLOC(ctx->bkind, (size_t)E * nf);
  ALLOC(ctx->bside, (size_t)E * nf);
  ALLOC(ctx->fnode, (size_t)nf * Nfn);
  ALLOC(ctx->ofn, ctx->h_ofn.size());
  ALLOC(ctx->Mref, (size_t)E * ctx->sM);
  ALLOC(ctx->Minv, (size_t)E * ctx->sM);
  ALLOC(ctx->Gk, (size_t)E * ctx->sG);
  ALLOC(ctx->Wk, (size_t)E * ctx->sG);
  ALLOC(ctx->Ghk, (size_t)E * ctx->sGh);
  ALLOC(ctx->Whk, (size_t)E * ctx->sGh);
  ALLOC(ctx->Bcat, (size_t)E * ctx->sB);
  ALLOC(ctx->vgeo, H.vgeo.size());
  ALLOC(ctx->fgeo, H.fgeo.size());
  ALLOC(ctx->xnode, H.xnode.size());
  ALLOC(ctx->sx_vtab, R.vtab.size());
  ALLOC(ctx->sx_vnode, R.vnode.size());
  ALLOC(ctx->sx_ftab, R.ftab.size());
  ALLOC(ctx->sx_fsub, R.fsub.size());
  CK(up(ctx->gather, ctx->h_gather.data(), sizeof(int) * ctx->h_gather.size()));
  CK(up(ctx->owner, ctx->h_owner.data(), sizeof(int) * ctx->h_owner.size()));
  CK(up(ctx->bkind, ctx->h_bkind.data(), sizeof(int) * ctx->h_bkind.size()));
  CK(up(ctx->bside, ctx->h_bside.data(), sizeof(int) * ctx->h_bside.size()));
  CK(up(ctx->fnode, ctx->facenode.data(), sizeof(int) * ctx->facenode.size()));
  CK(up(ctx->ofn, ctx->h_ofn.data(), sizeof(int) * ctx->h_ofn.size()));
  CK(up(ctx->Mref, H.M.data(), sizeof(double) * H.M.size()));
  CK(up(ctx->Minv, H.Minv.data(), sizeof(double) * H.Minv.size()));
  CK(up(ctx->Gk, H.Gk.data(), sizeof(double) * H.Gk.size()));
  CK(up(ctx->Wk, H.Wk.data(), sizeof(double) * H.Wk.size()));
  CK(up(ctx->Ghk, H.Ghk.data(), sizeof(double) * H.Ghk.size()));
  CK(up(ctx->Whk, H.Whk.data(), sizeof(double) * H.Whk.size()));
  CK(up(ctx->Bcat, H.Bcat.data(), sizeof(double) * H.Bcat.size()));
  CK(up(ctx->vgeo, H.vgeo.data(), sizeof(double) * H.vgeo.size()));
  CK(up(ctx->fgeo, H.fgeo.data(), sizeof(double) * H.fgeo.size()));
  CK(up(ctx->xnode, H.xnode.data(), sizeof(double) * H.xnode.size()));
  CK(up(ctx->sx_vtab, R.vtab.data(), sizeof(double) * R.vtab.size()));
  CK(up(ctx->sx_vnode, R.vnode.data(), sizeof(int) * R.vnode.size()));
  CK(up(ctx->sx_ftab, R.ftab.data(), sizeof(double) * R.ftab.size()));
  CK(up(ctx->sx_fsub, R.fsub.data(), sizeof(int) * R.fsub.size()));
  if (int r_ = setup_common(ctx, std::vector<double>(), std::vector<double>(), std::vector<double>())) return r_;
  // closed-form data: the source at the volume points, the boundary data at the face points
  const long long nvol = (long long)E * ctx->nel * ctx->Ng, nfac = (long long)E * nf * ctx->nsf * ctx->nfp;
  double* xtmp = nullptr;
  CK(cudaMalloc(&xtmp, sizeof(double) * std::max(H.xq.size(), H.xf.size())));
  int rc = MEHDG_OK;
  if (pr.field == MEHDG_FIELD_MMS || pr.field == MEHDG_FIELD_COUETTE3D) {
    rc = alloc(ctx, (void**)&ctx->src, sizeof(double) * (size_t)nvol * ns);
    if (!rc && up(xtmp, H.xq.data(), sizeof(double) * H.xq.size()) != cudaSuccess)
      rc = ctx_fail(ctx, MEHDG_ERR_CUDA, "simplex: point upload");
    if (!rc) rc = sx_source(ctx, xtmp, nvol, ctx->src);
    if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = ctx_fail(ctx, MEHDG_ERR_CUDA, "simplex: source");
  }
  if (!rc) rc = alloc(ctx, (void**)&ctx->uD, sizeof(double) * (size_t)nfac * ns);
  if (!rc && up(xtmp, H.xf.data(), sizeof(double) * H.xf.size()) != cudaSuccess)
    rc = ctx_fail(ctx, MEHDG_ERR_CUDA, "simplex: point upload");
  if (!rc) rc = sx_bdata(ctx, xtmp, nfac, ctx->nsf * ctx->nfp, ctx->uD);
  if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = ctx_fail(ctx, MEHDG_ERR_CUDA, "simplex: boundary data");
  cudaFree(xtmp);
  return rc;
}

static int setup(mehdg_ctx* ctx) {
  const mehdg_problem& pr = ctx->prob;
  if (pr.mesh_kind == MEHDG_MESH_SIMPLEX) return setup_simplex(ctx);
  const int d = pr.dim;
  ctx->d = d;
  ctx->ns = d + 2;
  ctx->m = pr.m;
  ctx->p = pr.p;
  ctx->n1 = pr.m * pr.p + 1;
  ctx->Np = 1; ctx->Nfn = 1; ctx->nel = 1; ctx->nloc = 1; ctx->Ng = 1; ctx->nsf = 1; ctx->nfs = 1; ctx->nfp = 1;
  ctx->ng1 = pr.p + 2;
  for (int k = 0; k < d; ++k) {
    ctx->Np *= ctx->n1;
    ctx->nel *= pr.m;
    ctx->nloc *= pr.p + 1;
    ctx->Ng *= ctx->ng1;
    if (k < d - 1) {
      ctx->Nfn *= ctx->n1;
      ctx->nsf *= pr.m;
      ctx->nfs *= pr.p + 1;
      ctx->nfp *= ctx->ng1;
    }
  }
  ctx->Nth = 2 * d * ctx->Nfn;
  ctx->Nu = ctx->ns * ctx->Np;
  ctx->Nq = d * ctx->Nu;
  ctx->Nt = ctx->ns * ctx->Nth;
  ctx->mapped = pr.mesh_kind == MEHDG_MESH_SHELL;
  ctx->nf = 2 * d;
  ctx->E = 1;
  ctx->F = 0;
  int npos[3] = {1, 1, 1};
  int goff[3] = {0, 0, 0};
  if (ctx->mapped) {
    // curved macros: sizes of the reference macro [0, 1]^3 (the tables then give d/dxi)
    ctx->E = 6 * pr.shell_n[0] * pr.shell_n[0] * pr.shell_n[1];
    const double r0 = pr.shell_r[0], r1 = pr.shell_r[1], q = pr.shell_r[2];
    const int nr = pr.shell_n[1];
    const double R1 = q == 1.0 ? r0 + (r1 - r0) / nr : r0 + (r1 - r0) * (q - 1.0) / (std::pow(q, (double)nr) - 1.0);
    for (int k = 0; k < 3; ++k) { ctx->hm[k] = 1.0; ctx->he[k] = 1.0 / pr.m; }
    ctx->h_supg = std::min(R1 - r0, r0 * M_PI / (2.0 * pr.shell_n[0])) / pr.m;
  } else {
    for (int k = 0; k < d; ++k) {
      ctx->E *= pr.nmac[k];
      npos[k] = pr.periodic[k] ? pr.nmac[k] : pr.nmac[k] + 1;
    }
    for (int k = 0; k < d; ++k) {
      goff[k] = ctx->F;
      int nt = 1;
      for (int j = 0; j < d; ++j)
        if (j != k) nt *= pr.nmac[j];
      ctx->F += npos[k] * nt;
    }
    ctx->ntr = (long long)ctx->F * ctx->ns * ctx->Nfn;
    double hmin = 1e300;
    for (int k = 0; k < 3; ++k) { ctx->hm[k] = 1.0; ctx->he[k] = 1.0; }
    for (int k = 0; k < d; ++k) {
      ctx->hm[k] = (pr.hi[k] - pr.lo[k]) / pr.nmac[k];
      ctx->he[k] = ctx->hm[k] / pr.m;
      hmin = std::min(hmin, ctx->he[k]);
    }
    ctx->h_supg = hmin;
  }
  ctx->ndir_v = ctx->ns * (1 + d);
  ctx->ndir_f = ctx->ns * (d + 2);

  // -- reference 1D data
  const int p = pr.p, n1 = ctx->n1, ng1 = ctx->ng1, m = pr.m;
  std::vector<double> xg, wg;
  gauss_rule(ng1, xg, wg);
  std::vector<double> xl = gll_nodes(p);
  ctx->b1.assign(ng1 * (p + 1), 0.0);
  ctx->db1.assign(ng1 * (p + 1), 0.0);
  for (int gq = 0; gq < ng1; ++gq) lagrange_at(xl, xg[gq], &ctx->b1[gq * (p + 1)], &ctx->db1[gq * (p + 1)]);
  ctx->gw = wg;
  // derivatives of the sub-element basis at xi = -1 and +1 (face Jacobians of curved macros)
  std::vector<double> dend(2 * (p + 1)), lend(p + 1);
  lagrange_at(xl, -1.0, lend.data(), dend.data());
  lagrange_at(xl, 1.0, lend.data(), dend.data() + (p + 1));

  // -- 1D macro matrices per axis: mass M1, C1[i][j] = int dphi_i phi_j, node coordinates
  std::vector<std::vector<double>> M1(d), C1(d), iM1(d), xn1(d);
  for (int k = 0; k < d; ++k) {
    M1[k].assign(n1 * n1, 0.0);
    C1[k].assign(n1 * n1, 0.0);
    xn1[k].assign(n1, 0.0);
    double he = ctx->he[k];
    for (int e = 0; e < m; ++e) {
      for (int i = 0; i <= p; ++i) xn1[k][e * p + i] = e * he + 0.5 * (xl[i] + 1.0) * he;
      for (int gq = 0; gq < ng1; ++gq) {
        double w = wg[gq] * he / 2;
        for (int i = 0; i <= p; ++i)
          for (int j = 0; j <= p; ++j) {
            double bi = ctx->b1[gq * (p + 1) + i], bj = ctx->b1[gq * (p + 1) + j];
            double dbi = ctx->db1[gq * (p + 1) + i] * 2.0 / he;
            M1[k][(e * p + i) * n1 + e * p + j] += w * bi * bj;
            C1[k][(e * p + i) * n1 + e * p + j] += w * dbi * bj;
          }
      }
    }
    xn1[k][0] = 0.0;
    xn1[k][n1 - 1] = ctx->hm[k];
    iM1[k] = M1[k];
    invert(iM1[k], n1);
  }
  const int Np = ctx->Np, Nth = ctx->Nth, Nfn = ctx->Nfn;
  std::vector<int> sq(3, n1);
  int R, C;
  std::vector<double> Mref, Minv, Gk(d * (size_t)Np * Np), Ghk(d * (size_t)Np * Nth, 0.0), tmp;
  {
    std::vector<const double*> f(d);
    for (int k = 0; k < d; ++k) f[k] = M1[k].data();
    kron_dense(d, n1, f, std::vector<int>(d, n1), Mref, R, C);
    for (int k = 0; k < d; ++k) f[k] = iM1[k].data();
    kron_dense(d, n1, f, std::vector<int>(d, n1), Minv, R, C);
    for (int kk = 0; kk < d; ++kk) {
      for (int k = 0; k < d; ++k) f[k] = (k == kk) ? C1[k].data() : M1[k].data();
      kron_dense(d, n1, f, std::vector<int>(d, n1), tmp, R, C);
      std::copy(tmp.begin(), tmp.end(), Gk.begin() + (size_t)kk * Np * Np);
    }
  }
  // face node tables and face mass matrices
  ctx->facenode.assign(2 * d * Nfn, 0);
  for (int fl = 0; fl < 2 * d; ++fl) {
    int k = fl / 2, side = fl % 2;
    for (int j = 0; j < Nfn; ++j) {
      int jj = j, idx[3] = {0, 0, 0};
      for (int kk = 0; kk < d; ++kk) {
        if (kk == k) idx[kk] = side ? n1 - 1 : 0;
        else { idx[kk] = jj % n1; jj /= n1; }
      }
      int a = 0;
      for (int kk = d - 1; kk >= 0; --kk) a = a * n1 + idx[kk];
      ctx->facenode[fl * Nfn + j] = a;
    }
    // face mass over tangential axes
    std::vector<const double*> f;
    std::vector<int> cols;
    for (int kk = 0; kk < d; ++kk)
      if (kk != k) { f.push_back(M1[kk].data()); cols.push_back(n1); }
    std::vector<double> Mf;
    if (d == 1) Mf.assign(1, 1.0);
    else kron_dense(d - 1, n1, f, cols, Mf, R, C);
    double nk = side ? 1.0 : -1.0;
    for (int j = 0; j < Nfn; ++j)
      for (int i = 0; i < Nfn; ++i)
        Ghk[(size_t)k * Np * Nth + (size_t)ctx->facenode[fl * Nfn + j] * Nth + fl * Nfn + i] -= nk * Mf[j * Nfn + i];
  }
  std::vector<double> Wk(d * (size_t)Np * Np, 0.0), Whk(d * (size_t)Np * Nth, 0.0);
  for (int k = 0; k < d; ++k)
    for (int a = 0; a < Np; ++a) {
      const double* mi = &Minv[(size_t)a * Np];
      for (int c = 0; c < Np; ++c) {
        double f = mi[c];
        if (f == 0.0) continue;
        const double* g = &Gk[(size_t)k * Np * Np + (size_t)c * Np];
        double* w = &Wk[(size_t)k * Np * Np + (size_t)a * Np];
        for (int b = 0; b < Np; ++b) w[b] += f * g[b];
        const double* gh = &Ghk[(size_t)k * Np * Nth + (size_t)c * Nth];
        double* wh = &Whk[(size_t)k * Np * Nth + (size_t)a * Nth];
        for (int i = 0; i < Nth; ++i) wh[i] += f * gh[i];
      }
    }

  // Kronecker factors of W_k and Wh_k: on a box macro M and G_k are products of 1D mass and
  // derivative matrices, so W_k = M^-1 G_k acts along axis k only and Wh_k lifts each face onto
  // the line normal to it.  The factors are read off the dense products and the whole
  // operators are checked against them; a mismatch keeps the dense condensation.
  std::vector<double> klift;
  if (n1 <= 8) {
    const int strides[3] = {1, n1, n1 * n1};
    klift.assign((size_t)d * n1 * n1 + 2 * d * n1, 0.0);
    for (int k = 0; k < d; ++k)
      for (int a = 0; a < n1; ++a) {
        for (int b = 0; b < n1; ++b)
          klift[(size_t)k * n1 * n1 + a * n1 + b] = Wk[(size_t)k * Np * Np + (size_t)a * strides[k] * Np + b * strides[k]];
      }
    for (int fl = 0; fl < 2 * d; ++fl) {
      const int k = fl / 2;
      for (int a = 0; a < n1; ++a)
        klift[(size_t)d * n1 * n1 + fl * n1 + a] = Whk[(size_t)k * Np * Nth + (size_t)a * strides[k] * Nth + fl * Nfn];
    }
    double wmax = 0.0, hmax = 0.0, werr = 0.0, herr = 0.0;
    for (size_t i = 0; i < Wk.size(); ++i) wmax = std::max(wmax, std::fabs(Wk[i]));
    for (size_t i = 0; i < Whk.size(); ++i) hmax = std::max(hmax, std::fabs(Whk[i]));
    auto digit = [&](int node, int k) { return (node / strides[k]) % n1; };
    for (int k = 0; k < d; ++k)
      for (int a = 0; a < Np; ++a) {
        for (int b = 0; b < Np; ++b) {
          bool line = true;
          for (int kk = 0; kk < d; ++kk)
            if (kk != k && digit(a, kk) != digit(b, kk)) line = false;
          const double ref = line ? klift[(size_t)k * n1 * n1 + digit(a, k) * n1 + digit(b, k)] : 0.0;
          werr = std::max(werr, std::fabs(Wk[(size_t)k * Np * Np + (size_t)a * Np + b] - ref));
        }
        for (int c = 0; c < Nth; ++c) {
          const int fl = c / Nfn, fn = ctx->facenode[c];
          bool line = fl / 2 == k;
          for (int kk = 0; kk < d && line; ++kk)
            if (kk != k && digit(a, kk) != digit(fn, kk)) line = false;
          const double ref = line ? klift[(size_t)d * n1 * n1 + fl * n1 + digit(a, k)] : 0.0;
          herr = std::max(herr, std::fabs(Whk[(size_t)k * Np * Nth + (size_t)a * Nth + c] - ref));
        }
      }
    if (!(werr <= 1e-12 * wmax && herr <= 1e-12 * hmax)) klift.clear();
  }
  if (ctx->mapped) klift.clear();   // per-macro (non-Kronecker) liftings on curved macros

  // -- maps
  std::vector<double> xnode_h;
  if (ctx->mapped) {
    int r_ = shell_maps(ctx, xn1[0], xnode_h);
    if (r_) return r_;
  }
  const int E = ctx->E, F = ctx->F, ns = ctx->ns, Nt = ctx->Nt;
  if (!ctx->mapped) {
  ctx->h_gather.assign((size_t)E * Nt, 0);
  ctx->h_owner.assign(2 * F, -1);
  ctx->h_bkind.assign(E * 2 * d, 0);
  ctx->h_bside.assign(E * 2 * d, -1);
  }
  for (int e = 0; e < E && !ctx->mapped; ++e) {
    int idx[3] = {0, 0, 0}, ee = e;
    for (int k = 0; k < d; ++k) { idx[k] = ee % pr.nmac[k]; ee /= pr.nmac[k]; }
    for (int k = 0; k < d; ++k)
      for (int side = 0; side < 2; ++side) {
        int fl = 2 * k + side;
        int pos = idx[k] + side;
        int bs = -1;
        if (pos == pr.nmac[k]) {
          if (pr.periodic[k]) pos = 0;
          else bs = 2 * k + 1;
        }
        if (pos == 0 && side == 0 && !pr.periodic[k]) bs = 2 * k;
        int loc = 0;
        for (int j = d - 1; j >= 0; --j)
          if (j != k) loc = loc * pr.nmac[j] + idx[j];
        int f = goff[k] + pos + npos[k] * loc;
        for (int s = 0; s < ns; ++s)
          for (int j = 0; j < Nfn; ++j)
            ctx->h_gather[(size_t)e * Nt + s * Nth + fl * Nfn + j] = (f * ns + s) * Nfn + j;
        int slotidx = (ctx->h_owner[2 * f] < 0) ? 0 : 1;
        if (ctx->h_owner[2 * f + slotidx] >= 0) return ctx_fail(ctx, MEHDG_ERR_ARG, "face with more than two owners");
        ctx->h_owner[2 * f + slotidx] = e * 2 * d + fl;
        ctx->h_bside[e * 2 * d + fl] = bs;
        ctx->h_bkind[e * 2 * d + fl] = bs >= 0 ? pr.bc[bs] : 0;
        if (bs >= 0 && pr.bc[bs] == MEHDG_BC_NONE)
          return ctx_fail(ctx, MEHDG_ERR_ARG, "boundary side without boundary condition");
      }
  }

  // -- device allocations
  const size_t Nu = ctx->Nu;
  ALLOC(ctx->gather, (size_t)E * Nt);
  ALLOC(ctx->owner, 2 * F);
  ALLOC(ctx->bkind, E * 2 * d);
  ALLOC(ctx->bside, E * 2 * d);
  ALLOC(ctx->fnode, 2 * d * Nfn);
  ALLOC(ctx->tab, 2 * ng1 * (p + 1) + 2 * ng1 + d * n1 + 2 * (p + 1));
  // geometric operators: one copy, or one per curved macro-element
  const size_t nge = ctx->mapped ? (size_t)E : 1;
  if (ctx->mapped) {
    ctx->sM = (size_t)Np * Np;
    ctx->sG = (size_t)d * Np * Np;
    ctx->sGh = (size_t)d * Np * Nth;
    ctx->sB = (size_t)d * Np * (Np + Nth);
  }
  ALLOC(ctx->Mref, nge * Np * Np);
  ALLOC(ctx->Minv, nge * Np * Np);
  ALLOC(ctx->Gk, nge * d * Np * Np);
  ALLOC(ctx->Ghk, nge * d * Np * Nth);
  ALLOC(ctx->Wk, nge * d * Np * Np);
  ALLOC(ctx->Whk, nge * d * Np * Nth);
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->gather, ctx->h_gather.data(), sizeof(int) * E * Nt, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->owner, ctx->h_owner.data(), sizeof(int) * 2 * F, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->bkind, ctx->h_bkind.data(), sizeof(int) * E * 2 * d, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->bside, ctx->h_bside.data(), sizeof(int) * E * 2 * d, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->fnode, ctx->facenode.data(), sizeof(int) * 2 * d * Nfn, cudaMemcpyHostToDevice, st));
  std::vector<double> tab;
  tab.insert(tab.end(), ctx->b1.begin(), ctx->b1.end());
  tab.insert(tab.end(), ctx->db1.begin(), ctx->db1.end());
  tab.insert(tab.end(), wg.begin(), wg.end());
  tab.insert(tab.end(), xg.begin(), xg.end());
  for (int k = 0; k < d; ++k) tab.insert(tab.end(), xn1[k].begin(), xn1[k].end());
  const size_t dend_off = tab.size();
  tab.insert(tab.end(), dend.begin(), dend.end());
  CK(cudaMemcpyAsync(ctx->tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st));
  if (ctx->mapped) {
    ALLOC(ctx->ofn, ctx->h_ofn.size());
    CK(cudaMemcpyAsync(ctx->ofn, ctx->h_ofn.data(), sizeof(int) * ctx->h_ofn.size(), cudaMemcpyHostToDevice, st));
    ALLOC(ctx->xnode, xnode_h.size());
    CK(cudaMemcpyAsync(ctx->xnode, xnode_h.data(), sizeof(double) * xnode_h.size(), cudaMemcpyHostToDevice, st));
    ALLOC(ctx->vgeo, (size_t)E * ctx->nel * ctx->Ng * (d * d + 1));
    ALLOC(ctx->fgeo, (size_t)E * 2 * d * ctx->nsf * ctx->nfp * (d + 1));
    ALLOC(ctx->dflag, 16);
    ALLOC(ctx->Bcat, (size_t)E * ctx->sB);
    int r_ = shell_geometry(ctx, ctx->tab + dend_off);
    if (r_) return r_;
  } else {
  CK(cudaMemcpyAsync(ctx->Mref, Mref.data(), sizeof(double) * Np * Np, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->Minv, Minv.data(), sizeof(double) * Np * Np, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->Gk, Gk.data(), sizeof(double) * d * Np * Np, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->Ghk, Ghk.data(), sizeof(double) * d * Np * Nth, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->Wk, Wk.data(), sizeof(double) * d * Np * Np, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->Whk, Whk.data(), sizeof(double) * d * Np * Nth, cudaMemcpyHostToDevice, st));
  }
  if (!klift.empty()) {
    ALLOC(ctx->klift, klift.size());
    CK(cudaMemcpyAsync(ctx->klift, klift.data(), sizeof(double) * klift.size(), cudaMemcpyHostToDevice, st));
  }
  if (!ctx->mapped) {
    // right factor of the fused condensation GEMM: [W_1 | -Wh_1; ...; W_d | -Wh_d], [d*Np][Np+Nth]
    const int nc = Np + Nth;
    std::vector<double> bc((size_t)d * Np * nc);
    for (int k = 0; k < d; ++k)
      for (int c = 0; c < Np; ++c) {
        double* row = bc.data() + ((size_t)k * Np + c) * nc;
        for (int j = 0; j < Np; ++j) row[j] = Wk[((size_t)k * Np + c) * Np + j];
        for (int j = 0; j < Nth; ++j) row[Np + j] = -Whk[((size_t)k * Np + c) * Nth + j];
      }
    ALLOC(ctx->Bcat, bc.size());
    CK(cudaMemcpy(ctx->Bcat, bc.data(), sizeof(double) * bc.size(), cudaMemcpyHostToDevice));
    if (ctx->opt.precision == MEHDG_PREC_MIXED) {
      std::vector<float> bc32(bc.begin(), bc.end());
      ALLOC(ctx->Bcat32, bc32.size());
      CK(cudaMemcpy(ctx->Bcat32, bc32.data(), sizeof(float) * bc32.size(), cudaMemcpyHostToDevice));
    }
  }
  CK(cudaStreamSynchronize(st));   // host vectors above go out of scope
  if (int r_ = setup_common(ctx, tab, Wk, Whk)) return r_;

  // closed-form data
  Geo g = make_geo(ctx);
  if (pr.field == MEHDG_FIELD_MMS || pr.field == MEHDG_FIELD_COUETTE3D) {
    long long tot = (long long)E * ctx->nel * ctx->Ng;
    ALLOC(ctx->src, tot * ns);
    int bs = 128;
    if (d == 2) k_source<2><<<(tot + bs - 1) / bs, bs, 0, st>>>(g, ctx->tab, pr, ctx->src);
    else k_source<3><<<(tot + bs - 1) / bs, bs, 0, st>>>(g, ctx->tab, pr, ctx->src);
    CKL();
    if (ctx->opt.precision == MEHDG_PREC_MIXED) {
      ALLOC(ctx->src32, tot * ns);
      if (int r_ = to_float(ctx, ctx->src, ctx->src32, tot * ns)) return r_;
    }
  }
  {
    long long tot = (long long)E * 2 * d * ctx->nsf * ctx->nfp;
    ALLOC(ctx->uD, tot * ns);
    int bs = 128;
    if (ctx->mapped) {
      int r_ = shell_bdata(ctx);
      if (r_) return r_;
    } else if (d == 2) {
      k_dirichlet<2><<<(tot + bs - 1) / bs, bs, 0, st>>>(g, ctx->tab, pr, ctx->bkind, ctx->uD);
    } else {
      k_dirichlet<3><<<(tot + bs - 1) / bs, bs, 0, st>>>(g, ctx->tab, pr, ctx->bkind, ctx->uD);
    }
    CKL();
    if (ctx->opt.precision == MEHDG_PREC_MIXED) {
      ALLOC(ctx->uD32, tot * ns);
      if (int r_ = to_float(ctx, ctx->uD, ctx->uD32, tot * ns)) return r_;
      ALLOC(ctx->uh32, ctx->ntr);
    }
  }
  CK(cudaStreamSynchronize(st));
  if (ctx->opt.apply_mode == 2) {
    int r_ = sparse_setup(ctx);
    if (r_) return r_;
  }
  if (ctx->opt.condense_layers == 1) {
    // one-layer condensation (FP64, explicit A^T_i): A_local of size NL = (d + 1) Nu must fit the
    // multi-right-hand-side solve (32 columns of NL doubles in shared memory)
    const size_t NL = (size_t)(d + 1) * Nu;
    if (ctx->opt.precision != MEHDG_PREC_FP64 || ctx->opt.apply_mode != 1)
      return ctx_fail(ctx, MEHDG_ERR_ARG, "condense_layers 1 needs precision FP64 and apply_mode 1");
    if (sizeof(double) * NL * 32 > 176 * 1024)
      return ctx_fail(ctx, MEHDG_ERR_ARG, "condense_layers 1: A_local too large for this degree (use the second layer)");
    ALLOC(ctx->Aloc, (size_t)E * NL * NL);
    ALLOC(ctx->Rloc, (size_t)E * NL * (Nt + 1));
    ALLOC(ctx->Xloc, (size_t)E * NL * (Nt + 1));
    ALLOC(ctx->permL, (size_t)E * NL);
  }
  return MEHDG_OK;
}

extern "C" int mehdg_mesh(mehdg_ctx** out, const mehdg_problem* prob, int nprob, const mehdg_options* opt,
                          void* stream) {
  if (!out || !prob) return MEHDG_ERR_ARG;
  *out = nullptr;
  if (nprob != 1) return MEHDG_ERR_ARG;
  const mehdg_problem& pr = prob[0];
  if (pr.dim < 2 || pr.dim > 3 || pr.m < 1 || pr.p < 1 || pr.p > 3 || pr.m * pr.p > 12) return MEHDG_ERR_ARG;
  if (pr.mesh_kind == MEHDG_MESH_SHELL) {
    // curved macros: FP64, second-layer condensation, per-macro M_J^-1 in shared memory (m p <= 4)
    if (pr.dim != 3 || pr.m * pr.p > 4 || pr.shell_n[0] < 1 || pr.shell_n[1] < 1 || !(pr.shell_r[0] > 0.0) ||
        !(pr.shell_r[1] > pr.shell_r[0]) || !(pr.shell_r[2] > 0.0))
      return MEHDG_ERR_ARG;
    if (pr.field != MEHDG_FIELD_UNIFORM && pr.field != MEHDG_FIELD_SPHERE) return MEHDG_ERR_ARG;
    for (int b = 0; b < 2; ++b)
      if (pr.bc[b] < MEHDG_BC_DIRICHLET || pr.bc[b] > MEHDG_BC_FARFIELD) return MEHDG_ERR_ARG;
    // (tc_mode 2 and 3 run the condensation with one lifting shared by all macro-elements)
    if (opt && (opt->condense_layers == 1 || opt->tc_mode == 2 || opt->tc_mode == 3)) return MEHDG_ERR_ARG;
  } else if (pr.mesh_kind == MEHDG_MESH_SIMPLEX) {
    // simplicial macros: FP64, second-layer condensation, the dense Algorithm-2 apply, SIMT
    // kernels, per-macro M^-1 and the sub-simplex tables in shared memory (m p <= 6)
    if (pr.m * pr.p > 6) return MEHDG_ERR_ARG;
    for (int k = 0; k < pr.dim; ++k)
      if (pr.nmac[k] < 1 || !(pr.hi[k] > pr.lo[k])) return MEHDG_ERR_ARG;
    if (opt && (opt->precision != MEHDG_PREC_FP64 || opt->apply_mode != 0 || opt->tc_mode != 0 ||
                opt->condense_layers != 2))
      return MEHDG_ERR_ARG;
  } else {
    if (pr.mesh_kind != MEHDG_MESH_BOX) return MEHDG_ERR_ARG;
    for (int k = 0; k < pr.dim; ++k)
      if (pr.nmac[k] < 1 || !(pr.hi[k] > pr.lo[k])) return MEHDG_ERR_ARG;
  }
  if (!(pr.gamma > 1.0) || !(pr.Re > 0.0) || !(pr.Pr > 0.0)) return MEHDG_ERR_ARG;
  if (opt && (opt->solver < 0 || opt->solver > 1 || opt->precond < 0 || opt->precond > 2 || opt->apply_mode < 0 ||
              opt->apply_mode > 2))
    return MEHDG_ERR_ARG;
  mehdg_ctx* ctx = new mehdg_ctx();
  ctx->prob = pr;
  default_options(&ctx->opt);
  if (opt) ctx->opt = *opt;
  ctx->stream = (cudaStream_t)stream;
  // tc_mode: 0 SIMT; 1 tensor cores (split TF32) for the LU trailing updates only;
  // 2 split TF32 for LU, condensation and forming A^T_i; 3 plain TF32 everywhere
  ctx->use_tc_lu = ctx->opt.tc_mode >= 1 && ctx->opt.tc_mode <= 3;
  ctx->use_tc_condense = ctx->use_tc_form = ctx->opt.tc_mode == 2 || ctx->opt.tc_mode == 3;
  ctx->tc_split = ctx->opt.tc_mode <= 2;
  // 4: forming A^T_i on tcgen05 with the swizzled K-major product (D += B (S^-1 C)), the rest SIMT
  ctx->use_tc_nt = ctx->opt.tc_mode == 4;
  int rc = setup(ctx);
  if (rc != MEHDG_OK) {
    std::string msg = ctx->err;
    mehdg_destroy(ctx);
    fprintf(stderr, "mehdg_mesh: %s\n", msg.c_str());
    return rc;
  }
  *out = ctx;
  return MEHDG_OK;
}

extern "C" int mehdg_query(const mehdg_ctx* c, mehdg_info* info) {
  if (!c || !info) return MEHDG_ERR_ARG;
  info->dim = c->d; info->ns = c->ns; info->Np = c->Np; info->Nfn = c->Nfn; info->Nth = c->Nth;
  info->Nu = c->Nu; info->Nq = c->Nq; info->Nt = c->Nt; info->n_macro = c->E; info->n_face = c->F;
  info->n_trace = c->ntr; info->bytes_device = c->bytes;
  return MEHDG_OK;
}

extern "C" int mehdg_init_state(mehdg_ctx* ctx, const double* du, const double* duh, int lift, double* u,
                                double* q, double* uh) {
  if (!ctx || !u || !q || !uh) return MEHDG_ERR_ARG;
  Geo g = make_geo(ctx);
  cudaStream_t st = ctx->stream;
  long long tot = (long long)ctx->E * ctx->Np;
  int bs = 128;
  if (ctx->simplex) {
    int r_ = sx_init_state(ctx, du, u);
    if (r_) return r_;
  } else if (ctx->mapped) {
    int r_ = shell_init_state(ctx, du, u);
    if (r_) return r_;
  } else {
    const double* xnode1 = ctx->tab + 2 * ctx->ng1 * (ctx->p + 1) + 2 * ctx->ng1;
    if (ctx->d == 2) k_init_state<2><<<(tot + bs - 1) / bs, bs, 0, st>>>(g, ctx->prob, xnode1, du, u);
    else k_init_state<3><<<(tot + bs - 1) / bs, bs, 0, st>>>(g, ctx->prob, xnode1, du, u);
    CKL();
  }
  k_init_trace<<<(ctx->ntr + bs - 1) / bs, bs, 0, st>>>(g, ctx->owner, ctx->fnode, u, duh, uh, ctx->F);
  CKL();
  long long nq = (long long)ctx->E * ctx->Nq;
  if (lift) {
    k_lift<<<(nq + bs - 1) / bs, bs, 0, st>>>(g, ctx->Wk, ctx->Whk, ctx->gather, u, uh, q, ctx->E, ctx->sG,
                                              ctx->sGh);
    CKL();
  } else {
    CK(cudaMemsetAsync(q, 0, sizeof(double) * nq, st));
  }
  return MEHDG_OK;
}

extern "C" int mehdg_get_block(mehdg_ctx* ctx, int which, int e, double* out, long long* count) {
  if (!ctx || e < 0 || e >= ctx->E) return MEHDG_ERR_ARG;
  const size_t Nu = ctx->Nu, Nt = ctx->Nt, d = ctx->d;
  const double* src = nullptr;
  size_t n = 0;
  bool ints = false;
  const int* isrc = nullptr;
  switch (which) {
    case 0: src = ctx->Auu + e * Nu * Nu; n = Nu * Nu; break;
    case 1: case 2: case 3:
      if (which > (int)d) return MEHDG_ERR_ARG;
      src = ctx->Auq + (e * d + (which - 1)) * Nu * Nu; n = Nu * Nu; break;
    case 4: src = ctx->Auh + e * Nu * Nt; n = Nu * Nt; break;
    case 5: src = ctx->Ahu + e * Nt * Nu; n = Nt * Nu; break;
    case 6: case 7: case 8:
      if (which - 5 > (int)d) return MEHDG_ERR_ARG;
      src = ctx->Ahq + (e * d + (which - 6)) * Nt * Nu; n = Nt * Nu; break;
    case 9: src = ctx->Ahh + e * Nt * Nt; n = Nt * Nt; break;
    case 10: src = ctx->RQ + e * d * Nu; n = d * Nu; break;
    case 11: src = ctx->RU + e * Nu; n = Nu; break;
    case 12: src = ctx->RUh + e * Nt; n = Nt; break;
    case 13: src = ctx->gv + e * Nu; n = Nu; break;
    case 14: src = ctx->hv + e * Nt; n = Nt; break;
    case 15: isrc = ctx->perm + e * Nu; n = Nu; ints = true; break;
    case 16: src = ctx->bloc + e * Nt; n = Nt; break;
    case 17:
      if (!ctx->S32) return MEHDG_ERR_ARG;
      n = Nu * Nu; break;
    default: return MEHDG_ERR_ARG;
  }
  if (count) *count = (long long)n;
  if (!out) return MEHDG_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  if (ints) {
    std::vector<int> tmp(n);
    CK(cudaMemcpy(tmp.data(), isrc, sizeof(int) * n, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) out[i] = tmp[i];
  } else if (which == 17) {
    std::vector<float> tmp(n);
    CK(cudaMemcpy(tmp.data(), ctx->S32 + e * Nu * Nu, sizeof(float) * n, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) out[i] = tmp[i];
  } else if (ctx->opt.precision == MEHDG_PREC_MIXED && which <= 9) {
    // blocks are FP32 in the mixed-precision path (same element offsets)
    const float* fsrc = nullptr;
    std::vector<float> tmp(n);
    const double* base = nullptr;
    size_t idx = 0;
    switch (which) {
      case 0: base = ctx->Auu; idx = e * Nu * Nu; break;
      case 1: case 2: case 3: base = ctx->Auq; idx = (e * d + (which - 1)) * Nu * Nu; break;
      case 4: base = ctx->Auh; idx = e * Nu * Nt; break;
      case 5: base = ctx->Ahu; idx = e * Nt * Nu; break;
      case 6: case 7: case 8: base = ctx->Ahq; idx = (e * d + (which - 6)) * Nt * Nu; break;
      default: base = ctx->Ahh; idx = e * Nt * Nt; break;
    }
    fsrc = reinterpret_cast<const float*>(base) + idx;
    CK(cudaMemcpy(tmp.data(), fsrc, sizeof(float) * n, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) out[i] = tmp[i];
  } else {
    CK(cudaMemcpy(out, src, sizeof(double) * n, cudaMemcpyDeviceToHost));
  }
  return MEHDG_OK;
}

extern "C" void mehdg_destroy(mehdg_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  void* ptrs[] = {ctx->gather, ctx->owner, ctx->bkind, ctx->bside, ctx->fnode, ctx->tab, ctx->Mref, ctx->Minv,
                  ctx->Gk, ctx->Ghk, ctx->Wk, ctx->Whk, ctx->src, ctx->uD, ctx->Auu, ctx->Auq, ctx->Auh,
                  ctx->Ahu, ctx->Ahq, ctx->Ahh, ctx->perm, ctx->RQ, ctx->RU, ctx->RUh, ctx->gv, ctx->hv,
                  ctx->MinvRQ, ctx->bloc, ctx->slot, ctx->Kvol, ctx->rvol, ctx->Kface, ctx->rface, ctx->fblk,
                  ctx->fperm, ctx->dflag, ctx->dred, ctx->S32,
                  ctx->V, ctx->Zk, ctx->wv, ctx->tv, ctx->tv2, ctx->rv, ctx->iV, ctx->iw, ctx->un,
                  ctx->ustage, ctx->hist, ctx->du, ctx->dq, ctx->duh, ctx->bhat, ctx->Xbuf, ctx->Wk32,
                  ctx->Whk32, ctx->dtcerr, ctx->finv32, ctx->u32, ctx->q32, ctx->h32, ctx->tab32, ctx->src32,
                  ctx->uD32, ctx->uh32, ctx->Bcat, ctx->Bcat32, ctx->klift, ctx->Aloc, ctx->Rloc, ctx->Xloc, ctx->permL, ctx->dHo, ctx->dHi, ctx->gin, ctx->gout, ctx->Ahat16, ctx->finv16,
                  ctx->vgeo, ctx->fgeo, ctx->xnode, ctx->ofn, ctx->ddiag, ctx->sx_vtab, ctx->sx_vnode, ctx->sx_ftab, ctx->sx_fsub};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ctx->hred) cudaFreeHost(ctx->hred);
  if (ctx->ig_exec) cudaGraphExecDestroy(ctx->ig_exec);
  if (ctx->xstart) cudaFree(ctx->xstart);
  mlp_destroy(ctx);
  sparse_destroy(ctx);
  for (int i = 0; i < 2 * PH_COUNT; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (int p = 0; p < PH_COUNT; ++p) {
    for (cudaEvent_t x : ctx->ring_b[p]) cudaEventDestroy(x);
    for (cudaEvent_t x : ctx->ring_e[p]) cudaEventDestroy(x);
  }
  delete ctx;
}

extern "C" const char* mehdg_last_error(const mehdg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
