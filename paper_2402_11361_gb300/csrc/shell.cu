// a0 / a3 for curved macro-elements: the cubed-sphere shell mesh of the flow past a sphere
// (Sec. 5.2 workload; the paper's own mesh is an unstructured tetrahedral one) and the
// geometric data of isoparametric macro-elements.
//
// Mesh (host): 6 cube panels x nq x nq equiangular cells x nr radial layers; the macro node
// with macro-lattice coordinates t in [0, 1]^3 of cell (i, j, k) on panel (e_n, e_1, e_2) sits
// at R(k + t_2) dir / |dir|, dir = e_n + tan(a) e_1 + tan(b) e_2 with the equiangular angles
// a, b of (i + t_0) and (j + t_1).  Faces are numbered in order of first appearance over
// (macro, local face), their nodes in the first owner's order; the second owner's nodes are
// matched by position, which gives its gather map and the owner's node map ofn.
//
// Geometry (device): the map x(xi) = sum_a x_a phi_a(xi) is the macro's own C0 interpolant of
// the node positions.  Per volume point: J = dx/dxi, J^-1 and the weight (reference weight x
// det J); per face point: the area-weighted outward normal +-det J (J^-T e_k), stored as unit
// normal and weight.  Per macro-element: M_J = int phi_a phi_b, G_k = int d_k phi_a phi_b,
// Gh_k = -sum_faces int phi_a n_k psi_j (the linear blocks of R_Q, so A_qq = I (x) M_J), the
// inverse of M_J (Gauss-Jordan in shared memory: M_J is symmetric positive definite), the
// liftings W_k = M_J^-1 G_k, Wh_k = M_J^-1 Gh_k and the right factor [W_k | -Wh_k] of the
// condensation product.
#include <cmath>
#include <unordered_map>

#include "internal.cuh"
#include "physics.cuh"

namespace {

template <int B, int E> struct SPow { static constexpr int v = B * SPow<B, E - 1>::v; };
template <int B> struct SPow<B, 0> { static constexpr int v = 1; };

// cube-panel frames (e_n, e_1, e_2), e_1 x e_2 = e_n: panels +x, -x, +y, -y, +z, -z
const int kFrames[6][3][3] = {{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},  {{-1, 0, 0}, {0, 0, 1}, {0, 1, 0}},
                              {{0, 1, 0}, {0, 0, 1}, {1, 0, 0}},  {{0, -1, 0}, {1, 0, 0}, {0, 0, 1}},
                              {{0, 0, 1}, {1, 0, 0}, {0, 1, 0}},  {{0, 0, -1}, {0, 1, 0}, {1, 0, 0}}};

double shell_R(double s, const mehdg_problem& pr) {
  const double r0 = pr.shell_r[0], r1 = pr.shell_r[1], q = pr.shell_r[2];
  const int nr = pr.shell_n[1];
  if (q == 1.0) return r0 + (r1 - r0) * s / nr;
  return r0 + (r1 - r0) * (std::pow(q, s) - 1.0) / (std::pow(q, (double)nr) - 1.0);
}

template <int D>
__device__ __forceinline__ double det_inv(const double (*J)[D], double (*Ji)[D]) {
  if constexpr (D == 2) {
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    return det;
  } else {
    double C[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        C[i][j] = J[i1][j1] * J[i2][j2] - J[i1][j2] * J[i2][j1];
      }
    const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Ji[i][j] = C[j][i] / det;
    return det;
  }
}

// table layout: b1 [NG1][P1], db1 [NG1][P1], Gauss weights, Gauss points, macro node
// coordinates [d][n1], then the derivatives of the sub-element basis at xi = -1 and +1 [2][P1]
template <int D, int P>
__global__ void k_geo_vol(Geo g, const double* __restrict__ tab, const double* __restrict__ xnode,
                          double* __restrict__ vgeo, int* __restrict__ flag, int E) {
  constexpr int P1 = P + 1, NG1 = P + 2, NLOC = SPow<P1, D>::v, NG = SPow<NG1, D>::v;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)E * g.nel * NG) return;
  const int gq = tid % NG;
  const int el = (tid / NG) % g.nel;
  const int e = (int)(tid / ((long long)NG * g.nel));
  const double* b1 = tab;
  const double* db1 = tab + NG1 * P1;
  const double* gw = tab + 2 * NG1 * P1;
  int gi[D], li[D];
  double w = 1.0;
  for (int k = 0, gg = gq, ll = el; k < D; ++k) {
    gi[k] = gg % NG1; gg /= NG1;
    li[k] = ll % g.m; ll /= g.m;
    w *= gw[gi[k]] * 0.5 * g.he[k];
  }
  double J[D][D] = {};
  for (int al = 0; al < NLOC; ++al) {
    int ai[D], a = 0;
    for (int k = 0, aa = al, st = 1; k < D; ++k) {
      ai[k] = aa % P1; aa /= P1;
      a += (li[k] * P + ai[k]) * st;
      st *= g.n1;
    }
    double bv[D], dv[D];
    for (int k = 0; k < D; ++k) {
      bv[k] = b1[gi[k] * P1 + ai[k]];
      dv[k] = db1[gi[k] * P1 + ai[k]] * 2.0 / g.he[k];
    }
    for (int j = 0; j < D; ++j) {
      double dphi = dv[j];
      for (int k = 0; k < D; ++k)
        if (k != j) dphi *= bv[k];
      for (int i = 0; i < D; ++i) J[i][j] += xnode[((size_t)e * D + i) * g.Np + a] * dphi;
    }
  }
  double Ji[D][D];
  const double det = det_inv<D>(J, Ji);
  if (!(det > 0.0)) atomicOr(flag, 1);
  double* out = vgeo + tid * (D * D + 1);
  for (int j = 0; j < D; ++j)
    for (int k = 0; k < D; ++k) out[j * D + k] = Ji[j][k];
  out[D * D] = w * det;
}

template <int D, int P>
__global__ void k_geo_face(Geo g, const double* __restrict__ tab, const double* __restrict__ dend,
                           const double* __restrict__ xnode, double* __restrict__ fgeo, int* __restrict__ flag,
                           int E) {
  constexpr int P1 = P + 1, NG1 = P + 2, NLOC = SPow<P1, D>::v, NFP = SPow<NG1, D - 1>::v;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)E * 2 * D * g.nsf * NFP) return;
  const int fp = tid % NFP;
  const int sf = (tid / NFP) % g.nsf;
  const int fl = (tid / ((long long)NFP * g.nsf)) % (2 * D);
  const int e = (int)(tid / ((long long)NFP * g.nsf * 2 * D));
  const int kn = fl / 2, side = fl % 2;
  const double* b1 = tab;
  const double* db1 = tab + NG1 * P1;
  const double* gw = tab + 2 * NG1 * P1;
  int gi[D], li[D];
  double wref = 1.0;
  for (int k = 0, c = 0, pp = fp, ss = sf; k < D; ++k) {
    if (k == kn) { gi[k] = -1; li[k] = side ? g.m - 1 : 0; continue; }
    gi[k] = pp % NG1; pp /= NG1;
    li[k] = ss % g.m; ss /= g.m;
    wref *= gw[gi[k]] * 0.5 * g.he[k];
    ++c;
  }
  double J[D][D] = {};
  for (int al = 0; al < NLOC; ++al) {
    int ai[D], a = 0;
    for (int k = 0, aa = al, st = 1; k < D; ++k) {
      ai[k] = aa % P1; aa /= P1;
      a += (li[k] * P + ai[k]) * st;
      st *= g.n1;
    }
    double bv[D], dv[D];
    for (int k = 0; k < D; ++k) {
      if (k == kn) {
        bv[k] = (ai[k] == (side ? P : 0)) ? 1.0 : 0.0;
        dv[k] = dend[side * P1 + ai[k]] * 2.0 / g.he[k];
      } else {
        bv[k] = b1[gi[k] * P1 + ai[k]];
        dv[k] = db1[gi[k] * P1 + ai[k]] * 2.0 / g.he[k];
      }
    }
    for (int j = 0; j < D; ++j) {
      double dphi = dv[j];
      for (int k = 0; k < D; ++k)
        if (k != j) dphi *= bv[k];
      for (int i = 0; i < D; ++i) J[i][j] += xnode[((size_t)e * D + i) * g.Np + a] * dphi;
    }
  }
  double Ji[D][D];
  const double det = det_inv<D>(J, Ji);
  if (!(det > 0.0)) atomicOr(flag, 2);
  double nw[D], area = 0.0;
  for (int i = 0; i < D; ++i) {
    nw[i] = (side ? 1.0 : -1.0) * det * Ji[kn][i];
    area += nw[i] * nw[i];
  }
  area = sqrt(area);
  double* out = fgeo + tid * (D + 1);
  for (int i = 0; i < D; ++i) out[i] = nw[i] / area;
  out[D] = wref * area;
}

// M_J[a][b] and G_k[a][b] of every macro-element, one thread per (macro, a, b)
template <int D, int P>
__global__ void k_geo_mats(Geo g, const double* __restrict__ tab, const double* __restrict__ vgeo,
                           double* __restrict__ Mo, double* __restrict__ Go, int E) {
  constexpr int P1 = P + 1, NG1 = P + 2, NG = SPow<NG1, D>::v;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int Np = g.Np;
  if (tid >= (long long)E * Np * Np) return;
  const int b = tid % Np;
  const int a = (tid / Np) % Np;
  const int e = (int)(tid / ((long long)Np * Np));
  const double* b1 = tab;
  const double* db1 = tab + NG1 * P1;
  int ia[D], ib[D];
  for (int k = 0, aa = a, bb = b; k < D; ++k) {
    ia[k] = aa % g.n1; aa /= g.n1;
    ib[k] = bb % g.n1; bb /= g.n1;
  }
  double M = 0.0, G[D] = {};
  for (int el = 0; el < g.nel; ++el) {
    int ra[D], rb[D];
    bool in = true;
    for (int k = 0, ll = el; k < D; ++k) {
      const int lk = ll % g.m;
      ll /= g.m;
      ra[k] = ia[k] - lk * P;
      rb[k] = ib[k] - lk * P;
      if (ra[k] < 0 || ra[k] > P || rb[k] < 0 || rb[k] > P) in = false;
    }
    if (!in) continue;
    for (int gq = 0; gq < NG; ++gq) {
      int gi[D];
      for (int k = 0, gg = gq; k < D; ++k) { gi[k] = gg % NG1; gg /= NG1; }
      double pa = 1.0, pb = 1.0, dref[D];
      for (int k = 0; k < D; ++k) {
        pa *= b1[gi[k] * P1 + ra[k]];
        pb *= b1[gi[k] * P1 + rb[k]];
      }
      for (int j = 0; j < D; ++j) {
        double v = db1[gi[j] * P1 + ra[j]] * 2.0 / g.he[j];
        for (int k = 0; k < D; ++k)
          if (k != j) v *= b1[gi[k] * P1 + ra[k]];
        dref[j] = v;
      }
      const double* vg = vgeo + (((size_t)e * g.nel + el) * NG + gq) * (D * D + 1);
      const double w = vg[D * D];
      M += w * pa * pb;
      for (int k = 0; k < D; ++k) {
        double dk = 0.0;
        for (int j = 0; j < D; ++j) dk += vg[j * D + k] * dref[j];
        G[k] += w * dk * pb;
      }
    }
  }
  Mo[tid] = M;
  for (int k = 0; k < D; ++k) Go[(((size_t)e * D + k) * Np + a) * Np + b] = G[k];
}

// Gh_k[a][(f, j)] = -sum over the face points of phi_a w n_k psi_j, one thread per (macro, a, c)
template <int D, int P>
__global__ void k_geo_ghk(Geo g, const double* __restrict__ tab, const double* __restrict__ fgeo,
                          double* __restrict__ Gho, int E) {
  constexpr int P1 = P + 1, NG1 = P + 2, NFP = SPow<NG1, D - 1>::v;
  const int Np = g.Np, Nth = g.Nth, Nfn = g.Nfn;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)E * Np * Nth) return;
  const int c = tid % Nth;
  const int a = (tid / Nth) % Np;
  const int e = (int)(tid / ((long long)Nth * Np));
  const int fl = c / Nfn, jf = c % Nfn;
  const int kn = fl / 2, side = fl % 2;
  const double* b1 = tab;
  int ia[D];
  for (int k = 0, aa = a; k < D; ++k) { ia[k] = aa % g.n1; aa /= g.n1; }
  double acc[D] = {};
  if (ia[kn] == (side ? g.n1 - 1 : 0)) {
    int at[D], jt[D], nt = 0;
    for (int k = 0, jj = jf; k < D; ++k) {
      if (k == kn) continue;
      at[nt] = ia[k];
      jt[nt] = jj % g.n1;
      jj /= g.n1;
      ++nt;
    }
    for (int sf = 0; sf < g.nsf; ++sf) {
      int ra[D], rj[D];
      bool in = true;
      for (int cc = 0, ss = sf; cc < D - 1; ++cc) {
        const int sc = ss % g.m;
        ss /= g.m;
        ra[cc] = at[cc] - sc * P;
        rj[cc] = jt[cc] - sc * P;
        if (ra[cc] < 0 || ra[cc] > P || rj[cc] < 0 || rj[cc] > P) in = false;
      }
      if (!in) continue;
      for (int fp = 0; fp < NFP; ++fp) {
        double v = 1.0;
        for (int cc = 0, pp = fp; cc < D - 1; ++cc) {
          const int gc = pp % NG1;
          pp /= NG1;
          v *= b1[gc * P1 + ra[cc]] * b1[gc * P1 + rj[cc]];
        }
        const double* fg = fgeo + ((((size_t)e * 2 * D + fl) * g.nsf + sf) * NFP + fp) * (D + 1);
        for (int k = 0; k < D; ++k) acc[k] += v * fg[D] * fg[k];
      }
    }
  }
  for (int k = 0; k < D; ++k) Gho[(((size_t)e * D + k) * Np + a) * Nth + c] = -acc[k];
}

// one CTA per macro-element: M_J^-1 by Gauss-Jordan in shared memory, then W_k = M_J^-1 G_k,
// Wh_k = M_J^-1 Gh_k and the condensation factor [W_k | -Wh_k]
__global__ void __launch_bounds__(256) k_geo_lift(int d, int Np, int Nth, const double* __restrict__ Mj,
                                                  const double* __restrict__ Gk, const double* __restrict__ Ghk,
                                                  double* __restrict__ Minv, double* __restrict__ Wk,
                                                  double* __restrict__ Whk, double* __restrict__ Bcat) {
  extern __shared__ double sh[];
  double* A = sh;               // [Np][Np]
  double* row = A + Np * Np;    // [Np]
  double* col = row + Np;       // [Np]
  const int e = blockIdx.x;
  const size_t NN = (size_t)Np * Np;
  for (int i = threadIdx.x; i < Np * Np; i += blockDim.x) A[i] = Mj[e * NN + i];
  __syncthreads();
  for (int c = 0; c < Np; ++c) {
    const double p = 1.0 / A[c * Np + c];
    for (int i = threadIdx.x; i < Np; i += blockDim.x) {
      row[i] = A[c * Np + i] * p;
      col[i] = A[i * Np + c];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Np * Np; t += blockDim.x) {
      const int i = t / Np, j = t % Np;
      if (i == c && j == c) A[t] = p;
      else if (i == c) A[t] = row[j];
      else if (j == c) A[t] = -col[i] * p;
      else A[t] -= col[i] * row[j];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < Np * Np; i += blockDim.x) Minv[e * NN + i] = A[i];
  const int ncol = d * Np + d * Nth, nb = Np + Nth;
  for (int q = threadIdx.x; q < ncol; q += blockDim.x) {
    const bool hat = q >= d * Np;
    const int k = hat ? (q - d * Np) / Nth : q / Np;
    const int b = hat ? (q - d * Np) % Nth : q % Np;
    const double* R = hat ? Ghk + (((size_t)e * d + k) * Np) * Nth + b : Gk + (((size_t)e * d + k) * Np) * Np + b;
    const int ld = hat ? Nth : Np;
    for (int a0 = 0; a0 < Np; a0 += 8) {
      double acc[8] = {};
      for (int cc = 0; cc < Np; ++cc) {
        const double r = R[(size_t)cc * ld];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (a0 + i < Np) acc[i] += A[(a0 + i) * Np + cc] * r;
      }
      for (int i = 0; i < 8 && a0 + i < Np; ++i) {
        const int a = a0 + i;
        double* brow = Bcat + (size_t)e * d * Np * nb + ((size_t)k * Np + a) * nb;
        if (hat) {
          Whk[(((size_t)e * d + k) * Np + a) * Nth + b] = acc[i];
          brow[Np + b] = -acc[i];
        } else {
          Wk[(((size_t)e * d + k) * Np + a) * Np + b] = acc[i];
          brow[b] = acc[i];
        }
      }
    }
  }
}

// Dirichlet and far-field data of the shell: the uniform state of field_par at every face point
template <int D>
__global__ void k_shell_bdata(long long npt, int per_e, mehdg_problem pr, const int* __restrict__ bkind,
                              double* __restrict__ uD) {
  constexpr int NS = D + 2;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= npt) return;
  const int ef = (int)(tid / per_e);   // e * 2D + fl
  const int bk = bkind[ef];
  double u[NS];
  field_uniform<D>(pr.field_par, pr.gamma, u);
  for (int s = 0; s < NS; ++s)
    uD[tid * NS + s] = (bk == MEHDG_BC_DIRICHLET || bk == MEHDG_BC_FARFIELD) ? u[s] : 0.0;
}

// initial state at the nodes: the free stream with the velocity blended to zero near the
// sphere (FIELD_SPHERE) or the uniform state of field_par
__global__ void k_shell_init(long long n, int Np, mehdg_problem pr, const double* __restrict__ xnode,
                             const double* __restrict__ du, double* __restrict__ u) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= n) return;
  const int a = tid % Np;
  const long long e = tid / Np;
  double x[3], r2 = 0.0;
  for (int i = 0; i < 3; ++i) {
    x[i] = xnode[(e * 3 + i) * Np + a];
    r2 += x[i] * x[i];
  }
  double beta = 1.0;
  if (pr.field == MEHDG_FIELD_SPHERE) {
    double s = (sqrt(r2) - 0.6) / 0.4;
    s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
    beta = s * s * (3.0 - 2.0 * s);
  }
  double par[8];
  for (int i = 0; i < 8; ++i) par[i] = pr.field_par[i];
  for (int i = 0; i < 3; ++i) par[1 + i] *= beta;
  double uu[5];
  field_uniform<3>(par, pr.gamma, uu);
  for (int s = 0; s < 5; ++s) {
    const long long o = (e * 5 + s) * Np + a;
    u[o] = uu[s] + (du ? du[o] : 0.0);
  }
}

template <int P>
int geometry_p(mehdg_ctx* ctx, const double* dend) {
  constexpr int D = 3;
  Geo g = make_geo(ctx);
  cudaStream_t st = ctx->stream;
  const int E = ctx->E, Np = ctx->Np, Nth = ctx->Nth;
  constexpr int NG = SPow<P + 2, D>::v, NFP = SPow<P + 2, D - 1>::v;
  CK(cudaMemsetAsync(ctx->dflag, 0, sizeof(int) * 16, st));
  long long n = (long long)E * ctx->nel * NG;
  k_geo_vol<D, P><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, ctx->tab, ctx->xnode, ctx->vgeo, ctx->dflag, E);
  CKL();
  n = (long long)E * 2 * D * ctx->nsf * NFP;
  k_geo_face<D, P><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, ctx->tab, dend, ctx->xnode, ctx->fgeo,
                                                                ctx->dflag, E);
  CKL();
  n = (long long)E * Np * Np;
  k_geo_mats<D, P><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, ctx->tab, ctx->vgeo, ctx->Mref, ctx->Gk, E);
  CKL();
  n = (long long)E * Np * Nth;
  k_geo_ghk<D, P><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, ctx->tab, ctx->fgeo, ctx->Ghk, E);
  CKL();
  const size_t smem = sizeof(double) * ((size_t)Np * Np + 2 * Np);
  CK(cudaFuncSetAttribute(k_geo_lift, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_geo_lift<<<E, 256, smem, st>>>(D, Np, Nth, ctx->Mref, ctx->Gk, ctx->Ghk, ctx->Minv, ctx->Wk, ctx->Whk,
                                   ctx->Bcat);
  CKL();
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag) return ctx_fail(ctx, MEHDG_ERR_ARG, "shell mesh: non-positive Jacobian of the isoparametric map");
  return MEHDG_OK;
}

}  // namespace

// host: node positions, face numbering, gather / owner / node maps and boundary kinds of the
// shell mesh.  t: the n1 macro-lattice coordinates in [0, 1].
int shell_maps(mehdg_ctx* ctx, const std::vector<double>& t, std::vector<double>& xnode) {
  const mehdg_problem& pr = ctx->prob;
  const int nq = pr.shell_n[0], nr = pr.shell_n[1], n1 = ctx->n1, Np = ctx->Np, Nfn = ctx->Nfn;
  const int ns = ctx->ns, Nt = ctx->Nt, Nth = ctx->Nth;
  const int E = ctx->E;
  const double PI = 3.14159265358979323846;
  xnode.assign((size_t)E * 3 * Np, 0.0);
  for (int e = 0; e < E; ++e) {
    const int i = e % nq, j = (e / nq) % nq, k = (e / (nq * nq)) % nr, pan = e / (nq * nq * nr);
    for (int a = 0; a < Np; ++a) {
      const int i0 = a % n1, i1 = (a / n1) % n1, i2 = a / (n1 * n1);
      const double ta = std::tan(-0.25 * PI + (i + t[i0]) * 0.5 * PI / nq);
      const double tb = std::tan(-0.25 * PI + (j + t[i1]) * 0.5 * PI / nq);
      const double R = shell_R(k + t[i2], pr);
      double dir[3], nrm = 0.0;
      for (int c = 0; c < 3; ++c) {
        dir[c] = kFrames[pan][0][c] + ta * kFrames[pan][1][c] + tb * kFrames[pan][2][c];
        nrm += dir[c] * dir[c];
      }
      nrm = std::sqrt(nrm);
      for (int c = 0; c < 3; ++c) xnode[((size_t)e * 3 + c) * Np + a] = R * dir[c] / nrm;
    }
  }
  // faces: match the centroids of the face nodes on a grid of cells of size tol_cell
  const double r1 = pr.shell_r[1];
  const double tol = 1e-9 * r1, cell = 1e-6 * r1;
  auto key3 = [&](long long x, long long y, long long z) {
    return (unsigned long long)(x * 73856093LL) ^ (unsigned long long)(y * 19349663LL) ^
           (unsigned long long)(z * 83492791LL);
  };
  std::unordered_multimap<unsigned long long, int> grid;
  std::vector<double> cen;   // [F][3]
  std::vector<int> first;    // first owner (e * 6 + fl) of each face
  ctx->h_gather.assign((size_t)E * Nt, 0);
  ctx->h_bkind.assign(E * 6, 0);
  ctx->h_bside.assign(E * 6, -1);
  std::vector<int> fid(E * 6, -1);
  int F = 0;
  std::vector<int> owner2;   // second owner per face (-1)
  for (int e = 0; e < E; ++e) {
    for (int fl = 0; fl < 6; ++fl) {
      double c[3] = {0.0, 0.0, 0.0};
      for (int jf = 0; jf < Nfn; ++jf) {
        const int a = ctx->facenode[fl * Nfn + jf];
        for (int q = 0; q < 3; ++q) c[q] += xnode[((size_t)e * 3 + q) * Np + a];
      }
      for (int q = 0; q < 3; ++q) c[q] /= Nfn;
      long long ic[3];
      for (int q = 0; q < 3; ++q) ic[q] = (long long)std::floor(c[q] / cell);
      int found = -1;
      for (int dx = -1; dx <= 1 && found < 0; ++dx)
        for (int dy = -1; dy <= 1 && found < 0; ++dy)
          for (int dz = -1; dz <= 1 && found < 0; ++dz) {
            auto rg = grid.equal_range(key3(ic[0] + dx, ic[1] + dy, ic[2] + dz));
            for (auto it = rg.first; it != rg.second; ++it) {
              const int f = it->second;
              double dmax = 0.0;
              for (int q = 0; q < 3; ++q) dmax = std::max(dmax, std::fabs(cen[3 * f + q] - c[q]));
              if (dmax < tol) { found = f; break; }
            }
          }
      if (found < 0) {
        found = F++;
        grid.emplace(key3(ic[0], ic[1], ic[2]), found);
        for (int q = 0; q < 3; ++q) cen.push_back(c[q]);
        first.push_back(e * 6 + fl);
        owner2.push_back(-1);
      } else {
        if (owner2[found] >= 0) return ctx_fail(ctx, MEHDG_ERR_ARG, "shell mesh: face with more than two owners");
        owner2[found] = e * 6 + fl;
      }
      fid[e * 6 + fl] = found;
    }
  }
  ctx->F = F;
  ctx->ntr = (long long)F * ns * Nfn;
  ctx->h_owner.assign(2 * F, -1);
  ctx->h_ofn.assign((size_t)2 * F * Nfn, 0);
  for (int f = 0; f < F; ++f) {
    ctx->h_owner[2 * f] = first[f];
    ctx->h_owner[2 * f + 1] = owner2[f];
    for (int jf = 0; jf < Nfn; ++jf) ctx->h_ofn[(size_t)2 * f * Nfn + jf] = jf;
    if (owner2[f] < 0) continue;
    // second owner: its local face node at the position of each face node of the first owner
    const int e0 = first[f] / 6, f0 = first[f] % 6, e1 = owner2[f] / 6, f1 = owner2[f] % 6;
    std::vector<char> used(Nfn, 0);
    for (int jf = 0; jf < Nfn; ++jf) {
      const int a0 = ctx->facenode[f0 * Nfn + jf];
      int best = -1;
      for (int l = 0; l < Nfn && best < 0; ++l) {
        const int a1 = ctx->facenode[f1 * Nfn + l];
        double dmax = 0.0;
        for (int q = 0; q < 3; ++q)
          dmax = std::max(dmax, std::fabs(xnode[((size_t)e0 * 3 + q) * Np + a0] - xnode[((size_t)e1 * 3 + q) * Np + a1]));
        if (dmax < tol) best = l;
      }
      if (best < 0 || used[best]) return ctx_fail(ctx, MEHDG_ERR_ARG, "shell mesh: face nodes of two owners do not match");
      used[best] = 1;
      ctx->h_ofn[((size_t)2 * f + 1) * Nfn + jf] = best;
    }
  }
  // gather maps (the macro's own face-node order) and boundary kinds
  for (int e = 0; e < E; ++e) {
    const int k = (e / (nq * nq)) % nr;
    for (int fl = 0; fl < 6; ++fl) {
      const int f = fid[e * 6 + fl];
      const int o = (ctx->h_owner[2 * f] == e * 6 + fl) ? 0 : 1;
      std::vector<int> loc2glob(Nfn);
      for (int jf = 0; jf < Nfn; ++jf) loc2glob[ctx->h_ofn[((size_t)2 * f + o) * Nfn + jf]] = jf;
      for (int s = 0; s < ns; ++s)
        for (int l = 0; l < Nfn; ++l)
          ctx->h_gather[(size_t)e * Nt + s * Nth + fl * Nfn + l] = (f * ns + s) * Nfn + loc2glob[l];
      int bs = -1;
      if (fl == 4 && k == 0) bs = 0;
      if (fl == 5 && k == nr - 1) bs = 1;
      if ((bs >= 0) != (ctx->h_owner[2 * f + 1] < 0))
        return ctx_fail(ctx, MEHDG_ERR_ARG, "shell mesh: boundary faces do not match the spheres");
      ctx->h_bside[e * 6 + fl] = bs;
      ctx->h_bkind[e * 6 + fl] = bs >= 0 ? pr.bc[bs] : 0;
    }
  }
  // the box numbering of the other maps is kept: owner slot o of face f is (e * 2d + fl)
  return MEHDG_OK;
}

// device: per-point geometry and per-macro operators of the shell (after the tables and
// node positions are on the device); dend: device [2][p+1]
int shell_geometry(mehdg_ctx* ctx, const double* dend) {
  switch (ctx->p) {
    case 1: return geometry_p<1>(ctx, dend);
    case 2: return geometry_p<2>(ctx, dend);
    case 3: return geometry_p<3>(ctx, dend);
  }
  return ctx_fail(ctx, MEHDG_ERR_ARG, "shell mesh: unsupported degree");
}

int shell_bdata(mehdg_ctx* ctx) {
  const int per_e = ctx->nsf * ctx->nfp;
  const long long npt = (long long)ctx->E * 6 * per_e;
  k_shell_bdata<3><<<(unsigned)((npt + 127) / 128), 128, 0, ctx->stream>>>(npt, per_e, ctx->prob, ctx->bkind,
                                                                          ctx->uD);
  CKL();
  return MEHDG_OK;
}

int shell_init_state(mehdg_ctx* ctx, const double* du, double* u) {
  const long long n = (long long)ctx->E * ctx->Np;
  k_shell_init<<<(unsigned)((n + 127) / 128), 128, 0, ctx->stream>>>(n, ctx->Np, ctx->prob, ctx->xnode, du, u);
  CKL();
  return MEHDG_OK;
}
