// a1-a2: residuals R_Q, R_U, R_Uhat (eq. C31221 from the weak form C38 / C242) and
// the Newton blocks of eq. C312 of every macro-element.
//
// Volume: one thread per (macro, sub-element, Gauss point, Jacobian input) runs the
// pointwise integrand (physics.cuh) in Dual<double,1> seeded on that input (a
// state component u_s or a gradient component q_{s,j}); nested inner duals inside
// the integrand give the flux Jacobian A_k and the strong-form divergence of the
// SUPG residual, so the outer derivative is exact.  The derivative with respect
// to the gradient of the input (d_l u_s, d_l q_{s,j}) enters only through the SUPG
// residual and equals tau A_k^T d(F+G)_l/d(input), assembled from the same pass.
// A second kernel contracts the pointwise kernels K[t,alpha;s,beta] with the
// tensor-product basis T[g][alpha][a] of each sub-element into the macro blocks.
// Faces: same structure with inputs (uhat, q, u) of the numerical flux and of B^.
#include <algorithm>

#include "internal.cuh"
#include "physics.cuh"

namespace {

template <int B, int E> struct IPow { static constexpr int v = B * IPow<B, E - 1>::v; };
template <int B> struct IPow<B, 0> { static constexpr int v = 1; };

template <class CT = double>
struct Tables {
  const CT* b1;   // [NG1][P1]
  const CT* db1;  // [NG1][P1] reference derivative
  const CT* gw;   // [NG1]
};
template <class CT>
__device__ __forceinline__ Tables<CT> tables(const CT* tab, int ng1, int p1) {
  Tables<CT> t;
  t.b1 = tab;
  t.db1 = tab + ng1 * p1;
  t.gw = tab + 2 * ng1 * p1;
  return t;
}

// ---------------------------------------------------------------- volume pointwise
// One thread per (macro, sub-element, Gauss point, input direction): interpolates
// u, grad u, q, grad q at the point, evaluates the volume integrand of eqs. C38a-b
// (with the SUPG term) on Dual numbers seeded along one input (u_s or q_js), and
// writes the Jacobian column K[X][t][s0][.] of the integrand, pre-weighted by the
// quadrature weight.  CT is the arithmetic type.  MODE 0 also writes the residual
// integrand (the FP64 path launches this mode as k_vol_point_sh, below, which shares the
// interpolation among the directions of a point); MODE 1 writes the Jacobian only (mixed path, CT = float:
// the Jacobian only shapes an inexact Newton step); MODE 2 writes the residual
// only, one thread per point, plain FP64 values (mixed path).
//
// MAPPED (curved macro-elements): vgeo holds per point (J^-1)[j][k] = dxi_j/dx_k, with xi the
// macro reference coordinates in [0, 1]^d (the tables' derivatives, scaled by 2/he with he =
// 1/m, are d/dxi), and the weight (reference weight times det J).  The interpolated gradients
// are mapped to physical ones, and the outputs are mapped back to d/dxi test and trial
// derivatives (K'[1+j] = sum_k J^-1[j][k] K[1+k] on both sides), so that the contraction
// kernels stay those of the reference element.
// Everything after the interpolation at one point for one input direction: the mapping of the
// interpolated gradients (curved macros), the pointwise integrand on dual numbers and the
// writes of the Jacobian columns and (MODE 0, direction 0; MODE 2) of the residual integrand.
template <int D, int P, class KT, class CT, int MODE, bool MAPPED>
__device__ __forceinline__ void vol_point_eval(const Geo& g, const Phys& ph, int e, int el, int gq, int dir, CT wq,
                                               CT (&U)[D + 2], CT (&GU)[D + 2][D], CT (&Q)[D + 2][D],
                                               CT (&GQ)[D + 2][D][D], const CT (&Hh)[D + 2], double coef,
                                               int supg_time, const CT* __restrict__ src, KT* __restrict__ Kvol,
                                               double* __restrict__ rvol, const double* __restrict__ vgeo,
                                               const int NG) {
  constexpr int NS = D + 2;
  constexpr int KA = (D + 1) * NS * (D + 1);
  const int nel = g.nel;
  CT Ji[D][D];
  if constexpr (MAPPED) {
    const double* vg = vgeo + (((size_t)e * nel + el) * NG + gq) * (D * D + 1);
    for (int j = 0; j < D; ++j)
      for (int k = 0; k < D; ++k) Ji[j][k] = (CT)vg[j * D + k];
    wq = (CT)vg[D * D];
    for (int s = 0; s < NS; ++s) {
      CT t[D];
      for (int k = 0; k < D; ++k) {
        t[k] = CT(0);
        for (int j = 0; j < D; ++j) t[k] += Ji[j][k] * GU[s][j];
      }
      for (int k = 0; k < D; ++k) GU[s][k] = t[k];
      for (int jq = 0; jq < D; ++jq) {
        for (int k = 0; k < D; ++k) {
          t[k] = CT(0);
          for (int j = 0; j < D; ++j) t[k] += Ji[j][k] * GQ[s][jq][j];
        }
        for (int k = 0; k < D; ++k) GQ[s][jq][k] = t[k];
      }
    }
  }
  CT f[NS];
  for (int s = 0; s < NS; ++s) f[s] = src ? src[(((size_t)e * nel + el) * NG + gq) * NS + s] : CT(0);

  if constexpr (MODE == 2) {
    // residual integrand only, plain values
    CT Ts[NS], W[NS], V[NS][D], FG[NS][D], A[D][NS][NS], tau;
    for (int s = 0; s < NS; ++s) Ts[s] = (CT)coef * U[s] + Hh[s];
    vol_integrand<D, CT, CT>(U, GU, Q, GQ, Ts, f, ph, supg_time, W, V, FG, A, tau);
    for (int t = 0; t < NS; ++t) {
      double* R = rvol + (((size_t)e * nel + el) * NG + gq) * NS * (D + 1) + t * (D + 1);
      R[0] = W[t] * wq;
      for (int k = 0; k < D; ++k) {
        CT vk = V[t][k];
        if constexpr (MAPPED) {
          vk = CT(0);
          for (int kk = 0; kk < D; ++kk) vk += Ji[k][kk] * V[t][kk];
        }
        R[1 + k] = vk * wq;
      }
    }
  } else {
    typedef Dual<CT, 1> S;
    const int X = dir / NS, s0 = dir % NS;
    S Us[NS], GUs[NS][D], Qs[NS][D], GQs[NS][D][D], Ts[NS];
    for (int s = 0; s < NS; ++s) {
      Us[s].v = U[s]; Us[s].d[0] = (X == 0 && s == s0) ? CT(1) : CT(0);
      for (int j = 0; j < D; ++j) {
        Qs[s][j].v = Q[s][j]; Qs[s][j].d[0] = (X == 1 + j && s == s0) ? CT(1) : CT(0);
        GUs[s][j].v = GU[s][j]; GUs[s][j].d[0] = CT(0);
        for (int l = 0; l < D; ++l) { GQs[s][j][l].v = GQ[s][j][l]; GQs[s][j][l].d[0] = CT(0); }
      }
      Ts[s] = coef * Us[s] + Hh[s];
    }
    S W[NS], V[NS][D], FG[NS][D], A[D][NS][NS], tau;
    vol_integrand<D, S, CT>(Us, GUs, Qs, GQs, Ts, f, ph, supg_time, W, V, FG, A, tau);

    if constexpr (MAPPED) {
      for (int t = 0; t < NS; ++t) {
        // physical block Kp[alpha][beta] (alpha: test value / d_k, beta: input value / d_l)
        CT Kp[D + 1][D + 1];
        Kp[0][0] = W[t].d[0];
        for (int l = 0; l < D; ++l) Kp[0][1 + l] = CT(0);
        for (int k = 0; k < D; ++k) {
          Kp[1 + k][0] = V[t][k].d[0];
          for (int l = 0; l < D; ++l) {
            CT val = CT(0);
            if (ph.supg) {
              for (int rr = 0; rr < NS; ++rr) val += A[k][rr][t].v * FG[rr][l].d[0];
              val *= tau.v;
            }
            Kp[1 + k][1 + l] = val;
          }
        }
        KT* K = Kvol + (((((size_t)e * (D + 1) + X) * NS + t) * nel + el) * NG + gq) * KA;
        K[(0 * NS + s0) * (D + 1) + 0] = (KT)(Kp[0][0] * wq);
        for (int j2 = 0; j2 < D; ++j2) K[(0 * NS + s0) * (D + 1) + 1 + j2] = (KT)0;
        for (int j = 0; j < D; ++j) {
          CT r0 = CT(0);
          for (int k = 0; k < D; ++k) r0 += Ji[j][k] * Kp[1 + k][0];
          K[((1 + j) * NS + s0) * (D + 1) + 0] = (KT)(r0 * wq);
          for (int j2 = 0; j2 < D; ++j2) {
            CT acc = CT(0);
            for (int k = 0; k < D; ++k)
              for (int l = 0; l < D; ++l) acc += Ji[j][k] * Kp[1 + k][1 + l] * Ji[j2][l];
            K[((1 + j) * NS + s0) * (D + 1) + 1 + j2] = (KT)(acc * wq);
          }
        }
        if (MODE == 0 && dir == 0) {
          double* R = rvol + (((size_t)e * nel + el) * NG + gq) * NS * (D + 1) + t * (D + 1);
          R[0] = W[t].v * wq;
          for (int j = 0; j < D; ++j) {
            CT acc = CT(0);
            for (int k = 0; k < D; ++k) acc += Ji[j][k] * V[t][k].v;
            R[1 + j] = acc * wq;
          }
        }
      }
      return;
    }
    for (int t = 0; t < NS; ++t) {
      KT* K = Kvol + (((((size_t)e * (D + 1) + X) * NS + t) * nel + el) * NG + gq) * KA;
      K[(0 * NS + s0) * (D + 1) + 0] = (KT)(W[t].d[0] * wq);
      for (int l = 0; l < D; ++l) K[(0 * NS + s0) * (D + 1) + 1 + l] = (KT)0;
      for (int k = 0; k < D; ++k) {
        K[((1 + k) * NS + s0) * (D + 1) + 0] = (KT)(V[t][k].d[0] * wq);
        for (int l = 0; l < D; ++l) {
          CT val = CT(0);
          if (ph.supg) {
            for (int rr = 0; rr < NS; ++rr) val += A[k][rr][t].v * FG[rr][l].d[0];
            val *= tau.v;
          }
          K[((1 + k) * NS + s0) * (D + 1) + 1 + l] = (KT)(val * wq);
        }
      }
      if (MODE == 0 && dir == 0) {
        double* R = rvol + (((size_t)e * nel + el) * NG + gq) * NS * (D + 1) + t * (D + 1);
        R[0] = W[t].v * wq;
        for (int k = 0; k < D; ++k) R[1 + k] = V[t][k].v * wq;
      }
    }
  }
}

template <int D, int P, class KT, class CT = double, int MODE = 0, bool MAPPED = false>
__global__ void __launch_bounds__(128) k_vol_point(Geo g, const CT* __restrict__ tab, Phys ph,
                                                    const CT* __restrict__ u, const CT* __restrict__ q,
                                                    const CT* __restrict__ hist, double coef, int supg_time,
                                                    const CT* __restrict__ src, KT* __restrict__ Kvol,
                                                    double* __restrict__ rvol, int E,
                                                    const double* __restrict__ vgeo = nullptr) {
  constexpr int NS = D + 2, P1 = P + 1, NG1 = P + 2;
  constexpr int NLOC = IPow<P1, D>::v, NG = IPow<NG1, D>::v;
  constexpr int NDIR = (MODE == 2) ? 1 : NS * (1 + D);
  constexpr int KA = (D + 1) * NS * (D + 1);
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nel = g.nel;
  if (tid >= (long long)E * nel * NG * NDIR) return;
  const int dir = tid % NDIR;
  long long r = tid / NDIR;
  const int gq = r % NG;
  r /= NG;
  const int el = r % nel;
  const int e = (int)(r / nel);
  Tables<CT> tb = tables(tab, NG1, P1);

  int gi[D], li[D];
  CT wq = CT(1), he[D];
  {
    int gg = gq, ll = el;
    for (int k = 0; k < D; ++k) {
      gi[k] = gg % NG1; gg /= NG1;
      li[k] = ll % g.m; ll /= g.m;
      he[k] = (CT)g.he[k];
      wq *= tb.gw[gi[k]] * CT(0.5) * he[k];
    }
  }
  CT U[NS], GU[NS][D], Q[NS][D], GQ[NS][D][D], Hh[NS];
  for (int s = 0; s < NS; ++s) {
    U[s] = CT(0); Hh[s] = CT(0);
    for (int l = 0; l < D; ++l) {
      GU[s][l] = CT(0);
      for (int j = 0; j < D; ++j) { GQ[s][j][l] = CT(0); }
      Q[s][l] = CT(0);
    }
  }
  const size_t Np = g.Np;
  for (int al = 0; al < NLOC; ++al) {
    int ai[D], a = 0, aa = al, stride = 1;
    for (int k = 0; k < D; ++k) {
      ai[k] = aa % P1; aa /= P1;
      a += (li[k] * P + ai[k]) * stride;
      stride *= g.n1;
    }
    CT bv[D], dv[D];
    for (int k = 0; k < D; ++k) {
      bv[k] = tb.b1[gi[k] * P1 + ai[k]];
      dv[k] = tb.db1[gi[k] * P1 + ai[k]] * CT(2) / he[k];
    }
    CT phi = CT(1), dphi[D];
    for (int k = 0; k < D; ++k) phi *= bv[k];
    for (int l = 0; l < D; ++l) {
      dphi[l] = dv[l];
      for (int k = 0; k < D; ++k)
        if (k != l) dphi[l] *= bv[k];
    }
    for (int s = 0; s < NS; ++s) {
      CT ua = u[((size_t)e * NS + s) * Np + a];
      U[s] += phi * ua;
      for (int l = 0; l < D; ++l) GU[s][l] += dphi[l] * ua;
      if (hist) Hh[s] += phi * hist[((size_t)e * NS + s) * Np + a];
      for (int j = 0; j < D; ++j) {
        CT qa = q[(((size_t)e * D + j) * NS + s) * Np + a];
        Q[s][j] += phi * qa;
        for (int l = 0; l < D; ++l) GQ[s][j][l] += dphi[l] * qa;
      }
    }
  }
  vol_point_eval<D, P, KT, CT, MODE, MAPPED>(g, ph, e, el, gq, dir, wq, U, GU, Q, GQ, Hh, coef, supg_time, src,
                                             Kvol, rvol, vgeo, NG);
}

// The FP64 Jacobian pass with the interpolation shared by the input directions of a point: one
// CTA takes VpCfg::PPB points with all NDIR directions of each.  The basis values and physical
// derivatives of the points' sub-element nodes (phase 0), then u, grad u, q, grad q and the
// history at each point (phase 1), are formed once in shared memory, with the operations of
// k_vol_point in the same order; each thread then runs the pointwise physics
// of one direction (phase 2).  k_vol_point repeats the interpolation in all NDIR threads of a
// point.
template <int D> struct VpCfg {
  static constexpr int NS = D + 2;
  static constexpr int NDIR = NS * (1 + D);
  static constexpr int PPB = 240 / NDIR;                 // D = 3: 12 points, D = 2: 20 points
  static constexpr int NT = PPB * NDIR;                  // 240 threads
  static constexpr int NV = NS * (2 + 2 * D + D * D);    // U, GU, Q, GQ, Hh of a point
  // offsets in a point's row of values
  static constexpr int OGU = NS, OQ = NS * (1 + D), OGQ = NS * (1 + 2 * D), OH = NS * (1 + 2 * D + D * D);
};

template <int D, int P, class KT, bool MAPPED>
__global__ void __launch_bounds__(VpCfg<D>::NT) k_vol_point_sh(Geo g, const double* __restrict__ tab, Phys ph,
                                                             const double* __restrict__ u,
                                                             const double* __restrict__ q,
                                                             const double* __restrict__ hist, double coef,
                                                             int supg_time, const double* __restrict__ src,
                                                             KT* __restrict__ Kvol, double* __restrict__ rvol,
                                                             int E, const double* __restrict__ vgeo) {
  typedef VpCfg<D> C;
  constexpr int NS = D + 2, P1 = P + 1, NG1 = P + 2;
  constexpr int NLOC = IPow<P1, D>::v, NG = IPow<NG1, D>::v;
  constexpr int NDIR = C::NDIR, PPB = C::PPB, NGRP = D + 2;
  __shared__ double sphi[PPB][NLOC][D + 1];   // phi and d phi / d x_l of each node of the point's sub-element
  __shared__ int snode[PPB][NLOC];            // its macro node
  __shared__ double sv[PPB][C::NV];
  const int nel = g.nel;
  const size_t Np = g.Np;
  const long long npts = (long long)E * nel * NG;
  const long long p0 = (long long)blockIdx.x * PPB;
  Tables<double> tb = tables(tab, NG1, P1);
  for (int i = threadIdx.x; i < PPB * NLOC; i += blockDim.x) {
    const int pl = i / NLOC, al = i % NLOC;
    const long long pt = p0 + pl;
    if (pt >= npts) continue;
    const int gq = (int)(pt % NG);
    const int el = (int)((pt / NG) % nel);
    int gi[D], li[D];
    double he[D];
    {
      int gg = gq, ll = el;
      for (int k = 0; k < D; ++k) {
        gi[k] = gg % NG1; gg /= NG1;
        li[k] = ll % g.m; ll /= g.m;
        he[k] = g.he[k];
      }
    }
    int a = 0, aa = al, stride = 1;
    double bv[D], dv[D];
    for (int k = 0; k < D; ++k) {
      const int ak = aa % P1;
      aa /= P1;
      a += (li[k] * P + ak) * stride;
      stride *= g.n1;
      bv[k] = tb.b1[gi[k] * P1 + ak];
      dv[k] = tb.db1[gi[k] * P1 + ak] * 2.0 / he[k];
    }
    double phi = 1.0, dphi[D];
    for (int k = 0; k < D; ++k) phi *= bv[k];
    for (int l = 0; l < D; ++l) {
      dphi[l] = dv[l];
      for (int k = 0; k < D; ++k)
        if (k != l) dphi[l] *= bv[k];
    }
    sphi[pl][al][0] = phi;
    for (int l = 0; l < D; ++l) sphi[pl][al][1 + l] = dphi[l];
    snode[pl][al] = a;
  }
  __syncthreads();
  // one task per (point, species, group): group 0 u (U, GU), 1 + j q_j (Q_j, GQ_j), D + 1 history
  for (int i = threadIdx.x; i < PPB * NS * NGRP; i += blockDim.x) {
    const int pl = i / (NS * NGRP), rr = i % (NS * NGRP);
    const int sp = rr / NGRP, grp = rr % NGRP;
    const long long pt = p0 + pl;
    if (pt >= npts) continue;
    const int e = (int)(pt / ((long long)nel * NG));
    double* out = sv[pl];
    if (grp == D + 1) {
      double h = 0.0;
      if (hist) {
        const double* hs = hist + ((size_t)e * NS + sp) * Np;
        for (int al = 0; al < NLOC; ++al) h += sphi[pl][al][0] * hs[snode[pl][al]];
      }
      out[C::OH + sp] = h;
    } else {
      const double* xs = grp == 0 ? u + ((size_t)e * NS + sp) * Np
                                  : q + (((size_t)e * D + (grp - 1)) * NS + sp) * Np;
      double v = 0.0, gv[D];
      for (int l = 0; l < D; ++l) gv[l] = 0.0;
      for (int al = 0; al < NLOC; ++al) {
        const double x = xs[snode[pl][al]];
        v += sphi[pl][al][0] * x;
        for (int l = 0; l < D; ++l) gv[l] += sphi[pl][al][1 + l] * x;
      }
      if (grp == 0) {
        out[sp] = v;
        for (int l = 0; l < D; ++l) out[C::OGU + sp * D + l] = gv[l];
      } else {
        const int j = grp - 1;
        out[C::OQ + sp * D + j] = v;
        for (int l = 0; l < D; ++l) out[C::OGQ + (sp * D + j) * D + l] = gv[l];
      }
    }
  }
  __syncthreads();
  const int pl = threadIdx.x / NDIR, dir = threadIdx.x % NDIR;
  const long long pt = p0 + pl;
  if (pl >= PPB || pt >= npts) return;
  const int gq = (int)(pt % NG);
  const int el = (int)((pt / NG) % nel);
  const int e = (int)(pt / ((long long)nel * NG));
  double wq = 1.0;
  {
    int gg = gq;
    for (int k = 0; k < D; ++k) {
      const int gk = gg % NG1;
      gg /= NG1;
      wq *= tb.gw[gk] * 0.5 * g.he[k];
    }
  }
  double U[NS], GU[NS][D], Q[NS][D], GQ[NS][D][D], Hh[NS];
  const double* in = sv[pl];
  for (int s2 = 0; s2 < NS; ++s2) {
    U[s2] = in[s2];
    Hh[s2] = in[C::OH + s2];
    for (int j = 0; j < D; ++j) {
      GU[s2][j] = in[C::OGU + s2 * D + j];
      Q[s2][j] = in[C::OQ + s2 * D + j];
      for (int l = 0; l < D; ++l) GQ[s2][j][l] = in[C::OGQ + (s2 * D + j) * D + l];
    }
  }
  vol_point_eval<D, P, KT, double, 0, MAPPED>(g, ph, e, el, gq, dir, wq, U, GU, Q, GQ, Hh, coef, supg_time, src,
                                              Kvol, rvol, vgeo, NG);
}

// basis value T[g][alpha][a] of a sub-element from 1D tables (alpha 0: value, 1+k: d/dx_k)
template <int D, int P, class CT = double>
__device__ __forceinline__ CT basis_T(const CT* sb, const CT* sdb, const CT* sc, const int* gi, const int* ai,
                                      int alpha) {
  constexpr int P1 = P + 1;
  CT v = CT(1);
#pragma unroll
  for (int k = 0; k < D; ++k)
    v *= (alpha == 1 + k) ? sdb[gi[k] * P1 + ai[k]] * sc[k] : sb[gi[k] * P1 + ai[k]];
  return v;
}

template <int D, int P, class CT = double> struct VolCfg {
  static constexpr int NS = D + 2, P1 = P + 1, NG1 = P + 2;
  static constexpr int NLOC = IPow<P1, D>::v, NG = IPow<NG1, D>::v;
  static constexpr int KA = (D + 1) * NS * (D + 1);
  static constexpr int NCOL = NS * NLOC;                  // output columns (s, b)
  static constexpr int ZG = (D + 1) * NCOL;               // Z entries per Gauss point
  static constexpr int GC = (ZG * 8 <= 1536) ? 32 : (ZG <= 600 ? 16 : 8);
  static constexpr int RPT0 = (NLOC + 3) / 4 * 4;
  static constexpr int RPT = RPT0 > 16 ? 16 : RPT0;       // output rows per thread (multiple of 4)
  static constexpr int RG = (NLOC + RPT - 1) / RPT;       // row groups
  static constexpr int NLOCP = RG * RPT;                  // padded basis count (row stride of T)
  static constexpr int TG = (D + 1) * NLOCP;              // basis entries per Gauss point
  static constexpr int ITEMS = NCOL * RG;                 // (column, row group) items
  static constexpr int NT0 = (ITEMS + 31) / 32 * 32;
  static constexpr int NT = NT0 > 512 ? 512 : NT0;
  static constexpr int OPT = (ITEMS + NT - 1) / NT;
  // basis table T for all Gauss points of a sub-element when it fits (it is the same
  // for every sub-element of every macro), else one chunk at a time
  static constexpr bool TFULL = (size_t)NG * TG * sizeof(CT) <= 48 * 1024;
  static constexpr int TROWS = TFULL ? NG : GC;
  static constexpr size_t SMEM =
      sizeof(CT) * ((size_t)GC * KA + (size_t)GC * ZG + (size_t)TROWS * TG + 2 * (size_t)NG1 * P1 + 4);
};

// A_X[(t, A)][(s, B)] += sum_g sum_{alpha,beta} T[g][alpha][a] K[g][alpha][s][beta] T[g][beta][b]
// per sub-element: with Z[g][alpha][(s, b)] = sum_beta K[g][alpha][s][beta] T[g][beta][b],
// the output block is the product T^T Z over the (g, alpha) index.  Per chunk of Gauss
// points the basis values T (rows padded to a multiple of 4) and Z are tabulated in
// shared memory; each thread owns one output column (s, b) and RPT rows a, so a step of
// the product costs one Z load, RPT/4 broadcast 16-byte T loads (FP32) and RPT FMAs.
template <int D, int P, class CT>
__global__ void __launch_bounds__(VolCfg<D, P, CT>::NT) k_vol_contract(Geo g, const double* __restrict__ tab,
                                                                      const CT* __restrict__ Kvol,
                                                                      CT* __restrict__ Auu, CT* __restrict__ Auq) {
  typedef VolCfg<D, P, CT> C;
  constexpr int NS = C::NS, P1 = C::P1, NG1 = C::NG1, NLOC = C::NLOC, NG = C::NG, KA = C::KA, ZG = C::ZG;
  constexpr int TG = C::TG, NCOL = C::NCOL, GC = C::GC, NT = C::NT, OPT = C::OPT, RPT = C::RPT;
  constexpr int NLOCP = C::NLOCP;
  constexpr int ITEMS = C::ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool TFULL = C::TFULL;
  CT* sT = reinterpret_cast<CT*>(smem_raw);   // [TROWS][D+1][NLOCP]
  CT* sK = sT + C::TROWS * TG;                // [GC][KA]
  CT* sZ = sK + GC * KA;                      // [GC][D+1][NCOL]
  CT* sb = sZ + GC * ZG;                      // 1D basis values [NG1][P1] in CT
  CT* sdb = sb + NG1 * P1;                    // 1D reference derivatives
  const int e = blockIdx.x, X = blockIdx.y, t = blockIdx.z;
  const int tid = threadIdx.x;
  CT sc[D];
  for (int k = 0; k < D; ++k) sc[k] = (CT)(2.0 / g.he[k]);
  for (int i = tid; i < NG1 * P1; i += NT) {
    sb[i] = (CT)tab[i];
    sdb[i] = (CT)tab[NG1 * P1 + i];
  }
  __syncthreads();
  // T[g][alpha][a] for points g0 .. g0 + ng - 1 into sT rows 0 .. ng - 1: value (alpha 0)
  // or derivative along x_{alpha-1} of basis a at point g (rows padded with zeros)
  auto tabulate_T = [&](int g0, int ng) {
    for (int i = tid; i < ng * TG; i += NT) {
      const int a = i % NLOCP, al = (i / NLOCP) % (D + 1), gg = i / TG;
      CT v = CT(0);
      if (a < NLOC) {
        int t1 = g0 + gg, t2 = a;
        v = CT(1);
        for (int k = 0; k < D; ++k) {
          const int gk = t1 % NG1, ak = t2 % P1;
          t1 /= NG1; t2 /= P1;
          v *= (al == 1 + k) ? sdb[gk * P1 + ak] * sc[k] : sb[gk * P1 + ak];
        }
      }
      sT[i] = v;
    }
  };
  if constexpr (TFULL) {
    tabulate_T(0, NG);
    __syncthreads();
  }
  const size_t Nu = g.Nu, Np = g.Np;
  CT* out = (X == 0) ? Auu + (size_t)e * Nu * Nu : Auq + ((size_t)e * D + X - 1) * Nu * Nu;
  int icol[OPT], irow[OPT];
  for (int o = 0; o < OPT; ++o) {
    int w = tid + o * NT;
    if (w >= ITEMS) w = ITEMS - 1;
    icol[o] = w % NCOL;
    irow[o] = (w / NCOL) * RPT;
  }
  for (int el = 0; el < g.nel; ++el) {
    int li[D];
    {
      int ll = el;
      for (int k = 0; k < D; ++k) { li[k] = ll % g.m; ll /= g.m; }
    }
    CT acc[OPT][RPT];
#pragma unroll
    for (int o = 0; o < OPT; ++o)
#pragma unroll
      for (int r = 0; r < RPT; ++r) acc[o][r] = CT(0);
    const CT* Kel = Kvol + ((((size_t)e * (D + 1) + X) * NS + t) * g.nel + el) * (size_t)NG * KA;
    for (int g0 = 0; g0 < NG; g0 += GC) {
      const int gc = min(GC, NG - g0);
      for (int i = tid; i < gc * KA; i += NT) sK[i] = Kel[(size_t)g0 * KA + i];
      if constexpr (!TFULL) tabulate_T(g0, gc);
      const CT* sTc = TFULL ? sT + (size_t)g0 * TG : sT;   // T rows of this chunk
      __syncthreads();
      for (int i = tid; i < gc * ZG; i += NT) {
        const int col = i % NCOL, al = (i / NCOL) % (D + 1), gg = i / ZG;
        const int s = col / NLOC, b = col % NLOC;
        const CT* Kp = sK + gg * KA + (al * NS + s) * (D + 1);
        const CT* Tp = sTc + gg * TG + b;
        CT z = CT(0);
#pragma unroll
        for (int be = 0; be <= D; ++be) z += Kp[be] * Tp[be * NLOCP];
        sZ[i] = z;
      }
      __syncthreads();
#pragma unroll
      for (int o = 0; o < OPT; ++o) {
        for (int k = 0; k < gc * (D + 1); ++k) {
          const CT z = sZ[k * NCOL + icol[o]];
          const CT* Tk = sTc + k * NLOCP + irow[o];
          if constexpr (sizeof(CT) == 4) {
#pragma unroll
            for (int r = 0; r < RPT; r += 4) {
              const float4 tv = *reinterpret_cast<const float4*>(Tk + r);
              acc[o][r] += tv.x * z;
              acc[o][r + 1] += tv.y * z;
              acc[o][r + 2] += tv.z * z;
              acc[o][r + 3] += tv.w * z;
            }
          } else {
#pragma unroll
            for (int r = 0; r < RPT; ++r) acc[o][r] += Tk[r] * z;
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
      if (tid + o * NT >= ITEMS) break;
      const int s = icol[o] / NLOC, b = icol[o] % NLOC;
      int B = 0, sa = 1, t2 = b;
      for (int k = 0; k < D; ++k) {
        B += (li[k] * P + t2 % P1) * sa;
        t2 /= P1; sa *= g.n1;
      }
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int a = irow[o] + r;
        if (a >= NLOC) break;
        int A = 0, sb = 1, t1 = a;
        for (int k = 0; k < D; ++k) {
          A += (li[k] * P + t1 % P1) * sb;
          t1 /= P1; sb *= g.n1;
        }
        out[((size_t)t * Np + A) * Nu + (size_t)s * Np + B] += acc[o][r];
      }
    }
    __syncthreads();
  }
}

// The same blocks by sum factorisation (used on the FP64 path, where the FP64 pipe is the
// bound).  On a sub-element both the basis T[g][alpha][a] and the Gauss points are tensor
// products: T is a product over the axes of 1D values v(g_k, a_k) or, on axis alpha-1, of
// the scaled 1D derivative d(g_k, a_k).  The bilinear sum
//   A[a][b] = sum_{alpha,beta} sum_g T[g][alpha][a] K[g][alpha,s,beta] T[g][beta][b]
// is contracted one axis at a time.  After the x axis the pairs (alpha, beta) whose
// remaining factors agree are added (alpha = 0 and alpha = 1 both carry values on y and
// z), and likewise after y, so the three passes run on 3 x 3, 2 x 2 and 2 x 2 classes
// instead of 13 pairs (3D).  Per (sub-element, trial species) that is
// 16 ((p+1)^2 (p+2)^2 + ...) multiply-adds instead of (p+1)^6 (p+2)^3 (d+1).
// One CTA per (macro, input X, test species t) runs every sub-element and trial species.
template <int D, int P, class CT>
struct SfCfg {
  static constexpr int NS = D + 2, P1 = P + 1, NG1 = P + 2;
  static constexpr int NLOC = IPow<P1, D>::v, NG = IPow<NG1, D>::v;
  static constexpr int KA = (D + 1) * NS * (D + 1);
  static constexpr int KAP = KA | 1;                                   // odd row stride: no bank repeats
  static constexpr int NC1 = D;                                        // classes after the x pass
  static constexpr int W1N = NC1 * NC1 * IPow<NG1, D - 1>::v * P1 * P1;
  static constexpr int W2N = D == 3 ? 2 * 2 * NG1 * P1 * P1 * P1 * P1 : 1;
  static constexpr int PT = 4 * NG1 * P1 * P1;                         // product table of one axis
  static constexpr int NT = 256;
  static constexpr size_t SMEM = sizeof(CT) * ((size_t)NG * KAP + W1N + W2N + D * PT);
};

// class of a test/trial index alpha (0 value, 1 + k derivative along k) once the first
// `done` axes are contracted: 0 when its remaining factors are all values, else alpha - done
__device__ __forceinline__ int sf_class(int alpha, int done) { return (alpha == 0 || alpha <= done) ? 0 : alpha - done; }

template <int D, int P, class CT>
__global__ void __launch_bounds__(256) k_vol_contract_sf(Geo g, const double* __restrict__ tab,
                                                         const CT* __restrict__ Kvol, CT* __restrict__ Auu,
                                                         CT* __restrict__ Auq) {
  typedef SfCfg<D, P, CT> C;
  constexpr int NS = C::NS, P1 = C::P1, NG1 = C::NG1, NLOC = C::NLOC, NG = C::NG, KA = C::KA, KAP = C::KAP;
  constexpr int NT = C::NT, PT = C::PT;
  extern __shared__ __align__(16) unsigned char sf_raw[];
  CT* sK = reinterpret_cast<CT*>(sf_raw);   // [NG][KAP] pointwise kernels of one sub-element
  CT* W1 = sK + NG * KAP;                   // after the x pass
  CT* W2 = W1 + C::W1N;                     // after the y pass (3D)
  // per axis k: products pt[k][ta][tb][g][a][b] = f_ta(g, a) f_tb(g, b), f_0 = 1D value,
  // f_1 = 1D derivative along k (scaled to the sub-element), so each term is one FMA
  CT* pt = W2 + C::W2N;
  const int e = blockIdx.x, X = blockIdx.y, t = blockIdx.z, tid = threadIdx.x;
  for (int i = tid; i < D * PT; i += NT) {
    const int b = i % P1, a = (i / P1) % P1, gq = (i / (P1 * P1)) % NG1, tb = (i / (P1 * P1 * NG1)) % 2;
    const int ta = (i / (P1 * P1 * NG1 * 2)) % 2, k = i / PT;
    const double sc = 2.0 / g.he[k];
    const double fa = ta ? tab[NG1 * P1 + gq * P1 + a] * sc : tab[gq * P1 + a];
    const double fb = tb ? tab[NG1 * P1 + gq * P1 + b] * sc : tab[gq * P1 + b];
    pt[i] = (CT)(fa * fb);
  }
  const size_t Nu = g.Nu, Np = g.Np;
  CT* out = (X == 0) ? Auu + (size_t)e * Nu * Nu : Auq + ((size_t)e * D + X - 1) * Nu * Nu;
  for (int el = 0; el < g.nel; ++el) {
    int li[D];
    {
      int ll = el;
      for (int k = 0; k < D; ++k) { li[k] = ll % g.m; ll /= g.m; }
    }
    __syncthreads();   // previous sub-element's readers of sK are done
    const CT* Kel = Kvol + ((((size_t)e * (D + 1) + X) * NS + t) * g.nel + el) * (size_t)NG * KA;
    for (int i = tid; i < NG * KA; i += NT) sK[(i / KA) * KAP + i % KA] = Kel[i];
    __syncthreads();
    for (int s = 0; s < NS; ++s) {
      // x pass: W1[ca][cb][g_rest][ax][bx], classes after one axis
      constexpr int GR = IPow<NG1, D - 1>::v;
      for (int i = tid; i < C::W1N; i += NT) {
        const int bx = i % P1, ax = (i / P1) % P1, gr = (i / (P1 * P1)) % GR;
        const int cb = (i / (P1 * P1 * GR)) % D, ca = i / (P1 * P1 * GR * D);
        CT acc = CT(0);
        for (int al = 0; al <= D; ++al) {
          if (sf_class(al, 1) != ca) continue;
          for (int be = 0; be <= D; ++be) {
            if (sf_class(be, 1) != cb || (al == 0 && be != 0)) continue;
            const CT* pp = pt + (((al == 1) * 2 + (be == 1)) * NG1) * P1 * P1 + ax * P1 + bx;
            const CT* kk = sK + (size_t)gr * NG1 * KAP + (al * NS + s) * (D + 1) + be;
#pragma unroll
            for (int gx = 0; gx < NG1; ++gx) acc += pp[gx * P1 * P1] * kk[gx * KAP];
          }
        }
        W1[i] = acc;
      }
      __syncthreads();
      const CT* last;   // the pass before the final one: [classes z][classes z][NG1 gz][rest...]
      if constexpr (D == 3) {
        // y pass: W2[za][zb][gz][ay][ax][by][bx]
        for (int i = tid; i < C::W2N; i += NT) {
          const int bx = i % P1, by = (i / P1) % P1, ax = (i / (P1 * P1)) % P1, ay = (i / (P1 * P1 * P1)) % P1;
          const int gz = (i / (P1 * P1 * P1 * P1)) % NG1, zb = (i / (P1 * P1 * P1 * P1 * NG1)) % 2;
          const int za = i / (P1 * P1 * P1 * P1 * NG1 * 2);
          CT acc = CT(0);
          for (int ca = 0; ca < 3; ++ca) {
            if ((ca == 2) != (za == 1)) continue;
            for (int cb = 0; cb < 3; ++cb) {
              if ((cb == 2) != (zb == 1)) continue;
              const CT* pp = pt + PT + (((ca == 1) * 2 + (cb == 1)) * NG1) * P1 * P1 + ay * P1 + by;
              const CT* ww = W1 + ((((ca * 3 + cb) * NG1 + gz) * NG1) * P1 + ax) * P1 + bx;
#pragma unroll
              for (int gy = 0; gy < NG1; ++gy) acc += pp[gy * P1 * P1] * ww[gy * P1 * P1];
            }
          }
          W2[i] = acc;
        }
        __syncthreads();
        last = W2;
      } else {
        last = W1;
      }
      // final pass (z in 3D, y in 2D) and the scatter into the macro block
      const CT* ptl = pt + (D - 1) * PT;
      for (int i = tid; i < NLOC * NLOC; i += NT) {
        const int a = i / NLOC, b = i % NLOC;
        int av[D], bv[D];
        {
          int aa = a, bb = b;
          for (int k = 0; k < D; ++k) { av[k] = aa % P1; aa /= P1; bv[k] = bb % P1; bb /= P1; }
        }
        CT acc = CT(0);
        for (int za = 0; za < 2; ++za)
          for (int zb = 0; zb < 2; ++zb) {
            const CT* pp = ptl + ((za * 2 + zb) * NG1) * P1 * P1 + av[D - 1] * P1 + bv[D - 1];
            const CT* ww;
            if constexpr (D == 3)
              ww = last + ((((za * 2 + zb) * NG1) * P1 + av[1]) * P1 + av[0]) * P1 * P1 + bv[1] * P1 + bv[0];
            else
              ww = last + (((za * 2 + zb) * NG1) * P1 + av[0]) * P1 + bv[0];
            constexpr int WS = D == 3 ? P1 * P1 * P1 * P1 : P1 * P1;   // stride of the last axis' point
#pragma unroll
            for (int gl = 0; gl < NG1; ++gl) acc += pp[gl * P1 * P1] * ww[gl * WS];
          }
        int A = 0, B = 0, sa = 1;
        for (int k = 0; k < D; ++k) {
          A += (li[k] * P + av[k]) * sa;
          B += (li[k] * P + bv[k]) * sa;
          sa *= g.n1;
        }
        out[((size_t)t * Np + A) * Nu + (size_t)s * Np + B] += acc;
      }
      __syncthreads();   // W1/W2 are rewritten for the next trial species
    }
  }
}

// R_U[t][A] += sum_g sum_alpha T[g][alpha][a] r[g][t][alpha]
template <int D, int P>
__global__ void k_vol_res(Geo g, const double* __restrict__ tab, const double* __restrict__ rvol,
                          double* __restrict__ RU) {
  constexpr int NS = D + 2, P1 = P + 1, NG1 = P + 2;
  constexpr int NLOC = IPow<P1, D>::v, NG = IPow<NG1, D>::v;
  __shared__ double sb[NG1 * P1], sdb[NG1 * P1];
  const int e = blockIdx.x;
  for (int i = threadIdx.x; i < NG1 * P1; i += blockDim.x) {
    sb[i] = tab[i];
    sdb[i] = tab[NG1 * P1 + i];
  }
  double sc[D];
  for (int k = 0; k < D; ++k) sc[k] = 2.0 / g.he[k];
  __syncthreads();
  for (int el = 0; el < g.nel; ++el) {
    int li[D];
    int ll = el;
    for (int k = 0; k < D; ++k) { li[k] = ll % g.m; ll /= g.m; }
    for (int oi = threadIdx.x; oi < NS * NLOC; oi += blockDim.x) {
      int t = oi / NLOC, al = oi % NLOC;
      int ai[D], A = 0, sa = 1, t2 = al;
      for (int k = 0; k < D; ++k) {
        ai[k] = t2 % P1; t2 /= P1;
        A += (li[k] * P + ai[k]) * sa;
        sa *= g.n1;
      }
      const double* R = rvol + ((size_t)e * g.nel + el) * NG * NS * (D + 1);
      double sum = 0.0;
      for (int gq = 0; gq < NG; ++gq) {
        int gi[D], t1 = gq;
        for (int k = 0; k < D; ++k) { gi[k] = t1 % NG1; t1 /= NG1; }
        for (int alpha = 0; alpha <= D; ++alpha)
          sum += basis_T<D, P>(sb, sdb, sc, gi, ai, alpha) * R[((size_t)gq * NS + t) * (D + 1) + alpha];
      }
      RU[((size_t)e * NS + t) * g.Np + A] += sum;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- faces
// tangential decomposition of a sub-face, sub-face node and face point
template <int D>
__device__ __forceinline__ void face_axes(int fl, int* tang) {
  int k = fl / 2, c = 0;
  for (int kk = 0; kk < D; ++kk)
    if (kk != k) tang[c++] = kk;
}

// One thread per (macro, face, sub-face, face Gauss point, input direction): the
// trace flux of eq. C38c (or the boundary operator B^) and the numerical flux tested
// against the volume space, differentiated along one input (u^_s, q_js or u_s).
// MODE 0: Jacobian and residual (FP64 path); MODE 1: Jacobian only, CT = float, from
// FP32 copies of the state (mixed path); MODE 2: residual only, one thread per point.
// The numerical flux and the trace equation (interior flux, or B^ of the face's boundary kind
// bk with side bs and data ud) at one face point with unit normal n and weight wf, for one input
// direction (uhat_s, q_sj, u_s): writes the Jacobian column (and, MODE 0 direction 0 or MODE 2,
// the residual integrands) of face point pidx.
template <int D, class CT, int MODE>
__device__ __forceinline__ void face_point_eval(const Phys& ph, const mehdg_problem& pr, int bk, int bs,
                                                const CT* __restrict__ ud, const double* n, CT wf,
                                                const CT (&Uf)[D + 2], const CT (&Qf)[D + 2][D],
                                                const CT (&UHf)[D + 2], int dir, size_t pidx,
                                                CT* __restrict__ Kface, double* __restrict__ rface) {
  constexpr int NS = D + 2;
  constexpr int NDIR_K = NS * (D + 2);
  if constexpr (MODE == 2) {
    CT fh[NS], eq[NS];
    trace_flux<D, CT>(UHf, Qf, Uf, n, ph, fh);
    if (bk == MEHDG_BC_DIRICHLET) {
      for (int s = 0; s < NS; ++s) eq[s] = UHf[s] - ud[s];
    } else if (bk == MEHDG_BC_WALL) {
      wall_operator<D, CT>(UHf, Uf, pr.wall_T[bs], pr.wall_v[bs], pr.gamma, eq);
    } else if (bk == MEHDG_BC_FARFIELD) {
      farfield_operator<D, CT, CT>(UHf, Uf, ud, n, pr.gamma, eq);
    } else {
      for (int s = 0; s < NS; ++s) eq[s] = fh[s];
    }
    double* R = rface + pidx * 2 * NS;
    for (int t = 0; t < NS; ++t) {
      R[t] = fh[t] * wf;
      R[NS + t] = eq[t] * wf;
    }
  } else {
    typedef Dual<CT, 1> S;
    S Us[NS], Qs[NS][D], UHs[NS], fh[NS], eq[NS];
    for (int s = 0; s < NS; ++s) {
      UHs[s].v = UHf[s]; UHs[s].d[0] = (dir == s) ? CT(1) : CT(0);
      for (int j = 0; j < D; ++j) {
        Qs[s][j].v = Qf[s][j];
        Qs[s][j].d[0] = (dir == NS + j * NS + s) ? CT(1) : CT(0);
      }
      Us[s].v = Uf[s]; Us[s].d[0] = (dir == NS + NS * D + s) ? CT(1) : CT(0);
    }
    trace_flux<D, S>(UHs, Qs, Us, n, ph, fh);
    if (bk == MEHDG_BC_DIRICHLET) {
      for (int s = 0; s < NS; ++s) eq[s] = UHs[s] - (double)ud[s];
    } else if (bk == MEHDG_BC_WALL) {
      wall_operator<D, S>(UHs, Us, pr.wall_T[bs], pr.wall_v[bs], pr.gamma, eq);
    } else if (bk == MEHDG_BC_FARFIELD) {
      farfield_operator<D, S, CT>(UHs, Us, ud, n, pr.gamma, eq);
    } else {
      for (int s = 0; s < NS; ++s) eq[s] = fh[s];
    }
    CT* K = Kface + (pidx * NDIR_K + dir) * 2 * NS;
    for (int t = 0; t < NS; ++t) {
      K[t] = fh[t].d[0] * wf;
      K[NS + t] = eq[t].d[0] * wf;
    }
    if (MODE == 0 && dir == 0) {
      double* R = rface + pidx * 2 * NS;
      for (int t = 0; t < NS; ++t) {
        R[t] = fh[t].v * wf;
        R[NS + t] = eq[t].v * wf;
      }
    }
  }
}

template <int D, int P, class CT = double, int MODE = 0>
__global__ void __launch_bounds__(128) k_face_point(Geo g, const CT* __restrict__ tab, Phys ph,
                                                     mehdg_problem pr, const int* __restrict__ bkind,
                                                     const int* __restrict__ bside, const int* __restrict__ fnode,
                                                     const int* __restrict__ gather, const CT* __restrict__ uD,
                                                     const CT* __restrict__ u, const CT* __restrict__ q,
                                                     const CT* __restrict__ uh, CT* __restrict__ Kface,
                                                     double* __restrict__ rface, int E,
                                                     const double* __restrict__ fgeo = nullptr) {
  constexpr int NS = D + 2, P1 = P + 1, NG1 = P + 2;
  constexpr int NFS = IPow<P1, D - 1>::v, NFP = IPow<NG1, D - 1>::v;
  constexpr int NDIR_K = NS * (D + 2);
  constexpr int NDIR = (MODE == 2) ? 1 : NDIR_K;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nsf = g.nsf;
  if (tid >= (long long)E * 2 * D * nsf * NFP * NDIR) return;
  const int dir = tid % NDIR;
  long long r = tid / NDIR;
  const int fp = r % NFP; r /= NFP;
  const int sf = r % nsf; r /= nsf;
  const int fl = r % (2 * D);
  const int e = (int)(r / (2 * D));
  Tables<CT> tb = tables(tab, NG1, P1);
  int tang[D];
  face_axes<D>(fl, tang);
  int gi[D], si[D];
  CT wf = CT(1);
  {
    int pp = fp, ss = sf;
    for (int c = 0; c < D - 1; ++c) {
      gi[c] = pp % NG1; pp /= NG1;
      si[c] = ss % g.m; ss /= g.m;
      wf *= tb.gw[gi[c]] * CT(0.5) * (CT)g.he[tang[c]];
    }
  }
  CT Uf[NS], Qf[NS][D], UHf[NS];
  for (int s = 0; s < NS; ++s) {
    Uf[s] = CT(0); UHf[s] = CT(0);
    for (int j = 0; j < D; ++j) Qf[s][j] = CT(0);
  }
  const size_t Np = g.Np;
  for (int il = 0; il < NFS; ++il) {
    int jf = 0, stride = 1, t2 = il;
    CT psi = CT(1);
    for (int c = 0; c < D - 1; ++c) {
      int ic = t2 % P1; t2 /= P1;
      psi *= tb.b1[gi[c] * P1 + ic];
      jf += (si[c] * P + ic) * stride;
      stride *= g.n1;
    }
    int a = fnode[fl * g.Nfn + jf];
    for (int s = 0; s < NS; ++s) {
      Uf[s] += psi * u[((size_t)e * NS + s) * Np + a];
      UHf[s] += psi * uh[gather[(size_t)e * g.Nt + s * g.Nth + fl * g.Nfn + jf]];
      for (int j = 0; j < D; ++j) Qf[s][j] += psi * q[(((size_t)e * D + j) * NS + s) * Np + a];
    }
  }
  double n[D];
  if (fgeo) {   // curved macro: unit outward normal and weight of this face point
    const double* fg = fgeo + ((((size_t)e * 2 * D + fl) * nsf + sf) * NFP + fp) * (D + 1);
    for (int k = 0; k < D; ++k) n[k] = fg[k];
    wf = (CT)fg[D];
  } else {
    for (int k = 0; k < D; ++k) n[k] = 0.0;
    n[fl / 2] = (fl % 2) ? 1.0 : -1.0;
  }
  const int bk = bkind[e * 2 * D + fl];
  const int bs = bside[e * 2 * D + fl];
  const CT* ud = uD ? uD + ((((size_t)e * 2 * D + fl) * nsf + sf) * NFP + fp) * NS : nullptr;
  const size_t pidx = (((size_t)e * 2 * D + fl) * nsf + sf) * NFP + fp;
  face_point_eval<D, CT, MODE>(ph, pr, bk, bs, ud, n, wf, Uf, Qf, UHf, dir, pidx, Kface, rface);
}

template <int D, int P, class BT, class KT = double>
__global__ void __launch_bounds__(256) k_face_contract(Geo g, const double* __restrict__ tab,
                                                        const int* __restrict__ fnode,
                                                        const KT* __restrict__ Kface,
                                                        const double* __restrict__ rface, BT* Auu, BT* Auq,
                                                        BT* Auh, BT* Ahu, BT* Ahq, BT* Ahh,
                                                        double* RU, double* RUh) {
  constexpr int NS = D + 2, P1 = P + 1, NG1 = P + 2;
  constexpr int NFS = IPow<P1, D - 1>::v, NFP = IPow<NG1, D - 1>::v;
  constexpr int NDIR = NS * (D + 2);
  __shared__ double spsi[NFS * NFP];
  __shared__ KT kpsi[NFS * NFP];
  const int e = blockIdx.x;
  const size_t Nu = g.Nu, Nt = g.Nt, Np = g.Np;
  const int Nth = g.Nth, Nfn = g.Nfn;
  const int tid = threadIdx.x;
  for (int fl = 0; fl < 2 * D; ++fl) {
    for (int sf = 0; sf < g.nsf; ++sf) {
      int si[D];
      {
        int ss = sf;
        for (int c = 0; c < D - 1; ++c) { si[c] = ss % g.m; ss /= g.m; }
      }
      __syncthreads();
      for (int i = tid; i < NFS * NFP; i += blockDim.x) {
        int il = i / NFP, fp = i % NFP;
        double v = 1.0;
        int t1 = il, t2 = fp;
        for (int c = 0; c < D - 1; ++c) {
          v *= tab[(t2 % NG1) * P1 + (t1 % P1)];
          t1 /= P1; t2 /= NG1;
        }
        spsi[i] = v;
        kpsi[i] = (KT)v;
      }
      __syncthreads();
      const KT* K = Kface + (((size_t)e * 2 * D + fl) * g.nsf + sf) * NFP * NDIR * 2 * NS;
      const double* R = rface + (((size_t)e * 2 * D + fl) * g.nsf + sf) * NFP * 2 * NS;
      // local node -> face node index and macro node
      auto jface = [&](int il) {
        int jf = 0, stride = 1, t2 = il;
        for (int c = 0; c < D - 1; ++c) {
          jf += (si[c] * P + t2 % P1) * stride;
          t2 /= P1;
          stride *= g.n1;
        }
        return jf;
      };
      const int NOUT = NDIR * 2 * NS * NFS * NFS;
      for (int oi = tid; oi < NOUT; oi += blockDim.x) {
        int jn = oi % NFS;
        int in = (oi / NFS) % NFS;
        int t = (oi / (NFS * NFS)) % NS;
        int et = (oi / (NFS * NFS * NS)) % 2;
        int dir = oi / (NFS * NFS * NS * 2);
        KT sum = KT(0);
        for (int fp = 0; fp < NFP; ++fp)
          sum += kpsi[in * NFP + fp] * K[((size_t)fp * NDIR + dir) * 2 * NS + et * NS + t] * kpsi[jn * NFP + fp];
        int ji = jface(in), jj = jface(jn);
        int ai = fnode[fl * Nfn + ji], aj = fnode[fl * Nfn + jj];
        int s, kind, jd = 0;
        if (dir < NS) { kind = 0; s = dir; }
        else if (dir < NS + NS * D) { kind = 1; jd = (dir - NS) / NS; s = (dir - NS) % NS; }
        else { kind = 2; s = dir - NS - NS * D; }
        if (et == 0) {   // numerical flux tested with phi (u rows)
          size_t row = (size_t)t * Np + ai;
          if (kind == 0) Auh[(size_t)e * Nu * Nt + row * Nt + (size_t)s * Nth + fl * Nfn + jj] += (BT)sum;
          else if (kind == 1) Auq[((size_t)e * D + jd) * Nu * Nu + row * Nu + (size_t)s * Np + aj] += (BT)sum;
          else Auu[(size_t)e * Nu * Nu + row * Nu + (size_t)s * Np + aj] += (BT)sum;
        } else {         // trace equation tested with psi (uhat rows)
          size_t row = (size_t)t * Nth + fl * Nfn + ji;
          if (kind == 0) Ahh[(size_t)e * Nt * Nt + row * Nt + (size_t)s * Nth + fl * Nfn + jj] += (BT)sum;
          else if (kind == 1) Ahq[((size_t)e * D + jd) * Nt * Nu + row * Nu + (size_t)s * Np + aj] += (BT)sum;
          else Ahu[(size_t)e * Nt * Nu + row * Nu + (size_t)s * Np + aj] += (BT)sum;
        }
      }
      for (int oi = tid; oi < 2 * NS * NFS; oi += blockDim.x) {
        int in = oi % NFS;
        int t = (oi / NFS) % NS;
        int et = oi / (NFS * NS);
        double sum = 0.0;
        for (int fp = 0; fp < NFP; ++fp) sum += spsi[in * NFP + fp] * R[(size_t)fp * 2 * NS + et * NS + t];
        int ji = jface(in);
        if (et == 0) RU[((size_t)e * NS + t) * Np + fnode[fl * Nfn + ji]] += sum;
        else RUh[(size_t)e * Nt + (size_t)t * Nth + fl * Nfn + ji] += sum;
      }
    }
  }
}

// R_Q[k][s][a] = M q_k,s + G_k u_s + Gh_k uh_loc,s   (linear part of eq. C38a)
// (M, G_k, Gh_k shared by all macro-elements, or per macro-element at strides sM, sG, sGh)
__global__ void k_rq(Geo g, const double* __restrict__ M, const double* __restrict__ Gk,
                     const double* __restrict__ Ghk, const int* __restrict__ gather, const double* __restrict__ u,
                     const double* __restrict__ q, const double* __restrict__ uh, double* __restrict__ RQ, int E,
                     size_t sM, size_t sG, size_t sGh) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)E * g.d * g.ns * g.Np;
  if (tid >= tot) return;
  int a = tid % g.Np;
  int s = (tid / g.Np) % g.ns;
  int k = (tid / ((long long)g.Np * g.ns)) % g.d;
  int e = (int)(tid / ((long long)g.Np * g.ns * g.d));
  const size_t Np = g.Np;
  const double* Mr = M + e * sM + (size_t)a * Np;
  const double* Gr = Gk + e * sG + ((size_t)k * Np + a) * Np;
  const double* Hr = Ghk + e * sGh + ((size_t)k * Np + a) * g.Nth;
  const double* qe = q + (((size_t)e * g.d + k) * g.ns + s) * Np;
  const double* ue = u + ((size_t)e * g.ns + s) * Np;
  const int* ge = gather + (size_t)e * g.Nt + (size_t)s * g.Nth;
  double acc = 0.0;
  for (int b = 0; b < g.Np; ++b) acc += Mr[b] * qe[b] + Gr[b] * ue[b];
  for (int i = 0; i < g.Nth; ++i) acc += Hr[i] * uh[ge[i]];
  RQ[tid] = acc;
}

template <int D, int P, class BT>
int assemble_dp(mehdg_ctx* ctx, const double* u, const double* q, const double* uh, const mehdg_time_term* tt) {
  Geo g = make_geo(ctx);
  cudaStream_t st = ctx->stream;
  const int E = ctx->E;
  const size_t Nu = ctx->Nu, Nt = ctx->Nt;
  Phys ph{ctx->prob.gamma, ctx->prob.Re, ctx->prob.Pr, ctx->prob.supg, ctx->h_supg, ctx->p};
  BT* Auu = reinterpret_cast<BT*>(ctx->Auu);
  BT* Auq = reinterpret_cast<BT*>(ctx->Auq);
  BT* Auh = reinterpret_cast<BT*>(ctx->Auh);
  BT* Ahu = reinterpret_cast<BT*>(ctx->Ahu);
  BT* Ahq = reinterpret_cast<BT*>(ctx->Ahq);
  BT* Ahh = reinterpret_cast<BT*>(ctx->Ahh);
  BT* Kvol = reinterpret_cast<BT*>(ctx->Kvol);
  CK(cudaMemsetAsync(Auu, 0, sizeof(BT) * E * Nu * Nu, st));
  CK(cudaMemsetAsync(Auq, 0, sizeof(BT) * E * D * Nu * Nu, st));
  CK(cudaMemsetAsync(Auh, 0, sizeof(BT) * E * Nu * Nt, st));
  CK(cudaMemsetAsync(Ahu, 0, sizeof(BT) * E * Nt * Nu, st));
  CK(cudaMemsetAsync(Ahq, 0, sizeof(BT) * E * D * Nt * Nu, st));
  CK(cudaMemsetAsync(Ahh, 0, sizeof(BT) * E * Nt * Nt, st));
  CK(cudaMemsetAsync(ctx->RU, 0, sizeof(double) * E * Nu, st));
  CK(cudaMemsetAsync(ctx->RUh, 0, sizeof(double) * E * Nt, st));
  constexpr int NS = D + 2;
  constexpr int NG = IPow<P + 2, D>::v;
  {
    long long tot = (long long)E * ctx->nel * NG * NS * (1 + D);
    const double* hist = tt ? tt->hist : nullptr;
    const double coef = tt ? tt->coef : 0.0;
    const int supg_time = tt ? tt->supg_time : 0;
    phase_begin(ctx, PH_VOL_POINT);
    if constexpr (sizeof(BT) == 4) {
      // Jacobian columns in FP32 from FP32 copies of the state; residual integrand in FP64
      const long long nu = (long long)E * NS * ctx->Np;
      int rc;
      if ((rc = to_float(ctx, u, ctx->u32, nu))) return rc;
      if ((rc = to_float(ctx, q, ctx->q32, nu * D))) return rc;
      if (hist && (rc = to_float(ctx, hist, ctx->h32, nu))) return rc;
      const long long tot2 = (long long)E * ctx->nel * NG;
      if (ctx->mapped) {
        k_vol_point<D, P, float, float, 1, true><<<(tot + 127) / 128, 128, 0, st>>>(
            g, ctx->tab32, ph, ctx->u32, ctx->q32, hist ? ctx->h32 : nullptr, coef, supg_time, ctx->src32, Kvol,
            nullptr, E, ctx->vgeo);
        CKL();
        k_vol_point<D, P, float, double, 2, true><<<(tot2 + 127) / 128, 128, 0, st>>>(
            g, ctx->tab, ph, u, q, hist, coef, supg_time, ctx->src, nullptr, ctx->rvol, E, ctx->vgeo);
        CKL();
      } else {
        k_vol_point<D, P, float, float, 1><<<(tot + 127) / 128, 128, 0, st>>>(
            g, ctx->tab32, ph, ctx->u32, ctx->q32, hist ? ctx->h32 : nullptr, coef, supg_time, ctx->src32, Kvol,
            nullptr, E);
        CKL();
        k_vol_point<D, P, float, double, 2><<<(tot2 + 127) / 128, 128, 0, st>>>(
            g, ctx->tab, ph, u, q, hist, coef, supg_time, ctx->src, nullptr, ctx->rvol, E);
        CKL();
      }
    } else {
      // FP64: the interpolation once per point, shared by its input directions
      typedef VpCfg<D> VC;
      const long long npts = (long long)E * ctx->nel * NG;
      const unsigned blocks = (unsigned)((npts + VC::PPB - 1) / VC::PPB);
      if (ctx->mapped)
        k_vol_point_sh<D, P, BT, true><<<blocks, VC::NT, 0, st>>>(g, ctx->tab, ph, u, q, hist, coef, supg_time,
                                                                  ctx->src, Kvol, ctx->rvol, E, ctx->vgeo);
      else
        k_vol_point_sh<D, P, BT, false><<<blocks, VC::NT, 0, st>>>(g, ctx->tab, ph, u, q, hist, coef, supg_time,
                                                                   ctx->src, Kvol, ctx->rvol, E, nullptr);
      CKL();
    }
    phase_end(ctx, PH_VOL_POINT);
  }
  {
    dim3 grid(E, D + 1, NS);
    if (ctx->opt.tc_mode != 5) {
      // sum factorisation (both precisions; the dense k_vol_contract is kept as tc_mode 5 for
      // comparison)
      typedef SfCfg<D, P, BT> C;
      CK(cudaFuncSetAttribute(k_vol_contract_sf<D, P, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)C::SMEM));
      phase_begin(ctx, PH_VOL_CONTRACT);
      k_vol_contract_sf<D, P, BT><<<grid, C::NT, C::SMEM, st>>>(g, ctx->tab, Kvol, Auu, Auq);
      CKL();
      phase_end(ctx, PH_VOL_CONTRACT);
    } else {
      typedef VolCfg<D, P, BT> C;
      CK(cudaFuncSetAttribute(k_vol_contract<D, P, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
      phase_begin(ctx, PH_VOL_CONTRACT);
      k_vol_contract<D, P, BT><<<grid, C::NT, C::SMEM, st>>>(g, ctx->tab, Kvol, Auu, Auq);
      CKL();
      phase_end(ctx, PH_VOL_CONTRACT);
    }
    phase_begin(ctx, PH_FACES);
    k_vol_res<D, P><<<E, 128, 0, st>>>(g, ctx->tab, ctx->rvol, ctx->RU);
    CKL();
  }
  {
    constexpr int NFP = IPow<P + 2, D - 1>::v;
    long long tot = (long long)E * 2 * D * ctx->nsf * NFP * NS * (D + 2);
    if constexpr (sizeof(BT) == 4) {
      // Jacobian in FP32 (state copies made for the volume pass), residual in FP64
      int rc;
      if ((rc = to_float(ctx, uh, ctx->uh32, ctx->ntr))) return rc;
      float* Kf = reinterpret_cast<float*>(ctx->Kface);
      k_face_point<D, P, float, 1><<<(tot + 127) / 128, 128, 0, st>>>(
          g, ctx->tab32, ph, ctx->prob, ctx->bkind, ctx->bside, ctx->fnode, ctx->gather, ctx->uD32, ctx->u32,
          ctx->q32, ctx->uh32, Kf, nullptr, E, ctx->fgeo);
      CKL();
      const long long tot2 = (long long)E * 2 * D * ctx->nsf * NFP;
      k_face_point<D, P, double, 2><<<(tot2 + 127) / 128, 128, 0, st>>>(
          g, ctx->tab, ph, ctx->prob, ctx->bkind, ctx->bside, ctx->fnode, ctx->gather, ctx->uD, u, q, uh, nullptr,
          ctx->rface, E, ctx->fgeo);
      CKL();
      k_face_contract<D, P, BT, float><<<E, 256, 0, st>>>(g, ctx->tab, ctx->fnode, Kf, ctx->rface, Auu, Auq, Auh,
                                                          Ahu, Ahq, Ahh, ctx->RU, ctx->RUh);
      CKL();
    } else {
      k_face_point<D, P><<<(tot + 127) / 128, 128, 0, st>>>(g, ctx->tab, ph, ctx->prob, ctx->bkind, ctx->bside,
                                                             ctx->fnode, ctx->gather, ctx->uD, u, q, uh,
                                                             ctx->Kface, ctx->rface, E, ctx->fgeo);
      CKL();
      k_face_contract<D, P, BT><<<E, 256, 0, st>>>(g, ctx->tab, ctx->fnode, ctx->Kface, ctx->rface, Auu, Auq,
                                                    Auh, Ahu, Ahq, Ahh, ctx->RU, ctx->RUh);
      CKL();
    }
  }
  {
    long long tot = (long long)E * ctx->Nq;
    k_rq<<<(tot + 127) / 128, 128, 0, st>>>(g, ctx->Mref, ctx->Gk, ctx->Ghk, ctx->gather, u, q, uh, ctx->RQ, E,
                                            ctx->sM, ctx->sG, ctx->sGh);
    CKL();
    phase_end(ctx, PH_FACES);
  }
  return MEHDG_OK;
}

template <class BT>
int assemble_bt(mehdg_ctx* ctx, const double* u, const double* q, const double* uh, const mehdg_time_term* tt) {
  const int d = ctx->d, p = ctx->p;
  if (d == 2 && p == 1) return assemble_dp<2, 1, BT>(ctx, u, q, uh, tt);
  if (d == 2 && p == 2) return assemble_dp<2, 2, BT>(ctx, u, q, uh, tt);
  if (d == 2 && p == 3) return assemble_dp<2, 3, BT>(ctx, u, q, uh, tt);
  if (d == 3 && p == 1) return assemble_dp<3, 1, BT>(ctx, u, q, uh, tt);
  if (d == 3 && p == 2) return assemble_dp<3, 2, BT>(ctx, u, q, uh, tt);
  if (d == 3 && p == 3) return assemble_dp<3, 3, BT>(ctx, u, q, uh, tt);
  return ctx_fail(ctx, MEHDG_ERR_ARG, "unsupported (dim, p)");
}

// ---------------------------------------------------------------- simplicial macro-elements
// P_p on m-refined simplices (csrc/simplex.cu holds the reference tables and the mesh).  The same
// pointwise physics as the tensor kernels (vol_point_eval in its curved form, face_point_eval),
// with the interpolation read from per-point tables: each Gauss point of sub-simplex el touches
// its NLOC nodes (values and d/dxi), each face point the NFS nodes of its sub-face (the volume
// basis restricted to a face is the trace basis).  The contractions run over sub-elements in
// turn, one CTA per (macro, input block, test species) or per macro, so that no two threads add
// to one block entry at a time.  FP64 only.
template <int D, int P> struct SxN {
  static constexpr int NLOC = (D == 2) ? (P + 1) * (P + 2) / 2 : (P + 1) * (P + 2) * (P + 3) / 6;
  static constexpr int NFS = (D == 2) ? P + 1 : (P + 1) * (P + 2) / 2;
  static constexpr int NG = IPow<P + 3, D>::v, NFP = IPow<P + 3, D - 1>::v;
};

template <int D, int P>
__global__ void __launch_bounds__(128) k_vol_point_sx(Geo g, const double* __restrict__ vtab,
                                                      const int* __restrict__ vnode, Phys ph,
                                                      const double* __restrict__ u, const double* __restrict__ q,
                                                      const double* __restrict__ hist, double coef, int supg_time,
                                                      const double* __restrict__ src, double* __restrict__ Kvol,
                                                      double* __restrict__ rvol, int E,
                                                      const double* __restrict__ vgeo) {
  constexpr int NS = D + 2, NLOC = SxN<D, P>::NLOC, NG = SxN<D, P>::NG;
  constexpr int NDIR = NS * (1 + D);
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nel = g.nel;
  if (tid >= (long long)E * nel * NG * NDIR) return;
  const int dir = (int)(tid % NDIR);
  long long r = tid / NDIR;
  const int gq = (int)(r % NG);
  r /= NG;
  const int el = (int)(r % nel);
  const int e = (int)(r / nel);
  double U[NS], GU[NS][D], Q[NS][D], GQ[NS][D][D], Hh[NS];
  for (int s = 0; s < NS; ++s) {
    U[s] = 0.0;
    Hh[s] = 0.0;
    for (int l = 0; l < D; ++l) {
      GU[s][l] = 0.0;
      Q[s][l] = 0.0;
      for (int j = 0; j < D; ++j) GQ[s][j][l] = 0.0;
    }
  }
  const double* T = vtab + ((size_t)el * NG + gq) * NLOC * (D + 1);
  const int* nd = vnode + (size_t)el * NLOC;
  const size_t Np = g.Np;
  for (int al = 0; al < NLOC; ++al) {
    const int a = nd[al];
    const double phi = T[al * (D + 1)];
    double dphi[D];
    for (int l = 0; l < D; ++l) dphi[l] = T[al * (D + 1) + 1 + l];
    for (int s = 0; s < NS; ++s) {
      const double ua = u[((size_t)e * NS + s) * Np + a];
      U[s] += phi * ua;
      for (int l = 0; l < D; ++l) GU[s][l] += dphi[l] * ua;
      if (hist) Hh[s] += phi * hist[((size_t)e * NS + s) * Np + a];
      for (int j = 0; j < D; ++j) {
        const double qa = q[(((size_t)e * D + j) * NS + s) * Np + a];
        Q[s][j] += phi * qa;
        for (int l = 0; l < D; ++l) GQ[s][j][l] += dphi[l] * qa;
      }
    }
  }
  vol_point_eval<D, P, double, double, 0, true>(g, ph, e, el, gq, dir, 1.0, U, GU, Q, GQ, Hh, coef, supg_time,
                                                src, Kvol, rvol, vgeo, NG);
}

// A_X[(t, a), (s, b)] += sum_g sum_{alpha, beta} T_alpha[g][a] K_X[t][g][(alpha, s), beta] T_beta[g][b]:
// X = 0 A_uu, X = 1 + j A_uq_j; one CTA per (macro, X, t), the sub-simplex's tables in shared memory
template <int D, int P>
__global__ void __launch_bounds__(256) k_vol_contract_sx(Geo g, const double* __restrict__ vtab,
                                                         const int* __restrict__ vnode,
                                                         const double* __restrict__ Kvol, double* Auu, double* Auq) {
  constexpr int NS = D + 2, NLOC = SxN<D, P>::NLOC, NG = SxN<D, P>::NG;
  constexpr int KA = (D + 1) * NS * (D + 1);
  extern __shared__ double sT[];   // [NG][NLOC][D + 1]
  const int e = blockIdx.x, X = blockIdx.y, t = blockIdx.z;
  const int nel = g.nel;
  const size_t Np = g.Np, Nu = g.Nu;
  double* A = (X == 0) ? Auu + (size_t)e * Nu * Nu : Auq + ((size_t)e * D + (X - 1)) * Nu * Nu;
  for (int el = 0; el < nel; ++el) {
    __syncthreads();
    for (int i = threadIdx.x; i < NG * NLOC * (D + 1); i += blockDim.x)
      sT[i] = vtab[(size_t)el * NG * NLOC * (D + 1) + i];
    __syncthreads();
    const double* K = Kvol + ((((size_t)e * (D + 1) + X) * NS + t) * nel + el) * NG * KA;
    const int* nd = vnode + (size_t)el * NLOC;
    for (int o = threadIdx.x; o < NS * NLOC * NLOC; o += blockDim.x) {
      const int s = o / (NLOC * NLOC), i = (o / NLOC) % NLOC, j = o % NLOC;
      double sum = 0.0;
      for (int gq = 0; gq < NG; ++gq) {
        const double* Kg = K + (size_t)gq * KA;
        const double* Ti = sT + ((size_t)gq * NLOC + i) * (D + 1);
        const double* Tj = sT + ((size_t)gq * NLOC + j) * (D + 1);
        for (int al = 0; al <= D; ++al) {
          double inner = 0.0;
          for (int be = 0; be <= D; ++be) inner += Kg[(al * NS + s) * (D + 1) + be] * Tj[be];
          sum += Ti[al] * inner;
        }
      }
      A[((size_t)t * Np + nd[i]) * Nu + (size_t)s * Np + nd[j]] += sum;
    }
  }
}

// R_U[t][a] += sum_g sum_alpha T_alpha[g][a] r[g][t][alpha], one CTA per macro
template <int D, int P>
__global__ void __launch_bounds__(128) k_vol_res_sx(Geo g, const double* __restrict__ vtab,
                                                    const int* __restrict__ vnode, const double* __restrict__ rvol,
                                                    double* __restrict__ RU) {
  constexpr int NS = D + 2, NLOC = SxN<D, P>::NLOC, NG = SxN<D, P>::NG;
  const int e = blockIdx.x, nel = g.nel;
  const size_t Np = g.Np;
  for (int el = 0; el < nel; ++el) {
    __syncthreads();
    const int* nd = vnode + (size_t)el * NLOC;
    for (int o = threadIdx.x; o < NS * NLOC; o += blockDim.x) {
      const int t = o / NLOC, i = o % NLOC;
      double sum = 0.0;
      for (int gq = 0; gq < NG; ++gq) {
        const double* T = vtab + (((size_t)el * NG + gq) * NLOC + i) * (D + 1);
        const double* R = rvol + (((size_t)e * nel + el) * NG + gq) * NS * (D + 1) + t * (D + 1);
        for (int al = 0; al <= D; ++al) sum += T[al] * R[al];
      }
      RU[((size_t)e * NS + t) * Np + nd[i]] += sum;
    }
  }
}

// one thread per (macro, face, sub-face, face point, input direction)
template <int D, int P>
__global__ void __launch_bounds__(128) k_face_point_sx(Geo g, const double* __restrict__ ftab,
                                                       const int* __restrict__ fsub, Phys ph, mehdg_problem pr,
                                                       const int* __restrict__ bkind, const int* __restrict__ bside,
                                                       const int* __restrict__ fnode, const int* __restrict__ gather,
                                                       const double* __restrict__ uD, const double* __restrict__ u,
                                                       const double* __restrict__ q, const double* __restrict__ uh,
                                                       double* __restrict__ Kface, double* __restrict__ rface, int E,
                                                       const double* __restrict__ fgeo) {
  constexpr int NS = D + 2, NFS = SxN<D, P>::NFS, NFP = SxN<D, P>::NFP;
  constexpr int NDIR = NS * (D + 2), NF = D + 1;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nsf = g.nsf;
  if (tid >= (long long)E * NF * nsf * NFP * NDIR) return;
  const int dir = (int)(tid % NDIR);
  long long r = tid / NDIR;
  const int fp = (int)(r % NFP);
  r /= NFP;
  const int sf = (int)(r % nsf);
  r /= nsf;
  const int fl = (int)(r % NF);
  const int e = (int)(r / NF);
  const double* T = ftab + (((size_t)fl * nsf + sf) * NFP + fp) * NFS;
  const int* js = fsub + ((size_t)fl * nsf + sf) * NFS;
  double Uf[NS], Qf[NS][D], UHf[NS];
  for (int s = 0; s < NS; ++s) {
    Uf[s] = 0.0;
    UHf[s] = 0.0;
    for (int j = 0; j < D; ++j) Qf[s][j] = 0.0;
  }
  const size_t Np = g.Np;
  for (int il = 0; il < NFS; ++il) {
    const int jf = js[il];
    const double psi = T[il];
    const int a = fnode[fl * g.Nfn + jf];
    for (int s = 0; s < NS; ++s) {
      Uf[s] += psi * u[((size_t)e * NS + s) * Np + a];
      UHf[s] += psi * uh[gather[(size_t)e * g.Nt + s * g.Nth + fl * g.Nfn + jf]];
      for (int j = 0; j < D; ++j) Qf[s][j] += psi * q[(((size_t)e * D + j) * NS + s) * Np + a];
    }
  }
  const size_t pidx = (((size_t)e * NF + fl) * nsf + sf) * NFP + fp;
  const double* fg = fgeo + pidx * (D + 1);
  double n[D];
  for (int k = 0; k < D; ++k) n[k] = fg[k];
  const int bk = bkind[e * NF + fl], bs = bside[e * NF + fl];
  face_point_eval<D, double, 0>(ph, pr, bk, bs, uD + pidx * NS, n, fg[D], Uf, Qf, UHf, dir, pidx, Kface, rface);
}

// the face blocks and residuals from the face-point columns, one CTA per macro (as k_face_contract)
template <int D, int P>
__global__ void __launch_bounds__(256) k_face_contract_sx(Geo g, const double* __restrict__ ftab,
                                                          const int* __restrict__ fsub, const int* __restrict__ fnode,
                                                          const double* __restrict__ Kface,
                                                          const double* __restrict__ rface, double* Auu, double* Auq,
                                                          double* Auh, double* Ahu, double* Ahq, double* Ahh,
                                                          double* RU, double* RUh) {
  constexpr int NS = D + 2, NFS = SxN<D, P>::NFS, NFP = SxN<D, P>::NFP;
  constexpr int NDIR = NS * (D + 2), NF = D + 1;
  __shared__ double spsi[NFS * NFP];
  const int e = blockIdx.x;
  const size_t Nu = g.Nu, Nt = g.Nt, Np = g.Np;
  const int Nth = g.Nth, Nfn = g.Nfn, nsf = g.nsf;
  const int tid = threadIdx.x;
  for (int fl = 0; fl < NF; ++fl) {
    for (int sf = 0; sf < nsf; ++sf) {
      __syncthreads();
      for (int i = tid; i < NFS * NFP; i += blockDim.x) {
        const int il = i / NFP, fp = i % NFP;
        spsi[i] = ftab[(((size_t)fl * nsf + sf) * NFP + fp) * NFS + il];
      }
      __syncthreads();
      const double* K = Kface + (((size_t)e * NF + fl) * nsf + sf) * NFP * NDIR * 2 * NS;
      const double* R = rface + (((size_t)e * NF + fl) * nsf + sf) * NFP * 2 * NS;
      const int* js = fsub + ((size_t)fl * nsf + sf) * NFS;
      const int NOUT = NDIR * 2 * NS * NFS * NFS;
      for (int oi = tid; oi < NOUT; oi += blockDim.x) {
        const int jn = oi % NFS;
        const int in = (oi / NFS) % NFS;
        const int t = (oi / (NFS * NFS)) % NS;
        const int et = (oi / (NFS * NFS * NS)) % 2;
        const int dir = oi / (NFS * NFS * NS * 2);
        double sum = 0.0;
        for (int fp = 0; fp < NFP; ++fp)
          sum += spsi[in * NFP + fp] * K[((size_t)fp * NDIR + dir) * 2 * NS + et * NS + t] * spsi[jn * NFP + fp];
        const int ji = js[in], jj = js[jn];
        const int ai = fnode[fl * Nfn + ji], aj = fnode[fl * Nfn + jj];
        int s, kind, jd = 0;
        if (dir < NS) { kind = 0; s = dir; }
        else if (dir < NS + NS * D) { kind = 1; jd = (dir - NS) / NS; s = (dir - NS) % NS; }
        else { kind = 2; s = dir - NS - NS * D; }
        if (et == 0) {   // numerical flux tested with phi (u rows)
          const size_t row = (size_t)t * Np + ai;
          if (kind == 0) Auh[(size_t)e * Nu * Nt + row * Nt + (size_t)s * Nth + fl * Nfn + jj] += sum;
          else if (kind == 1) Auq[((size_t)e * D + jd) * Nu * Nu + row * Nu + (size_t)s * Np + aj] += sum;
          else Auu[(size_t)e * Nu * Nu + row * Nu + (size_t)s * Np + aj] += sum;
        } else {         // trace equation tested with psi (uhat rows)
          const size_t row = (size_t)t * Nth + fl * Nfn + ji;
          if (kind == 0) Ahh[(size_t)e * Nt * Nt + row * Nt + (size_t)s * Nth + fl * Nfn + jj] += sum;
          else if (kind == 1) Ahq[((size_t)e * D + jd) * Nt * Nu + row * Nu + (size_t)s * Np + aj] += sum;
          else Ahu[(size_t)e * Nt * Nu + row * Nu + (size_t)s * Np + aj] += sum;
        }
      }
      for (int oi = tid; oi < 2 * NS * NFS; oi += blockDim.x) {
        const int in = oi % NFS;
        const int t = (oi / NFS) % NS;
        const int et = oi / (NFS * NS);
        double sum = 0.0;
        for (int fp = 0; fp < NFP; ++fp) sum += spsi[in * NFP + fp] * R[(size_t)fp * 2 * NS + et * NS + t];
        const int ji = js[in];
        if (et == 0) RU[((size_t)e * NS + t) * Np + fnode[fl * Nfn + ji]] += sum;
        else RUh[(size_t)e * Nt + (size_t)t * Nth + fl * Nfn + ji] += sum;
      }
    }
  }
}

template <int D, int P>
int assemble_sx(mehdg_ctx* ctx, const double* u, const double* q, const double* uh, const mehdg_time_term* tt) {
  typedef SxN<D, P> C;
  constexpr int NS = D + 2;
  Geo g = make_geo(ctx);
  cudaStream_t st = ctx->stream;
  const int E = ctx->E;
  const size_t Nu = ctx->Nu, Nt = ctx->Nt;
  Phys ph{ctx->prob.gamma, ctx->prob.Re, ctx->prob.Pr, ctx->prob.supg, ctx->h_supg, ctx->p};
  CK(cudaMemsetAsync(ctx->Auu, 0, sizeof(double) * E * Nu * Nu, st));
  CK(cudaMemsetAsync(ctx->Auq, 0, sizeof(double) * E * D * Nu * Nu, st));
  CK(cudaMemsetAsync(ctx->Auh, 0, sizeof(double) * E * Nu * Nt, st));
  CK(cudaMemsetAsync(ctx->Ahu, 0, sizeof(double) * E * Nt * Nu, st));
  CK(cudaMemsetAsync(ctx->Ahq, 0, sizeof(double) * E * D * Nt * Nu, st));
  CK(cudaMemsetAsync(ctx->Ahh, 0, sizeof(double) * E * Nt * Nt, st));
  CK(cudaMemsetAsync(ctx->RU, 0, sizeof(double) * E * Nu, st));
  CK(cudaMemsetAsync(ctx->RUh, 0, sizeof(double) * E * Nt, st));
  const double* hist = tt ? tt->hist : nullptr;
  const double coef = tt ? tt->coef : 0.0;
  const int supg_time = tt ? tt->supg_time : 0;
  {
    const long long tot = (long long)E * ctx->nel * C::NG * NS * (1 + D);
    phase_begin(ctx, PH_VOL_POINT);
    k_vol_point_sx<D, P><<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(
        g, ctx->sx_vtab, ctx->sx_vnode, ph, u, q, hist, coef, supg_time, ctx->src, ctx->Kvol, ctx->rvol, E, ctx->vgeo);
    CKL();
    phase_end(ctx, PH_VOL_POINT);
    const size_t smem = sizeof(double) * C::NG * C::NLOC * (D + 1);
    CK(cudaFuncSetAttribute(k_vol_contract_sx<D, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    phase_begin(ctx, PH_VOL_CONTRACT);
    k_vol_contract_sx<D, P><<<dim3(E, D + 1, NS), 256, smem, st>>>(g, ctx->sx_vtab, ctx->sx_vnode, ctx->Kvol, ctx->Auu,
                                                                  ctx->Auq);
    CKL();
    phase_end(ctx, PH_VOL_CONTRACT);
  }
  phase_begin(ctx, PH_FACES);
  k_vol_res_sx<D, P><<<E, 128, 0, st>>>(g, ctx->sx_vtab, ctx->sx_vnode, ctx->rvol, ctx->RU);
  CKL();
  {
    const long long tot = (long long)E * (D + 1) * ctx->nsf * C::NFP * NS * (D + 2);
    k_face_point_sx<D, P><<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(
        g, ctx->sx_ftab, ctx->sx_fsub, ph, ctx->prob, ctx->bkind, ctx->bside, ctx->fnode, ctx->gather, ctx->uD, u, q,
        uh, ctx->Kface, ctx->rface, E, ctx->fgeo);
    CKL();
    k_face_contract_sx<D, P><<<E, 256, 0, st>>>(g, ctx->sx_ftab, ctx->sx_fsub, ctx->fnode, ctx->Kface, ctx->rface,
                                               ctx->Auu, ctx->Auq, ctx->Auh, ctx->Ahu, ctx->Ahq, ctx->Ahh, ctx->RU,
                                               ctx->RUh);
    CKL();
  }
  {
    const long long tot = (long long)E * ctx->Nq;
    k_rq<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(g, ctx->Mref, ctx->Gk, ctx->Ghk, ctx->gather, u, q, uh, ctx->RQ,
                                                        E, ctx->sM, ctx->sG, ctx->sGh);
    CKL();
  }
  phase_end(ctx, PH_FACES);
  return MEHDG_OK;
}

int assemble_simplex(mehdg_ctx* ctx, const double* u, const double* q, const double* uh, const mehdg_time_term* tt) {
  const int d = ctx->d, p = ctx->p;
  if (d == 2 && p == 1) return assemble_sx<2, 1>(ctx, u, q, uh, tt);
  if (d == 2 && p == 2) return assemble_sx<2, 2>(ctx, u, q, uh, tt);
  if (d == 2 && p == 3) return assemble_sx<2, 3>(ctx, u, q, uh, tt);
  if (d == 3 && p == 1) return assemble_sx<3, 1>(ctx, u, q, uh, tt);
  if (d == 3 && p == 2) return assemble_sx<3, 2>(ctx, u, q, uh, tt);
  if (d == 3 && p == 3) return assemble_sx<3, 3>(ctx, u, q, uh, tt);
  return ctx_fail(ctx, MEHDG_ERR_ARG, "unsupported (dim, p)");
}

// ---------------------------------------------------------------- flow diagnostics (Sec. 5.3)
// Per macro-element (one CTA): the integrals of rho |v|^2 / 2, rho (omega . omega) / 2 and 1 by the
// volume quadrature, threads striding over the (sub-element, Gauss point) pairs.  v = m / rho and
// omega = curl v, with the velocity gradient from the HDG gradient q = grad u: d_j v_i = (q_{j,1+i}
// - v_i q_{j,0}) / rho.  Only rho and the momentum are interpolated.  The CTA's sums are reduced by a
// fixed tree into part[e][3] (blockDim.x == FD_NT).
constexpr int FD_NT = 128;

template <int D, int P>
__global__ void __launch_bounds__(FD_NT) k_flow_diag(Geo g, const double* __restrict__ tab,
                                                     const double* __restrict__ u, const double* __restrict__ q,
                                                     const double* __restrict__ vgeo, double* __restrict__ part) {
  constexpr int NS = D + 2, P1 = P + 1, NG1 = P + 2;
  constexpr int NLOC = IPow<P1, D>::v, NG = IPow<NG1, D>::v;
  __shared__ double sb[NG1 * P1], sw[NG1];
  __shared__ double red[3][FD_NT];
  const int e = blockIdx.x;
  for (int i = threadIdx.x; i < NG1 * P1; i += blockDim.x) sb[i] = tab[i];
  for (int i = threadIdx.x; i < NG1; i += blockDim.x) sw[i] = tab[2 * NG1 * P1 + i];
  __syncthreads();
  const size_t Np = g.Np;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int pt = threadIdx.x; pt < g.nel * NG; pt += blockDim.x) {
    const int el = pt / NG, gq = pt % NG;
    int gi[D], li[D];
    double wq = 1.0;
    {
      int gg = gq, ll = el;
      for (int k = 0; k < D; ++k) {
        gi[k] = gg % NG1; gg /= NG1;
        li[k] = ll % g.m; ll /= g.m;
        wq *= sw[gi[k]] * 0.5 * g.he[k];
      }
    }
    if (vgeo) wq = vgeo[(((size_t)e * g.nel + el) * NG + gq) * (D * D + 1) + D * D];
    double U[D + 1], Q[D][D + 1];
    for (int s = 0; s <= D; ++s) {
      U[s] = 0.0;
      for (int j = 0; j < D; ++j) Q[j][s] = 0.0;
    }
    for (int al = 0; al < NLOC; ++al) {
      int a = 0, aa = al, stride = 1;
      double phi = 1.0;
      for (int k = 0; k < D; ++k) {
        const int ak = aa % P1;
        aa /= P1;
        a += (li[k] * P + ak) * stride;
        stride *= g.n1;
        phi *= sb[gi[k] * P1 + ak];
      }
      for (int s = 0; s <= D; ++s) {
        U[s] += phi * u[((size_t)e * NS + s) * Np + a];
        for (int j = 0; j < D; ++j) Q[j][s] += phi * q[(((size_t)e * D + j) * NS + s) * Np + a];
      }
    }
    const double rho = U[0];
    double v[D], gv[D][D], v2 = 0.0;
    for (int i = 0; i < D; ++i) {
      v[i] = U[1 + i] / rho;
      v2 += v[i] * v[i];
    }
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) gv[i][j] = (Q[j][1 + i] - v[i] * Q[j][0]) / rho;
    double w2;
    if constexpr (D == 3) {
      const double o0 = gv[2][1] - gv[1][2], o1 = gv[0][2] - gv[2][0], o2 = gv[1][0] - gv[0][1];
      w2 = o0 * o0 + o1 * o1 + o2 * o2;
    } else {
      const double o = gv[1][0] - gv[0][1];
      w2 = o * o;
    }
    acc[0] += wq * 0.5 * rho * v2;
    acc[1] += wq * 0.5 * rho * w2;
    acc[2] += wq;
  }
  for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int h = FD_NT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) part[(size_t)e * 3 + k] = red[k][0];
}

// out[k] = sum_e part[e][k], one CTA of FD_NT threads, fixed order
__global__ void __launch_bounds__(FD_NT) k_flow_diag_sum(const double* __restrict__ part, int E,
                                                         double* __restrict__ out) {
  __shared__ double red[3][FD_NT];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int e = threadIdx.x; e < E; e += blockDim.x)
    for (int k = 0; k < 3; ++k) acc[k] += part[(size_t)e * 3 + k];
  for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int h = FD_NT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x] = red[threadIdx.x][0];
}

template <int D, int P>
int flow_diag_dp(mehdg_ctx* ctx, const double* u, const double* q) {
  Geo g = make_geo(ctx);
  k_flow_diag<D, P><<<ctx->E, FD_NT, 0, ctx->stream>>>(g, ctx->tab, u, q, ctx->mapped ? ctx->vgeo : nullptr,
                                                        ctx->ddiag);
  CKL();
  k_flow_diag_sum<<<1, FD_NT, 0, ctx->stream>>>(ctx->ddiag, ctx->E, ctx->ddiag + (size_t)ctx->E * 3);
  CKL();
  return MEHDG_OK;
}

}  // namespace

int assemble_all(mehdg_ctx* ctx, const double* u, const double* q, const double* uh, const mehdg_time_term* tt,
                 double* norms) {
  int rc;
  if (ctx->simplex) rc = assemble_simplex(ctx, u, q, uh, tt);
  else if (ctx->opt.precision == MEHDG_PREC_MIXED) rc = assemble_bt<float>(ctx, u, q, uh, tt);
  else rc = assemble_bt<double>(ctx, u, q, uh, tt);
  if (rc) return rc;
  ctx->condensed = false;
  if (norms) {
    double a, b, c;
    rc = vec_dot(ctx, ctx->RQ, ctx->RQ, (long long)ctx->E * ctx->Nq, &a);
    if (rc) return rc;
    rc = vec_dot(ctx, ctx->RU, ctx->RU, (long long)ctx->E * ctx->Nu, &b);
    if (rc) return rc;
    rc = face_reduce(ctx, ctx->RUh, ctx->tv2);
    if (rc) return rc;
    rc = vec_dot(ctx, ctx->tv2, ctx->tv2, ctx->ntr, &c);
    if (rc) return rc;
    norms[0] = sqrt(a);
    norms[1] = sqrt(b);
    norms[2] = sqrt(c);
    norms[3] = sqrt(a + b + c);
  }
  return MEHDG_OK;
}

extern "C" int mehdg_assemble_local(mehdg_ctx* ctx, const double* u, const double* q, const double* uhat,
                                    const mehdg_time_term* tt, double* res_norms) {
  if (!ctx || !u || !q || !uhat) return MEHDG_ERR_ARG;
  return assemble_all(ctx, u, q, uhat, tt, res_norms);
}

extern "C" int mehdg_flow_integrals(mehdg_ctx* ctx, const double* u, const double* q, double* out) {
  if (!ctx || !u || !q || !out) return MEHDG_ERR_ARG;
  if (ctx->simplex) return ctx_fail(ctx, MEHDG_ERR_ARG, "flow integrals: box and shell meshes only");
  const int d = ctx->d, p = ctx->p;
  int rc;
  if (d == 2 && p == 1) rc = flow_diag_dp<2, 1>(ctx, u, q);
  else if (d == 2 && p == 2) rc = flow_diag_dp<2, 2>(ctx, u, q);
  else if (d == 2 && p == 3) rc = flow_diag_dp<2, 3>(ctx, u, q);
  else if (d == 3 && p == 1) rc = flow_diag_dp<3, 1>(ctx, u, q);
  else if (d == 3 && p == 2) rc = flow_diag_dp<3, 2>(ctx, u, q);
  else if (d == 3 && p == 3) rc = flow_diag_dp<3, 3>(ctx, u, q);
  else return ctx_fail(ctx, MEHDG_ERR_ARG, "unsupported (dim, p)");
  if (rc) return rc;
  double* h = ctx->hred;
  CK(cudaMemcpyAsync(h, ctx->ddiag + (size_t)ctx->E * 3, sizeof(double) * 3, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < 3; ++k) out[k] = h[k];
  return MEHDG_OK;
}
