// Pointwise physics of the nondimensional compressible Navier-Stokes system,
// templated on the scalar type so that Dual numbers give exact derivatives.
//
// Sec. 2.1 (eqs. C4-C6): u = (rho, rho v, rho E), q = grad u, gamma P = rho T,
// P = (gamma-1)(rho E - rho |v|^2/2), tau = (1/Re_c)(grad v + grad v^T - (2/d) div v I),
// heat flux phi = -(1/(Re_c Pr (gamma-1))) grad T (mu = kappa = 1), F = [rho v,
// rho v v + P I, rho H v], G = -[0, tau, tau v - phi].  Numerical flux and S of
// Sec. 2.3; SUPG term of eq. C38b with a scalar tau (the paper defines tau only
// by reference; this scalar form is the library's reading).
#pragma once
#include "dual.cuh"

struct Phys {
  double gamma, Re, Pr;
  int supg;
  double h;   // sub-element size used by tau_SUPG
  int p;
};

template <int D, class T>
HD void primitives(const T* u, double g, T& rho, T* v, T& E, T& P, T& Tt) {
  rho = u[0];
  T inv = 1.0 / rho;
  T ke = zero<T>();
#pragma unroll
  for (int i = 0; i < D; ++i) {
    v[i] = u[1 + i] * inv;
    ke = ke + v[i] * v[i];
  }
  E = u[D + 1] * inv;
  P = (g - 1.0) * (u[D + 1] - 0.5 * (rho * ke));
  Tt = g * (P * inv);
}

// F[s][k] (eq. C5a)
template <int D, class T>
HD void inviscid_flux(const T* u, double g, T (*F)[D]) {
  T rho, v[D], E, P, Tt;
  primitives<D, T>(u, g, rho, v, E, P, Tt);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    F[0][k] = u[1 + k];
#pragma unroll
    for (int i = 0; i < D; ++i) F[1 + i][k] = u[1 + i] * v[k];
    F[1 + k][k] = F[1 + k][k] + P;
    F[D + 1][k] = (u[D + 1] + P) * v[k];
  }
}

// G[s][k] (eq. C5b, C6), q[s][k] = d u_s / d x_k
template <int D, class T>
HD void viscous_flux(const T* u, const T (*q)[D], const Phys& ph, T (*G)[D]) {
  const double g = ph.gamma;
  T rho, v[D], E, P, Tt;
  primitives<D, T>(u, g, rho, v, E, P, Tt);
  T inv = 1.0 / rho;
  T gv[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) gv[i][k] = (q[1 + i][k] - v[i] * q[0][k]) * inv;
  T div = gv[0][0];
#pragma unroll
  for (int i = 1; i < D; ++i) div = div + gv[i][i];
  const double rinv = 1.0 / ph.Re;
  const double kc = 1.0 / (ph.Re * ph.Pr * (g - 1.0));
#pragma unroll
  for (int k = 0; k < D; ++k) {
    T gE = (q[D + 1][k] - E * q[0][k]) * inv;
    T vgv = v[0] * gv[0][k];
#pragma unroll
    for (int i = 1; i < D; ++i) vgv = vgv + v[i] * gv[i][k];
    T gT = (g * (g - 1.0)) * (gE - vgv);
    T work = zero<T>();
    G[0][k] = zero<T>();
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T tau = (gv[i][k] + gv[k][i]) * rinv;
      if (i == k) tau = tau - div * ((2.0 / D) * rinv);
      G[1 + i][k] = -tau;
      work = work + tau * v[i];
    }
    // -(tau v - phi) with phi = -kc grad T
    G[D + 1][k] = -(work + kc * gT);
  }
}

// (F^ + G^) n = (F(uh) + G(uh, q)) n + (lambda_max(uh) + S_vis)(u - uh)
template <int D, class T>
HD void trace_flux(const T* uh, const T (*q)[D], const T* u, const double* n, const Phys& ph, T* out) {
  T F[D + 2][D], G[D + 2][D];
  inviscid_flux<D, T>(uh, ph.gamma, F);
  viscous_flux<D, T>(uh, q, ph, G);
  T rho, v[D], E, P, Tt;
  primitives<D, T>(uh, ph.gamma, rho, v, E, P, Tt);
  T vn = v[0] * n[0];
#pragma unroll
  for (int k = 1; k < D; ++k) vn = vn + v[k] * n[k];
  T lam = dabs(vn) + dsqrt(Tt);
  const double rinv = 1.0 / ph.Re;
#pragma unroll
  for (int s = 0; s < D + 2; ++s) {
    T fn = (F[s][0] + G[s][0]) * n[0];
#pragma unroll
    for (int k = 1; k < D; ++k) fn = fn + (F[s][k] + G[s][k]) * n[k];
    double sv = (s == 0) ? 0.0 : (s == D + 1 ? rinv / ((ph.gamma - 1.0) * ph.Pr) : rinv);
    out[s] = fn + (lam + sv) * (u[s] - uh[s]);
  }
}

// isothermal no-slip wall: (rho^ - rho, rho^ v^ - rho^ v_w, rho^ E^ - rho^ (e_w + |v_w|^2/2))
template <int D, class T>
HD void wall_operator(const T* uh, const T* u, double Tw, const double* vw, double g, T* out) {
  double ew = Tw / (g * (g - 1.0));
  double kw = 0.0;
  for (int i = 0; i < D; ++i) kw += vw[i] * vw[i];
  out[0] = uh[0] - u[0];
#pragma unroll
  for (int i = 0; i < D; ++i) out[1 + i] = uh[1 + i] - uh[0] * vw[i];
  out[D + 1] = uh[D + 1] - uh[0] * (ew + 0.5 * kw);
}

// characteristic far field towards the uniform state uinf:
//   B^ = A_n^+(uh) (u - uh) - A_n^-(uh) (uinf - uh),  A_n^+- = (A_n +- |A_n|_delta) / 2,
// A_n = d(F(uh) n)/du.  A jump w splits into the two acoustic waves (speeds v_n -/+ c, right
// eigenvectors (1, v -/+ c n, H -/+ c v_n), strengths (dp -/+ rho c dv_n) / (2 c^2) with dp and
// dv_n the pressure and normal-velocity perturbations of w) and a remainder moving at v_n.
// |lambda|_delta = sqrt(lambda^2 + (0.05 c)^2) keeps the operator smooth (and invertible where
// the flow is tangent to the boundary).
template <int D, class T, class U>
HD void farfield_operator(const T* uh, const T* u, const U* uinf, const double* n, double g, T* out) {
  const double delta = 0.05;
  T rho, v[D], E, P, Tt;
  primitives<D, T>(uh, g, rho, v, E, P, Tt);
  T c = dsqrt(Tt);
  T H = E + P / rho;
  T vn = v[0] * n[0], ke = v[0] * v[0];
#pragma unroll
  for (int k = 1; k < D; ++k) {
    vn = vn + v[k] * n[k];
    ke = ke + v[k] * v[k];
  }
  ke = 0.5 * ke;
  T dc2 = (delta * c) * (delta * c);
  T lam[3] = {vn - c, vn, vn + c};
  T lp[3], lm[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T a = dsqrt(lam[i] * lam[i] + dc2);
    lp[i] = 0.5 * (lam[i] + a);
    lm[i] = 0.5 * (lam[i] - a);
  }
#pragma unroll
  for (int s = 0; s < D + 2; ++s) out[s] = zero<T>();
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    T w[D + 2];
#pragma unroll
    for (int s = 0; s < D + 2; ++s) w[s] = side == 0 ? u[s] - uh[s] : (double)uinf[s] - uh[s];
    T mw = w[1] * v[0], nw = w[1] * n[0];
#pragma unroll
    for (int k = 1; k < D; ++k) {
      mw = mw + w[1 + k] * v[k];
      nw = nw + w[1 + k] * n[k];
    }
    T dp = (g - 1.0) * (w[D + 1] - mw + ke * w[0]);
    T dvn = (nw - vn * w[0]) / rho;
    T i2c2 = 0.5 / Tt;
    T s1 = (dp - rho * c * dvn) * i2c2, s5 = (dp + rho * c * dvn) * i2c2;
    const T* L = side == 0 ? lp : lm;
    T c1 = (L[0] - L[1]) * s1, c5 = (L[2] - L[1]) * s5;
    T r[D + 2];
    r[0] = L[1] * w[0] + c1 + c5;
#pragma unroll
    for (int k = 0; k < D; ++k) r[1 + k] = L[1] * w[1 + k] + c1 * (v[k] - c * n[k]) + c5 * (v[k] + c * n[k]);
    r[D + 1] = L[1] * w[D + 1] + c1 * (H - c * vn) + c5 * (H + c * vn);
#pragma unroll
    for (int s = 0; s < D + 2; ++s) out[s] = side == 0 ? out[s] + r[s] : out[s] - r[s];
  }
}

// scalar tau_SUPG = ((2 (|v|+c) p/h)^2 + (4 p^2 /(Re rho h^2))^2)^(-1/2), |v| with derivative 0
// at v = 0
template <int D, class T>
HD T supg_tau(const T* u, const Phys& ph) {
  T rho, v[D], E, P, Tt;
  primitives<D, T>(u, ph.gamma, rho, v, E, P, Tt);
  T vv = v[0] * v[0];
#pragma unroll
  for (int i = 1; i < D; ++i) vv = vv + v[i] * v[i];
  T a = (2.0 * ph.p / ph.h) * (dsqrt0(vv) + dsqrt(Tt));
  T b = (4.0 * ph.p * ph.p / (ph.Re * ph.h * ph.h)) / rho;
  return 1.0 / dsqrt(a * a + b * b);
}

// Volume integrand of R_U at a point: R_U[t,a] += w (phi_a W_t + sum_k d_k phi_a V_tk).
// Also returns FG = F + G (so that outer derivatives give the flux Jacobians),
// A[k][t][s] = dF_tk/du_s and tau (used only when SUPG is on).
// S is a plain scalar (values) or Dual<., 1> (one Jacobian column), in FP64 or FP32.
template <int D, class S, class FT = double>
HD void vol_integrand(const S* U, const S (*GU)[D], const S (*Q)[D], const S (*GQ)[D][D],
                      const S* time, const FT* f, const Phys& ph, int supg_time,
                      S* W, S (*V)[D], S (*FG)[D], S (*A)[D + 2][D + 2], S& tau) {
  constexpr int NS = D + 2;
#pragma unroll
  for (int t = 0; t < NS; ++t) W[t] = time[t] - f[t];
  if (!ph.supg) {
    S F[NS][D], G[NS][D];
    inviscid_flux<D, S>(U, ph.gamma, F);
    viscous_flux<D, S>(U, Q, ph, G);
#pragma unroll
    for (int t = 0; t < NS; ++t)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        FG[t][k] = F[t][k] + G[t][k];
        V[t][k] = -FG[t][k];
      }
    tau = zero<S>();
    return;
  }
  // A_k = dF_k/du by a forward pass over the NS state directions
  {
    typedef Dual<S, NS> IA;
    IA ua[NS], Fa[NS][D];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      ua[s] = zero<IA>();
      ua[s].v = U[s];
      ua[s].d[s] = cst<S>(1.0);
    }
    inviscid_flux<D, IA>(ua, ph.gamma, Fa);
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int t = 0; t < NS; ++t)
#pragma unroll
        for (int s = 0; s < NS; ++s) A[k][t][s] = Fa[t][k].d[s];
  }
  // strong-form flux divergence: column l differentiated along (d_l u, d_l q)
  S div[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) div[t] = zero<S>();
#pragma unroll
  for (int l = 0; l < D; ++l) {
    typedef Dual<S, 1> IB;
    IB ub[NS], qb[NS][D], Fb[NS][D], Gb[NS][D];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      ub[s].v = U[s];
      ub[s].d[0] = GU[s][l];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        qb[s][j].v = Q[s][j];
        qb[s][j].d[0] = GQ[s][j][l];
      }
    }
    inviscid_flux<D, IB>(ub, ph.gamma, Fb);
    viscous_flux<D, IB>(ub, qb, ph, Gb);
#pragma unroll
    for (int t = 0; t < NS; ++t) div[t] = div[t] + (Fb[t][l].d[0] + Gb[t][l].d[0]);
    if (l == 0) {
#pragma unroll
      for (int t = 0; t < NS; ++t)
#pragma unroll
        for (int k = 0; k < D; ++k) FG[t][k] = Fb[t][k].v + Gb[t][k].v;
    }
  }
  tau = supg_tau<D, S>(U, ph);
  S tR[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    S R = div[s] - f[s];
    if (supg_time) R = R + time[s];
    tR[s] = tau * R;
  }
#pragma unroll
  for (int t = 0; t < NS; ++t)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      S acc = -FG[t][k];
#pragma unroll
      for (int s = 0; s < NS; ++s) acc = acc + A[k][s][t] * tR[s];
      V[t][k] = acc;
    }
}

// ---------------------------------------------------------------- closed-form fields
// conserved state from primitives, templated on the coordinate scalar X
template <int D, class X>
HD void conserved_from(const X& rho, const X* v, const X& P, double g, X* u) {
  u[0] = rho;
  X ke = zero<X>();
#pragma unroll
  for (int i = 0; i < D; ++i) {
    u[1 + i] = rho * v[i];
    ke = ke + v[i] * v[i];
  }
  u[D + 1] = P / (g - 1.0) + 0.5 * (rho * ke);
}

// manufactured solution: rho = 1 + A prod sin(pi x_k); v_k = V sin(2 pi x_k) (k even),
// V cos(2 pi x_k) (k odd); P = 1/gamma + Pa cos(pi sum x_k)
template <int D, class X>
HD void field_mms(const X* x, const double* par, double g, X* u) {
  const double PI = 3.14159265358979323846;
  X prod = cst<X>(1.0);
  X sx = zero<X>();
  X v[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    prod = prod * dsin(PI * x[k]);
    sx = sx + x[k];
    v[k] = (k % 2 == 0) ? par[1] * dsin((2.0 * PI) * x[k]) : par[1] * dcos((2.0 * PI) * x[k]);
  }
  X rho = 1.0 + par[0] * prod;
  X P = (1.0 / g) + par[2] * dcos(PI * sx);
  conserved_from<D, X>(rho, v, P, g, u);
}

// Taylor-Green initial state (L = rho0 = 1, P0 = 1/gamma, isothermal)
template <int D, class X>
HD void field_tgv(const X* x, const double* par, double g, X* u) {
  const double V0 = par[0];
  const double P0 = 1.0 / g;
  X v[D];
  X cz = (D == 3) ? dcos(x[D - 1]) : cst<X>(1.0);
  v[0] = V0 * ((dsin(x[0]) * dcos(x[1])) * cz);
  v[1] = -V0 * ((dcos(x[0]) * dsin(x[1])) * cz);
  if (D == 3) v[D - 1] = zero<X>();
  X c2z = (D == 3) ? dcos(2.0 * x[D - 1]) + 2.0 : cst<X>(3.0);
  X P = P0 + (V0 * V0 / 16.0) * ((dcos(2.0 * x[0]) + dcos(2.0 * x[1])) * c2z);
  X rho = P / P0;
  conserved_from<D, X>(rho, v, P, g, u);
}

// compressible Couette flow with a source term (Sec. 5.1, eq. CF0; the reading in acoustic units):
// v_1 = M x_2 log(1 + x_2), v_2 = v_3 = 0, T = alpha + x_2 (beta - alpha) + K x_2 (1 - x_2),
// P = 1/gamma, rho = gamma P / T; par: M, alpha, beta, K
template <int D, class X>
HD void field_couette3d(const X* x, const double* par, double g, X* u) {
  const X y = x[1];
  X v[D];
  v[0] = par[0] * (y * dlog(1.0 + y));
  for (int k = 1; k < D; ++k) v[k] = zero<X>();
  X T = par[1] + y * (par[2] - par[1]) + par[3] * (y * (1.0 - y));
  X P = cst<X>(1.0 / g);
  X rho = 1.0 / T;
  conserved_from<D, X>(rho, v, P, g, u);
}

// the source f = div (F + G) of a closed-form field (the manufactured solution, or the 3D Couette
// flow when couette3d) at the point x: the field on second-order duals gives u, grad u and the
// derivatives of grad u, first-order duals carry the fluxes' divergence
template <int D>
HD void closed_form_source(bool couette3d, const double* par, double g, double Re, double Pr, const double* x,
                           double* f) {
  constexpr int NS = D + 2;
  typedef Dual<Dual<double, D>, D> X2;
  typedef Dual<double, D> T1;
  X2 xs[D];
  for (int k = 0; k < D; ++k) {
    xs[k] = zero<X2>();
    xs[k].v.v = x[k];
    xs[k].v.d[k] = 1.0;
    xs[k].d[k].v = 1.0;
  }
  X2 u2[NS];
  if (couette3d) field_couette3d<D, X2>(xs, par, g, u2);
  else field_mms<D, X2>(xs, par, g, u2);
  T1 uu[NS], qq[NS][D], F[NS][D], G[NS][D];
  for (int s = 0; s < NS; ++s) {
    uu[s].v = u2[s].v.v;
    for (int l = 0; l < D; ++l) uu[s].d[l] = u2[s].v.d[l];
    for (int j = 0; j < D; ++j) {
      qq[s][j].v = u2[s].d[j].v;
      for (int l = 0; l < D; ++l) qq[s][j].d[l] = u2[s].d[j].d[l];
    }
  }
  Phys ph{g, Re, Pr, 0, 1.0, 1};
  inviscid_flux<D, T1>(uu, g, F);
  viscous_flux<D, T1>(uu, qq, ph, G);
  for (int s = 0; s < NS; ++s) {
    double v = 0.0;
    for (int l = 0; l < D; ++l) v += F[s][l].d[l] + G[s][l].d[l];
    f[s] = v;
  }
}

template <int D>
HD void field_uniform(const double* par, double g, double* u) {
  double rho = par[0], v[D];
  for (int i = 0; i < D; ++i) v[i] = par[1 + i];
  double P = rho * par[4] / g;
  conserved_from<D, double>(rho, v, P, g, u);
}

// the closed-form state of a problem's field at the point x: kind 1 the manufactured solution,
// 3 the Taylor-Green vortex, 5 the 3D Couette flow, otherwise the uniform state of par (the
// values of the library's field kinds)
template <int D>
HD void closed_form_state(int kind, const double* par, double g, const double* x, double* u) {
  if (kind == 1) field_mms<D, double>(x, par, g, u);
  else if (kind == 5) field_couette3d<D, double>(x, par, g, u);
  else if (kind == 3) field_tgv<D, double>(x, par, g, u);
  else field_uniform<D>(par, g, u);
}
