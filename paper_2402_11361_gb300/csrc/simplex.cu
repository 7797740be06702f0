// Simplicial macro-elements (Sec. 2.2: the paper's element type): P_p on m-refined simplices.
//
// Reference macro-element: the Kuhn simplex K = {1 >= xi_1 >= ... >= xi_d >= 0}.  Its
// m-refinement is the Freudenthal subdivision of the m-grid of [0, 1]^d restricted to K: the
// cells c with c_1 >= ... >= c_d, each with the axis orders pi that keep tied cell indices in
// axis order, give the m^d sub-simplices {1 >= y_pi1 >= ... >= y_pid >= 0}, y = m xi - c.  P_p
// with equispaced Lagrange nodes on each; all nodes are lattice points a / (m p) of K,
// m p >= a_1 >= ... >= a_d >= 0 (lexicographic order, a_d fastest), so the space is
// continuous.  Faces, in this order: xi_1 = 1, xi_k = xi_{k+1} (k = 1 .. d-1), xi_d = 0 (face
// k is opposite the vertex P_k = e_1 + ... + e_k); the trace space on a face is continuous P_p
// on its m^(d-1) sub-faces, with the face's lattice points (lattice order) as nodes; the
// volume basis restricted to a face is that trace basis.
//
// Quadrature: on every sub-simplex the collapsed Gauss-Legendre rule with p + 3 points per
// direction, z_k = s_k prod_{i<k} (1 - s_i), mapped by y_pi_j = z_j + ... + z_d; on every
// sub-face the (d-1)-dimensional rule mapped onto the sub-face in face coordinates t (the
// barycentric coordinates of the face's vertices but the first), from the sub-face's first
// vertex.  Mesh: every cell of a box grid is split into d! macro-elements x = C + H P_sigma xi
// (x_sigma_k = C_sigma_k + H_sigma_k xi_k), e = cell d! + (rank of sigma among the
// permutations in lexicographic order), cell index axis 0 fastest.  All macro-elements are
// affine, so their mass, derivative and face matrices come from the reference tables on the
// host; the curved-macro path then applies (per-macro liftings, dense condensation).
#include <algorithm>
#include <cmath>
#include <map>

#include "internal.cuh"
#include "physics.cuh"

namespace {

int binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return (int)r;
}

// all integer tuples in [0, n]^d, last entry fastest
std::vector<std::vector<int>> tuples(int d, int n) {
  std::vector<std::vector<int>> out;
  std::vector<int> a(d, 0);
  long long tot = 1;
  for (int k = 0; k < d; ++k) tot *= (n + 1);
  for (long long i = 0; i < tot; ++i) {
    long long r = i;
    for (int k = d - 1; k >= 0; --k) {
      a[k] = (int)(r % (n + 1));
      r /= (n + 1);
    }
    out.push_back(a);
  }
  return out;
}

// collapsed Gauss-Legendre rule on the unit simplex of dimension d (points [Q][d], weights [Q])
void collapsed_rule(int d, int nq, std::vector<double>& z, std::vector<double>& w) {
  z.clear();
  w.clear();
  if (d == 0) {
    w.push_back(1.0);
    return;
  }
  std::vector<double> xg, wg;
  gauss_rule(nq, xg, wg);
  for (auto& idx : tuples(d, nq - 1)) {
    double rem = 1.0, wt = 1.0;
    for (int k = 0; k < d; ++k) {
      const double s = 0.5 * (xg[idx[k]] + 1.0), ws = 0.5 * wg[idx[k]];
      z.push_back(s * rem);
      wt *= ws * rem;
      rem *= 1.0 - s;
    }
    w.push_back(wt);
  }
}

// monomial exponents |alpha| <= p in dimension dy (last entry fastest)
std::vector<std::vector<int>> exponents(int dy, int p) {
  std::vector<std::vector<int>> out;
  for (auto& a : tuples(dy, p)) {
    int s = 0;
    for (int v : a) s += v;
    if (s <= p) out.push_back(a);
  }
  return out;
}

// Lagrange basis of P_p on nodes [n][dy]: coefficient matrix C (phi_i = sum_j mono_j C[j][i])
struct Lagr {
  int dy = 0;
  std::vector<std::vector<int>> ex;
  std::vector<double> C;
  void build(const std::vector<double>& nodes, int n, int dy_, int p) {
    dy = dy_;
    ex = exponents(dy, p);
    std::vector<double> V((size_t)n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = 1.0;
        for (int k = 0; k < dy; ++k) v *= std::pow(nodes[(size_t)i * dy + k], ex[j][k]);
        V[(size_t)i * n + j] = v;
      }
    invert(V, n);
    C = V;
  }
  // values phi[n] and derivatives dphi[dy][n] at y
  void eval(const double* y, double* phi, double* dphi) const {
    const int n = (int)ex.size();
    for (int i = 0; i < n; ++i) {
      phi[i] = 0.0;
      for (int l = 0; l < dy; ++l) dphi[(size_t)l * n + i] = 0.0;
    }
    for (int j = 0; j < n; ++j) {
      double mono = 1.0;
      for (int k = 0; k < dy; ++k) mono *= std::pow(y[k], ex[j][k]);
      for (int i = 0; i < n; ++i) phi[i] += mono * C[(size_t)j * n + i];
      for (int l = 0; l < dy; ++l) {
        if (ex[j][l] == 0) continue;
        double dm = ex[j][l] * std::pow(y[l], ex[j][l] - 1);
        for (int k = 0; k < dy; ++k)
          if (k != l) dm *= std::pow(y[k], ex[j][k]);
        for (int i = 0; i < n; ++i) dphi[(size_t)l * n + i] += dm * C[(size_t)j * n + i];
      }
    }
  }
};

// face fl of K: does lattice point a (integer, spacing 1/n) lie on it; unit outward normal
bool on_face(int d, int n, int fl, const int* a) {
  if (fl == 0) return a[0] == n;
  if (fl == d) return a[d - 1] == 0;
  return a[fl - 1] == a[fl];
}
bool on_face_xi(int d, int fl, const double* x) {
  const double tol = 1e-12;
  if (fl == 0) return std::fabs(x[0] - 1.0) < tol;
  if (fl == d) return std::fabs(x[d - 1]) < tol;
  return std::fabs(x[fl - 1] - x[fl]) < tol;
}

}  // namespace

// ---------------------------------------------------------------- reference tables (host)
int sx_reference(int d, int m, int p, SxRef& R) {
  R = SxRef();
  R.d = d;
  R.m = m;
  R.p = p;
  const int n = m * p, nq = p + 3;
  for (auto& a : tuples(d, n)) {
    bool ok = true;
    for (int k = 0; k + 1 < d; ++k) ok = ok && a[k] >= a[k + 1];
    if (ok) R.lat.insert(R.lat.end(), a.begin(), a.end());
  }
  R.Np = (int)R.lat.size() / d;
  std::map<std::vector<int>, int> index;
  for (int i = 0; i < R.Np; ++i) index[std::vector<int>(R.lat.begin() + (size_t)i * d, R.lat.begin() + (size_t)(i + 1) * d)] = i;
  R.nloc = binom(p + d, d);
  R.nfs = binom(p + d - 1, d - 1);
  R.Nfn = binom(n + d - 1, d - 1);
  std::vector<double> zr, wr, zf, wf;
  collapsed_rule(d, nq, zr, wr);
  collapsed_rule(d - 1, nq, zf, wf);
  R.ng = (int)wr.size();
  R.nfp = (int)wf.size();
  // sub-simplices
  std::vector<int> perm(d);
  struct Sub { std::vector<int> c, pi, verts, nodes; Lagr basis; };
  std::vector<Sub> subs;
  for (auto& c : tuples(d, m - 1)) {
    bool mono = true;
    for (int k = 0; k + 1 < d; ++k) mono = mono && c[k] >= c[k + 1];
    if (!mono) continue;
    for (int k = 0; k < d; ++k) perm[k] = k;
    do {
      std::vector<int> pos(d);
      for (int r = 0; r < d; ++r) pos[perm[r]] = r;
      bool ok = true;
      for (int k = 0; k + 1 < d; ++k)
        if (c[k] == c[k + 1] && pos[k] > pos[k + 1]) ok = false;
      if (!ok) continue;
      Sub sb;
      sb.c = c;
      sb.pi = perm;
      sb.verts.assign(c.begin(), c.end());
      std::vector<int> v = c;
      for (int k = 0; k < d; ++k) {
        v[perm[k]] += 1;
        sb.verts.insert(sb.verts.end(), v.begin(), v.end());
      }
      std::vector<double> ynodes;
      for (auto& b : tuples(d, p)) {
        bool inb = true;
        for (int k = 0; k + 1 < d; ++k) inb = inb && b[perm[k]] >= b[perm[k + 1]];
        if (!inb) continue;
        std::vector<int> a(d);
        for (int k = 0; k < d; ++k) a[k] = c[k] * p + b[k];
        auto it = index.find(a);
        if (it == index.end()) return MEHDG_ERR_ARG;
        sb.nodes.push_back(it->second);
        for (int k = 0; k < d; ++k) ynodes.push_back((double)b[k] / p);
      }
      if ((int)sb.nodes.size() != R.nloc) return MEHDG_ERR_ARG;
      sb.basis.build(ynodes, R.nloc, d, p);
      subs.push_back(sb);
    } while (std::next_permutation(perm.begin(), perm.end()));
  }
  R.nel = (int)subs.size();
  if (R.nel != (int)std::lround(std::pow((double)m, d))) return MEHDG_ERR_ARG;
  // volume points: y_pi_j = z_j + ... + z_d, xi = (c + y) / m
  const double md = std::pow((double)m, d);
  R.vxi.assign((size_t)R.nel * R.ng * d, 0.0);
  R.vw.assign((size_t)R.nel * R.ng, 0.0);
  R.vtab.assign((size_t)R.nel * R.ng * R.nloc * (d + 1), 0.0);
  R.vnode.assign((size_t)R.nel * R.nloc, 0);
  std::vector<double> phi(R.nloc), dphi((size_t)d * R.nloc), y(d);
  for (int el = 0; el < R.nel; ++el) {
    const Sub& sb = subs[el];
    for (int al = 0; al < R.nloc; ++al) R.vnode[(size_t)el * R.nloc + al] = sb.nodes[al];
    for (int g = 0; g < R.ng; ++g) {
      for (int j = 0; j < d; ++j) {
        double acc = 0.0;
        for (int k = j; k < d; ++k) acc += zr[(size_t)g * d + k];
        y[sb.pi[j]] = acc;
      }
      const size_t pt = (size_t)el * R.ng + g;
      for (int k = 0; k < d; ++k) R.vxi[pt * d + k] = (sb.c[k] + y[k]) / m;
      R.vw[pt] = wr[g] / md;
      sb.basis.eval(y.data(), phi.data(), dphi.data());
      for (int al = 0; al < R.nloc; ++al) {
        double* T = &R.vtab[(pt * R.nloc + al) * (d + 1)];
        T[0] = phi[al];
        for (int l = 0; l < d; ++l) T[1 + l] = dphi[(size_t)l * R.nloc + al] * m;
      }
    }
  }
  // faces
  const int nf = d + 1;
  R.nsf = (int)std::lround(std::pow((double)m, d - 1));
  R.fnodes.assign((size_t)nf * R.Nfn, 0);
  R.nref.assign((size_t)nf * d, 0.0);
  R.fM.assign((size_t)nf * d * (d - 1), 0.0);
  R.fxi.assign((size_t)nf * R.nsf * R.nfp * d, 0.0);
  R.fwt.assign((size_t)nf * R.nsf * R.nfp, 0.0);
  R.ftab.assign((size_t)nf * R.nsf * R.nfp * R.nfs, 0.0);
  R.fsub.assign((size_t)nf * R.nsf * R.nfs, 0);
  for (int fl = 0; fl < nf; ++fl) {
    int cnt = 0;
    std::vector<int> fpos(R.Np, -1);
    for (int i = 0; i < R.Np; ++i)
      if (on_face(d, n, fl, &R.lat[(size_t)i * d])) {
        if (cnt >= R.Nfn) return MEHDG_ERR_ARG;
        fpos[i] = cnt;
        R.fnodes[(size_t)fl * R.Nfn + cnt++] = i;
      }
    if (cnt != R.Nfn) return MEHDG_ERR_ARG;
    double* nr = &R.nref[(size_t)fl * d];
    if (fl == 0) nr[0] = 1.0;
    else if (fl == d) nr[d - 1] = -1.0;
    else { nr[fl - 1] = -std::sqrt(0.5); nr[fl] = std::sqrt(0.5); }
    // face vertices: P_j (first j coordinates 1), j != fl, in increasing j
    std::vector<std::vector<double>> W;
    for (int j = 0; j <= d; ++j) {
      if (j == fl) continue;
      std::vector<double> v(d, 0.0);
      for (int k = 0; k < j; ++k) v[k] = 1.0;
      W.push_back(v);
    }
    double* M = &R.fM[(size_t)fl * d * (d - 1)];   // [d][d-1]
    for (int i = 0; i < d - 1; ++i)
      for (int k = 0; k < d; ++k) M[k * (d - 1) + i] = W[i + 1][k] - W[0][k];
    // face coordinates t of a point on the face: (M^T M) t = M^T (xi - W0)
    std::vector<double> MtM((size_t)(d - 1) * (d - 1), 0.0);
    for (int i = 0; i < d - 1; ++i)
      for (int j = 0; j < d - 1; ++j)
        for (int k = 0; k < d; ++k) MtM[i * (d - 1) + j] += M[k * (d - 1) + i] * M[k * (d - 1) + j];
    std::vector<double> MtMi = MtM;
    invert(MtMi, d - 1);
    auto tcoord = [&](const double* xi, double* t) {
      std::vector<double> r(d - 1, 0.0);
      for (int i = 0; i < d - 1; ++i)
        for (int k = 0; k < d; ++k) r[i] += M[k * (d - 1) + i] * (xi[k] - W[0][k]);
      for (int i = 0; i < d - 1; ++i) {
        t[i] = 0.0;
        for (int j = 0; j < d - 1; ++j) t[i] += MtMi[i * (d - 1) + j] * r[j];
      }
    };
    int sf = 0;
    for (int el = 0; el < R.nel; ++el) {
      const Sub& sb = subs[el];
      for (int drop = 0; drop <= d; ++drop) {
        std::vector<std::vector<double>> sv;
        bool all = true;
        for (int i = 0; i <= d; ++i) {
          if (i == drop) continue;
          std::vector<double> v(d);
          for (int k = 0; k < d; ++k) v[k] = (double)sb.verts[(size_t)i * d + k] / m;
          all = all && on_face_xi(d, fl, v.data());
          sv.push_back(v);
        }
        if (!all) continue;
        if (sf >= R.nsf) return MEHDG_ERR_ARG;
        // the sub-face's nodes (sub-simplex nodes on the face) and their trace basis in t
        std::vector<double> tn;
        int il = 0;
        std::vector<double> tt(std::max(1, d - 1));
        for (int al = 0; al < R.nloc; ++al) {
          const int a = sb.nodes[al];
          if (fpos[a] < 0) continue;
          if (il >= R.nfs) return MEHDG_ERR_ARG;
          R.fsub[((size_t)fl * R.nsf + sf) * R.nfs + il++] = fpos[a];
          std::vector<double> xa(d);
          for (int k = 0; k < d; ++k) xa[k] = (double)R.lat[(size_t)a * d + k] / n;
          tcoord(xa.data(), tt.data());
          tn.insert(tn.end(), tt.begin(), tt.begin() + (d - 1));
        }
        if (il != R.nfs) return MEHDG_ERR_ARG;
        Lagr tb;
        tb.build(tn, R.nfs, d - 1, p);
        std::vector<double> T0(d - 1), Tm((size_t)(d - 1) * (d - 1));
        tcoord(sv[0].data(), T0.data());
        for (int i = 1; i < d; ++i) {
          tcoord(sv[i].data(), tt.data());
          for (int r = 0; r < d - 1; ++r) Tm[r * (d - 1) + (i - 1)] = tt[r] - T0[r];
        }
        // |det Tm|
        std::vector<double> LU = Tm;
        double det = 1.0;
        const int k1 = d - 1;
        for (int c = 0; c < k1; ++c) {
          int piv = c;
          for (int r = c + 1; r < k1; ++r)
            if (std::fabs(LU[r * k1 + c]) > std::fabs(LU[piv * k1 + c])) piv = r;
          if (piv != c)
            for (int j = 0; j < k1; ++j) std::swap(LU[c * k1 + j], LU[piv * k1 + j]);
          det *= LU[c * k1 + c];
          for (int r = c + 1; r < k1; ++r) {
            const double f = LU[r * k1 + c] / LU[c * k1 + c];
            for (int j = c; j < k1; ++j) LU[r * k1 + j] -= f * LU[c * k1 + j];
          }
        }
        det = std::fabs(det);
        std::vector<double> psi(R.nfs), dpsi((size_t)std::max(1, d - 1) * R.nfs), t(d - 1);
        for (int g = 0; g < R.nfp; ++g) {
          for (int r = 0; r < d - 1; ++r) {
            t[r] = T0[r];
            for (int i = 0; i < d - 1; ++i) t[r] += Tm[r * (d - 1) + i] * zf[(size_t)g * (d - 1) + i];
          }
          const size_t fp = ((size_t)fl * R.nsf + sf) * R.nfp + g;
          for (int k = 0; k < d; ++k) {
            double x = W[0][k];
            for (int i = 0; i < d - 1; ++i) x += M[k * (d - 1) + i] * t[i];
            R.fxi[fp * d + k] = x;
          }
          R.fwt[fp] = wf[g] * det;
          tb.eval(t.data(), psi.data(), dpsi.data());
          for (int i = 0; i < R.nfs; ++i) R.ftab[fp * R.nfs + i] = psi[i];
        }
        ++sf;
      }
    }
    if (sf != R.nsf) return MEHDG_ERR_ARG;
  }
  return MEHDG_OK;
}

// Inspection (host only, no device needed): the reference tables above.  counts[0..8] = Np,
// Nfn, nel, ng, nloc, nsf, nfp, nfs (always written); the arrays may be NULL: lattice [Np][d],
// vxi [nel ng][d], vw [nel ng], vtab [nel ng][nloc][d + 1], vnode [nel][nloc], fnodes
// [d + 1][Nfn], fxi [d + 1][nsf nfp][d], fwt [d + 1][nsf nfp].
extern "C" int mehdg_simplex_reference(int d, int m, int p, int* counts, int* lattice, double* vxi, double* vw,
                                       double* vtab, int* vnode, int* fnodes, double* fxi, double* fwt) {
  if (d < 2 || d > 3 || m < 1 || p < 1 || p > 3 || m * p > 12 || !counts) return MEHDG_ERR_ARG;
  SxRef R;
  int rc = sx_reference(d, m, p, R);
  if (rc) return rc;
  counts[0] = R.Np; counts[1] = R.Nfn; counts[2] = R.nel; counts[3] = R.ng;
  counts[4] = R.nloc; counts[5] = R.nsf; counts[6] = R.nfp; counts[7] = R.nfs;
  if (lattice) std::copy(R.lat.begin(), R.lat.end(), lattice);
  if (vxi) std::copy(R.vxi.begin(), R.vxi.end(), vxi);
  if (vw) std::copy(R.vw.begin(), R.vw.end(), vw);
  if (vtab) std::copy(R.vtab.begin(), R.vtab.end(), vtab);
  if (vnode) std::copy(R.vnode.begin(), R.vnode.end(), vnode);
  if (fnodes) std::copy(R.fnodes.begin(), R.fnodes.end(), fnodes);
  if (fxi) std::copy(R.fxi.begin(), R.fxi.end(), fxi);
  if (fwt) std::copy(R.fwt.begin(), R.fwt.end(), fwt);
  return MEHDG_OK;
}

// ---------------------------------------------------------------- mesh and geometry (host)
// Sizes, maps, per-macro geometry and operators of a simplicial box mesh; fills the host
// vectors that setup() uploads (gather, owner, boundary kinds and sides, owner node maps,
// face node table) and sx_host (per-macro M, G_k, Gh_k, M^-1, W_k, Wh_k, Bcat, point geometry,
// node, volume-point and face-point positions).
int sx_maps(mehdg_ctx* ctx, SxRef& R, SxHost& H) {
  const mehdg_problem& pr = ctx->prob;
  const int d = pr.dim, m = pr.m, p = pr.p, n = m * p, nf = d + 1;
  int rc = sx_reference(d, m, p, R);
  if (rc) return ctx_fail(ctx, rc, "simplex reference tables");
  const int Np = R.Np, Nfn = R.Nfn, ns = ctx->ns;
  ctx->Np = Np;
  ctx->Nfn = Nfn;
  ctx->nf = nf;
  ctx->Nth = nf * Nfn;
  ctx->Nu = ns * Np;
  ctx->Nq = d * ctx->Nu;
  ctx->Nt = ns * ctx->Nth;
  ctx->nel = R.nel;
  ctx->Ng = R.ng;
  ctx->nloc = R.nloc;
  ctx->nsf = R.nsf;
  ctx->nfp = R.nfp;
  ctx->nfs = R.nfs;
  const int Nth = ctx->Nth, Nt = ctx->Nt;
  int nperm = 1;
  for (int k = 2; k <= d; ++k) nperm *= k;
  int ncell = 1, N[3] = {0, 0, 0};
  double Hc[3] = {1.0, 1.0, 1.0}, hmin = 1e300;
  for (int k = 0; k < d; ++k) {
    ncell *= pr.nmac[k];
    N[k] = pr.nmac[k] * n;
    Hc[k] = (pr.hi[k] - pr.lo[k]) / pr.nmac[k];
    hmin = std::min(hmin, Hc[k]);
  }
  for (int k = 0; k < 3; ++k) { ctx->hm[k] = Hc[k]; ctx->he[k] = Hc[k] / m; }
  ctx->h_supg = hmin / m;
  const int E = ncell * nperm;
  ctx->E = E;
  std::vector<std::vector<int>> perms;
  {
    std::vector<int> pm(d);
    for (int k = 0; k < d; ++k) pm[k] = k;
    do perms.push_back(pm); while (std::next_permutation(pm.begin(), pm.end()));
  }
  // integer lattice coordinates (spacing H / n) of every macro node
  std::vector<int> cellof(E * 3, 0), sigof(E);
  std::vector<long long> ilat((size_t)E * Np * d);
  for (int e = 0; e < E; ++e) {
    int c = e / nperm, s = e % nperm;
    sigof[e] = s;
    for (int k = 0; k < d; ++k) { cellof[e * 3 + k] = c % pr.nmac[k]; c /= pr.nmac[k]; }
    const std::vector<int>& sg = perms[s];
    for (int a = 0; a < Np; ++a)
      for (int k = 0; k < d; ++k)
        ilat[((size_t)e * Np + a) * d + sg[k]] = (long long)cellof[e * 3 + sg[k]] * n + R.lat[(size_t)a * d + k];
  }
  auto wrapped = [&](int e, int a, int k) {
    long long v = ilat[((size_t)e * Np + a) * d + k];
    if (pr.periodic[k]) v = ((v % N[k]) + N[k]) % N[k];
    return v;
  };
  // faces by their wrapped node sets; owners; node maps
  std::map<std::vector<long long>, int> keys;
  std::vector<std::vector<int>> owners;
  std::vector<int> fid((size_t)E * nf);
  for (int e = 0; e < E; ++e)
    for (int fl = 0; fl < nf; ++fl) {
      std::vector<std::vector<long long>> pts;
      for (int j = 0; j < Nfn; ++j) {
        std::vector<long long> x(d);
        for (int k = 0; k < d; ++k) x[k] = wrapped(e, R.fnodes[(size_t)fl * Nfn + j], k);
        pts.push_back(x);
      }
      std::sort(pts.begin(), pts.end());
      std::vector<long long> key;
      for (auto& x : pts) key.insert(key.end(), x.begin(), x.end());
      auto it = keys.find(key);
      int f;
      if (it == keys.end()) {
        f = (int)owners.size();
        keys[key] = f;
        owners.push_back({});
      } else {
        f = it->second;
      }
      if (owners[f].size() >= 2) return ctx_fail(ctx, MEHDG_ERR_ARG, "face with more than two owners");
      owners[f].push_back(e * nf + fl);
      fid[(size_t)e * nf + fl] = f;
    }
  const int F = (int)owners.size();
  ctx->F = F;
  ctx->ntr = (long long)F * ns * Nfn;
  ctx->h_gather.assign((size_t)E * Nt, 0);
  ctx->h_owner.assign(2 * (size_t)F, -1);
  ctx->h_bkind.assign((size_t)E * nf, 0);
  ctx->h_bside.assign((size_t)E * nf, -1);
  ctx->h_ofn.assign((size_t)2 * F * Nfn, 0);
  for (int f = 0; f < F; ++f) {
    const int o0 = owners[f][0], e0 = o0 / nf, f0 = o0 % nf;
    ctx->h_owner[2 * f] = o0;
    for (int j = 0; j < Nfn; ++j) ctx->h_ofn[(size_t)2 * f * Nfn + j] = j;
    if (owners[f].size() == 2) {
      const int o1 = owners[f][1], e1 = o1 / nf, f1 = o1 % nf;
      ctx->h_owner[2 * f + 1] = o1;
      std::map<std::vector<long long>, int> loc;
      for (int l = 0; l < Nfn; ++l) {
        std::vector<long long> x(d);
        for (int k = 0; k < d; ++k) x[k] = wrapped(e1, R.fnodes[(size_t)f1 * Nfn + l], k);
        loc[x] = l;
      }
      for (int j = 0; j < Nfn; ++j) {
        std::vector<long long> x(d);
        for (int k = 0; k < d; ++k) x[k] = wrapped(e0, R.fnodes[(size_t)f0 * Nfn + j], k);
        auto it = loc.find(x);
        if (it == loc.end()) return ctx_fail(ctx, MEHDG_ERR_ARG, "face nodes of two owners do not match");
        ctx->h_ofn[((size_t)2 * f + 1) * Nfn + j] = it->second;
      }
    }
    for (size_t o = 0; o < owners[f].size(); ++o) {
      const int e = owners[f][o] / nf, fl = owners[f][o] % nf;
      std::vector<int> loc2glob(Nfn);
      for (int j = 0; j < Nfn; ++j) loc2glob[ctx->h_ofn[((size_t)2 * f + o) * Nfn + j]] = j;
      for (int s = 0; s < ns; ++s)
        for (int l = 0; l < Nfn; ++l)
          ctx->h_gather[(size_t)e * Nt + (size_t)s * Nth + fl * Nfn + l] = (f * ns + s) * Nfn + loc2glob[l];
      // boundary side: all nodes on a non-periodic boundary plane
      int bs = -1;
      for (int k = 0; k < d; ++k) {
        if (pr.periodic[k]) continue;
        bool lo = true, hi = true;
        for (int j = 0; j < Nfn; ++j) {
          const long long v = ilat[((size_t)e * Np + R.fnodes[(size_t)fl * Nfn + j]) * d + k];
          lo = lo && v == 0;
          hi = hi && v == N[k];
        }
        if (lo) bs = 2 * k;
        else if (hi) bs = 2 * k + 1;
      }
      if ((bs >= 0) != (owners[f].size() == 1))
        return ctx_fail(ctx, MEHDG_ERR_ARG, "simplex mesh: boundary faces and single owners disagree");
      ctx->h_bside[(size_t)e * nf + fl] = bs;
      ctx->h_bkind[(size_t)e * nf + fl] = bs >= 0 ? pr.bc[bs] : 0;
      if (bs >= 0 && pr.bc[bs] == MEHDG_BC_NONE)
        return ctx_fail(ctx, MEHDG_ERR_ARG, "boundary side without boundary condition");
    }
  }
  ctx->facenode.assign(R.fnodes.begin(), R.fnodes.end());

  // per-macro geometry: x = x0 + J xi, J[sigma_k][k] = H_sigma_k
  const int G = R.nel * R.ng, GF = R.nsf * R.nfp;
  H.vgeo.assign((size_t)E * G * (d * d + 1), 0.0);
  H.fgeo.assign((size_t)E * nf * GF * (d + 1), 0.0);
  H.xnode.assign((size_t)E * d * Np, 0.0);
  H.xq.assign((size_t)E * G * d, 0.0);
  H.xf.assign((size_t)E * nf * GF * d, 0.0);
  H.M.assign((size_t)E * Np * Np, 0.0);
  H.Minv.assign((size_t)E * Np * Np, 0.0);
  H.Gk.assign((size_t)E * d * Np * Np, 0.0);
  H.Ghk.assign((size_t)E * d * Np * Nth, 0.0);
  H.Wk.assign((size_t)E * d * Np * Np, 0.0);
  H.Whk.assign((size_t)E * d * Np * Nth, 0.0);
  H.Bcat.assign((size_t)E * d * Np * (Np + Nth), 0.0);
  std::vector<double> J(d * d), Ji(d * d), dphys((size_t)d * R.nloc);
  for (int e = 0; e < E; ++e) {
    const std::vector<int>& sg = perms[sigof[e]];
    double x0[3], detJ = 1.0;
    std::fill(J.begin(), J.end(), 0.0);
    std::fill(Ji.begin(), Ji.end(), 0.0);
    for (int k = 0; k < d; ++k) {
      x0[k] = pr.lo[k] + Hc[k] * cellof[e * 3 + k];
      J[sg[k] * d + k] = Hc[sg[k]];
      Ji[k * d + sg[k]] = 1.0 / Hc[sg[k]];   // dxi_k / dx_sigma_k
      detJ *= Hc[sg[k]];
    }
    for (int a = 0; a < Np; ++a)
      for (int i = 0; i < d; ++i) {
        double x = x0[i];
        for (int k = 0; k < d; ++k) x += J[i * d + k] * (double)R.lat[(size_t)a * d + k] / n;
        H.xnode[((size_t)e * d + i) * Np + a] = x;
      }
    double* Me = &H.M[(size_t)e * Np * Np];
    double* Ge = &H.Gk[(size_t)e * d * Np * Np];
    double* Ghe = &H.Ghk[(size_t)e * d * Np * Nth];
    for (int el = 0; el < R.nel; ++el)
      for (int g = 0; g < R.ng; ++g) {
        const size_t pt = (size_t)el * R.ng + g;
        const double w = R.vw[pt] * detJ;
        double* vg = &H.vgeo[((size_t)e * G + pt) * (d * d + 1)];
        for (int j = 0; j < d * d; ++j) vg[j] = Ji[j];
        vg[d * d] = w;
        for (int i = 0; i < d; ++i) {
          double x = x0[i];
          for (int k = 0; k < d; ++k) x += J[i * d + k] * R.vxi[pt * d + k];
          H.xq[((size_t)e * G + pt) * d + i] = x;
        }
        const double* T = &R.vtab[pt * R.nloc * (d + 1)];
        const int* nd = &R.vnode[(size_t)el * R.nloc];
        for (int al = 0; al < R.nloc; ++al)
          for (int k = 0; k < d; ++k) {
            double v = 0.0;
            for (int j = 0; j < d; ++j) v += Ji[j * d + k] * T[al * (d + 1) + 1 + j];
            dphys[(size_t)k * R.nloc + al] = v;
          }
        for (int ai = 0; ai < R.nloc; ++ai)
          for (int bi = 0; bi < R.nloc; ++bi) {
            const int a = nd[ai], b = nd[bi];
            Me[(size_t)a * Np + b] += w * T[ai * (d + 1)] * T[bi * (d + 1)];
            for (int k = 0; k < d; ++k)
              Ge[((size_t)k * Np + a) * Np + b] += w * dphys[(size_t)k * R.nloc + ai] * T[bi * (d + 1)];
          }
      }
    for (int fl = 0; fl < nf; ++fl) {
      // physical unit normal Ji^T nref / |.| and area factor sqrt(det((J M)^T (J M)))
      double nn[3] = {0.0, 0.0, 0.0}, nrm = 0.0;
      for (int k = 0; k < d; ++k) {
        for (int j = 0; j < d; ++j) nn[k] += Ji[j * d + k] * R.nref[(size_t)fl * d + j];
        nrm += nn[k] * nn[k];
      }
      nrm = std::sqrt(nrm);
      for (int k = 0; k < d; ++k) nn[k] /= nrm;
      const double* M = &R.fM[(size_t)fl * d * (d - 1)];
      std::vector<double> JM((size_t)d * (d - 1), 0.0), Gm((size_t)(d - 1) * (d - 1), 0.0);
      for (int i = 0; i < d; ++i)
        for (int c = 0; c < d - 1; ++c)
          for (int k = 0; k < d; ++k) JM[i * (d - 1) + c] += J[i * d + k] * M[k * (d - 1) + c];
      for (int a = 0; a < d - 1; ++a)
        for (int b = 0; b < d - 1; ++b)
          for (int i = 0; i < d; ++i) Gm[a * (d - 1) + b] += JM[i * (d - 1) + a] * JM[i * (d - 1) + b];
      const double area = (d == 2) ? std::sqrt(Gm[0]) : std::sqrt(std::fabs(Gm[0] * Gm[3] - Gm[1] * Gm[2]));
      for (int sf = 0; sf < R.nsf; ++sf)
        for (int g = 0; g < R.nfp; ++g) {
          const size_t fp = ((size_t)fl * R.nsf + sf) * R.nfp + g;
          const double w = R.fwt[fp] * area;
          double* fg = &H.fgeo[(((size_t)e * nf + fl) * GF + (size_t)sf * R.nfp + g) * (d + 1)];
          for (int k = 0; k < d; ++k) fg[k] = nn[k];
          fg[d] = w;
          for (int i = 0; i < d; ++i) {
            double x = x0[i];
            for (int k = 0; k < d; ++k) x += J[i * d + k] * R.fxi[fp * d + k];
            H.xf[(((size_t)e * nf + fl) * GF + (size_t)sf * R.nfp + g) * d + i] = x;
          }
          const double* psi = &R.ftab[fp * R.nfs];
          const int* sfn = &R.fsub[((size_t)fl * R.nsf + sf) * R.nfs];
          for (int i = 0; i < R.nfs; ++i)
            for (int j = 0; j < R.nfs; ++j) {
              const int a = R.fnodes[(size_t)fl * Nfn + sfn[i]];   // volume basis on the face = trace basis
              const double v = w * psi[i] * psi[j];
              for (int k = 0; k < d; ++k) Ghe[((size_t)k * Np + a) * Nth + fl * Nfn + sfn[j]] -= nn[k] * v;
            }
        }
    }
    // M^-1, W_k = M^-1 G_k, Wh_k = M^-1 Gh_k, Bcat = [W_k | -Wh_k]
    std::vector<double> Mi(Me, Me + (size_t)Np * Np);
    invert(Mi, Np);
    std::copy(Mi.begin(), Mi.end(), H.Minv.begin() + (size_t)e * Np * Np);
    const int nb = Np + Nth;
    for (int k = 0; k < d; ++k)
      for (int a = 0; a < Np; ++a) {
        double* wrow = &H.Wk[(((size_t)e * d + k) * Np + a) * Np];
        double* whrow = &H.Whk[(((size_t)e * d + k) * Np + a) * Nth];
        for (int c = 0; c < Np; ++c) {
          const double f = Mi[(size_t)a * Np + c];
          if (f == 0.0) continue;
          const double* gr = &Ge[((size_t)k * Np + c) * Np];
          const double* ghr = &Ghe[((size_t)k * Np + c) * Nth];
          for (int b = 0; b < Np; ++b) wrow[b] += f * gr[b];
          for (int i = 0; i < Nth; ++i) whrow[i] += f * ghr[i];
        }
        double* brow = &H.Bcat[(size_t)e * d * Np * nb + ((size_t)k * Np + a) * nb];
        for (int b = 0; b < Np; ++b) brow[b] = wrow[b];
        for (int i = 0; i < Nth; ++i) brow[Np + i] = -whrow[i];
      }
  }
  return MEHDG_OK;
}

// ---------------------------------------------------------------- closed-form data at points
namespace {


// source f = div (F + G) of the closed form at the volume points x [n][D]
template <int D>
__global__ void k_sx_source(long long n, mehdg_problem pr, const double* __restrict__ x, double* __restrict__ src) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  closed_form_source<D>(pr.field == MEHDG_FIELD_COUETTE3D, pr.field_par, pr.gamma, pr.Re, pr.Pr, x + i * D,
                        src + i * (D + 2));
}

// boundary data at the face points x [E][nf][per_f][D]: the closed form on Dirichlet faces, the
// free stream on far-field faces, zero elsewhere
template <int D>
__global__ void k_sx_bdata(long long n, int per_f, mehdg_problem pr, const int* __restrict__ bkind,
                           const double* __restrict__ x, double* __restrict__ uD) {
  constexpr int NS = D + 2;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int bk = bkind[i / per_f];
  double* out = uD + i * NS;
  if (bk == MEHDG_BC_DIRICHLET) closed_form_state<D>(pr.field, pr.field_par, pr.gamma, x + i * D, out);
  else if (bk == MEHDG_BC_FARFIELD) field_uniform<D>(pr.field_par, pr.gamma, out);
  else
    for (int s = 0; s < NS; ++s) out[s] = 0.0;
}

// u at the macro nodes from the closed form (+ du)
template <int D>
__global__ void k_sx_init(long long n, int Np, mehdg_problem pr, const double* __restrict__ xnode,
                          const double* __restrict__ du, double* __restrict__ u) {
  constexpr int NS = D + 2;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = (int)(i % Np);
  const long long e = i / Np;
  double x[D], uu[NS];
  for (int k = 0; k < D; ++k) x[k] = xnode[(e * D + k) * Np + a];
  closed_form_state<D>(pr.field, pr.field_par, pr.gamma, x, uu);
  for (int s = 0; s < NS; ++s) {
    const size_t o = ((size_t)e * NS + s) * Np + a;
    u[o] = uu[s] + (du ? du[o] : 0.0);
  }
}

}  // namespace

int sx_source(mehdg_ctx* ctx, const double* xq, long long n, double* src) {
  const unsigned b = (unsigned)((n + 127) / 128);
  if (ctx->d == 2) k_sx_source<2><<<b, 128, 0, ctx->stream>>>(n, ctx->prob, xq, src);
  else k_sx_source<3><<<b, 128, 0, ctx->stream>>>(n, ctx->prob, xq, src);
  CKL();
  return MEHDG_OK;
}

int sx_bdata(mehdg_ctx* ctx, const double* xf, long long n, int per_f, double* uD) {
  const unsigned b = (unsigned)((n + 127) / 128);
  if (ctx->d == 2) k_sx_bdata<2><<<b, 128, 0, ctx->stream>>>(n, per_f, ctx->prob, ctx->bkind, xf, uD);
  else k_sx_bdata<3><<<b, 128, 0, ctx->stream>>>(n, per_f, ctx->prob, ctx->bkind, xf, uD);
  CKL();
  return MEHDG_OK;
}

int sx_init_state(mehdg_ctx* ctx, const double* du, double* u) {
  const long long n = (long long)ctx->E * ctx->Np;
  const unsigned b = (unsigned)((n + 127) / 128);
  if (ctx->d == 2) k_sx_init<2><<<b, 128, 0, ctx->stream>>>(n, ctx->Np, ctx->prob, ctx->xnode, du, u);
  else k_sx_init<3><<<b, 128, 0, ctx->stream>>>(n, ctx->Np, ctx->prob, ctx->xnode, du, u);
  CKL();
  return MEHDG_OK;
}

// Inspection (host only, no device needed): the maps and per-macro operators of a simplicial
// mesh.  counts (host int[5], required): E, F, Np, Nfn, Nth; the other host arrays may be NULL:
// gather [E][Nt], owner [F][2] (e (d + 1) + local face, -1 for none), bside [E][d + 1],
// M [E][Np][Np], Gk [E][d][Np][Np], Ghk [E][d][Np][Nth], xnode [E][d][Np].
extern "C" int mehdg_simplex_mesh(const mehdg_problem* prob, int* counts, int* gather, int* owner, int* bside,
                                  double* M, double* Gk, double* Ghk, double* xnode) {
  if (!prob || !counts || prob->dim < 2 || prob->dim > 3 || prob->m < 1 || prob->p < 1 || prob->p > 3 ||
      prob->m * prob->p > 6)
    return MEHDG_ERR_ARG;
  for (int k = 0; k < prob->dim; ++k)
    if (prob->nmac[k] < 1 || !(prob->hi[k] > prob->lo[k])) return MEHDG_ERR_ARG;
  mehdg_ctx* ctx = new mehdg_ctx();
  ctx->prob = *prob;
  ctx->d = prob->dim;
  ctx->ns = prob->dim + 2;
  ctx->m = prob->m;
  ctx->p = prob->p;
  SxRef R;
  SxHost H;
  int rc = sx_maps(ctx, R, H);
  if (rc == MEHDG_OK) {
    counts[0] = ctx->E; counts[1] = ctx->F; counts[2] = ctx->Np; counts[3] = ctx->Nfn; counts[4] = ctx->Nth;
    if (gather) std::copy(ctx->h_gather.begin(), ctx->h_gather.end(), gather);
    if (owner) std::copy(ctx->h_owner.begin(), ctx->h_owner.end(), owner);
    if (bside) std::copy(ctx->h_bside.begin(), ctx->h_bside.end(), bside);
    if (M) std::copy(H.M.begin(), H.M.end(), M);
    if (Gk) std::copy(H.Gk.begin(), H.Gk.end(), Gk);
    if (Ghk) std::copy(H.Ghk.begin(), H.Ghk.end(), Ghk);
    if (xnode) std::copy(H.xnode.begin(), H.xnode.end(), xnode);
  }
  delete ctx;
  return rc;
}
