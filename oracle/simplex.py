"""Simplicial macro-elements (Sec. 2.2): P_p on m-refined simplices, and a box mesh of them.

Test infrastructure only (see ``oracle/__init__``).

Reference macro-element: the Kuhn simplex K = {1 >= xi_1 >= xi_2 >= ... >= xi_d >= 0}.
Refining it m times (the Freudenthal subdivision of the m-grid of [0, 1]^d restricted to K)
gives m^d sub-simplices, each a translated, axis-permuted copy of K / m.  On each the space is
P_p with equispaced Lagrange nodes; the nodes of all sub-simplices are the lattice points
a / (m p), m p >= a_1 >= ... >= a_d >= 0, so the macro space is continuous (C(m p + d, d)
nodes).  The d + 1 faces of K, in this order: xi_1 = 1, xi_k = xi_{k+1} (k = 1 .. d - 1),
xi_d = 0; the trace space on each face is continuous P_p on its m^(d-1) sub-faces
(C(m p + d - 1, d - 1) nodes, the face's lattice points), independent across faces.

Quadrature: on every sub-simplex and sub-face, the collapsed (Duffy) Gauss-Legendre rule
with p + 3 points per direction (exact for total degree 2 p + 6 - d on a d-simplex).

Mesh: each cell of a box grid is split into d! macro-elements x = C + H P_sigma xi, one per
permutation sigma of the axes (the Kuhn triangulation, conforming across cells).  Faces are
numbered in order of first appearance over (macro, local face); a face's nodes are in its
first owner's order, the second owner's nodes matched by position (periodic axes wrapped).
Boundary sides 2k / 2k + 1 are the planes x_k = lo_k / hi_k as on box meshes.
"""
import itertools

import numpy as np
from numpy.polynomial.legendre import leggauss


def kuhn_lattice(d, n):
    """Integer points a with n >= a_1 >= ... >= a_d >= 0, in lexicographic order."""
    return np.array([a for a in itertools.product(range(n + 1), repeat=d)
                     if all(a[i] >= a[i + 1] for i in range(d - 1))], dtype=np.int64).reshape(-1, d)


def simplex_rule(d, n):
    """Collapsed Gauss-Legendre rule on the unit simplex {z >= 0, sum z <= 1}: z_k = s_k
    prod_{i<k} (1 - s_i), weight prod_k w_k prod_{i<k} (1 - s_i); exact for total degree
    <= 2 n - d.  Returns points [Q, d] and weights [Q]."""
    if d == 0:
        return np.zeros((1, 0)), np.ones(1)
    g, w = leggauss(n)
    s, ws = (g + 1.0) / 2.0, w / 2.0
    pts, wts = [], []
    for idx in itertools.product(range(n), repeat=d):
        z, rem, wt = [], 1.0, 1.0
        for i in idx:
            z.append(s[i] * rem)
            wt *= ws[i] * rem
            rem *= 1.0 - s[i]
        pts.append(z)
        wts.append(wt)
    return np.array(pts), np.array(wts)


def monomials(d, p):
    """Exponents alpha with |alpha| <= p."""
    return [a for a in itertools.product(range(p + 1), repeat=d) if sum(a) <= p]


def _mono_vals(y, alphas):
    """Monomials and their derivatives at points y [Q, d]: V [Q, nm], dV [d, Q, nm]."""
    y = np.atleast_2d(y)
    Q, d = y.shape
    V = np.ones((Q, len(alphas)))
    dV = np.zeros((d, Q, len(alphas)))
    for j, a in enumerate(alphas):
        for k in range(d):
            V[:, j] *= y[:, k] ** a[k]
        for l in range(d):
            if a[l] == 0:
                continue
            t = a[l] * y[:, l] ** (a[l] - 1)
            for k in range(d):
                if k != l:
                    t = t * y[:, k] ** a[k]
            dV[l, :, j] = t
    return V, dV


class Lagrange:
    """Lagrange basis of P_p on the given nodes (in coordinates y, dimension dy)."""

    def __init__(self, nodes, p):
        nodes = np.atleast_2d(np.asarray(nodes, dtype=float))
        self.alphas = monomials(nodes.shape[1], p)
        V, _ = _mono_vals(nodes, self.alphas)
        if V.shape[0] != V.shape[1]:
            raise ValueError("node count does not match dim P_p")
        self.C = np.linalg.inv(V)                     # phi_i(y) = sum_j mono_j(y) C[j, i]

    def __call__(self, y):
        V, dV = _mono_vals(y, self.alphas)
        return V @ self.C, np.array([D @ self.C for D in dV])   # [Q, n], [dy, Q, n]


class KuhnMacro:
    """Reference tables of the m-refined Kuhn macro-element with P_p sub-elements
    (tables=False: the node lattice, the sub-simplices and the face node lists only)."""

    def __init__(self, d, m, p, tables=True):
        self.d, self.m, self.p = d, m, p
        n = m * p
        self.lat = kuhn_lattice(d, n)                       # [Np, d] integer node coordinates
        self.Np = len(self.lat)
        index = {tuple(a): i for i, a in enumerate(self.lat)}
        self.xn = self.lat / float(n)                       # [Np, d] node positions in K
        nq = p + 3
        zr, wr = simplex_rule(d, nq)
        # sub-simplices (c, pi): cell c non-increasing, ties of c ordered by axis in pi
        self.subs = []
        for c in itertools.product(range(m), repeat=d):
            if any(c[i] < c[i + 1] for i in range(d - 1)):
                continue
            for pi in itertools.permutations(range(d)):
                pos = {ax: r for r, ax in enumerate(pi)}
                if any(c[i] == c[i + 1] and pos[i] > pos[i + 1] for i in range(d - 1)):
                    continue
                verts = [np.array(c, dtype=np.int64)]
                for k in range(d):
                    v = verts[-1].copy()
                    v[pi[k]] += 1
                    verts.append(v)
                loc = [b for b in itertools.product(range(p + 1), repeat=d)
                       if all(b[pi[k]] >= b[pi[k + 1]] for k in range(d - 1))]
                nodes = [index[tuple(np.array(c) * p + np.array(b))] for b in loc]
                basis = Lagrange(np.array(loc, dtype=float) / p, p) if tables else None
                self.subs.append(dict(c=np.array(c), pi=pi, verts=np.array(verts), nodes=np.array(nodes),
                                      basis=basis))
        if len(self.subs) != m ** d:
            raise ValueError("subdivision count")
        if not tables:
            self.face_nodes = []
            for fl in range(d + 1):
                on_node, _ = self._face_eq(fl)
                self.face_nodes.append(np.array([i for i, a in enumerate(self.lat) if on_node(a)], dtype=np.int64))
            self.Nfn = len(self.face_nodes[0])
            return
        # volume quadrature: y[pi_j] = sum_{k >= j} z_k maps the unit simplex onto the cell's Kuhn
        # simplex (det 1); xi = (c + y) / m
        xq, wq, B0, Bd = [], [], [], []
        for sb in self.subs:
            y = np.zeros_like(zr)
            for j in range(d):
                y[:, sb["pi"][j]] = zr[:, j:].sum(axis=1)
            phi, dphi = sb["basis"](y)
            Q = len(wr)
            b0 = np.zeros((Q, self.Np))
            bd = np.zeros((d, Q, self.Np))
            b0[:, sb["nodes"]] = phi
            bd[:, :, sb["nodes"]] = dphi * m                 # d/dxi = m d/dy
            xq.append((sb["c"][None, :] + y) / m)
            wq.append(wr / m ** d)
            B0.append(b0)
            Bd.append(bd)
        self.xq = np.vstack(xq).T                             # [d, G]
        self.wq = np.concatenate(wq)
        self.B0 = np.vstack(B0)                               # [G, Np]
        self.Bd = np.concatenate(Bd, axis=1)                  # [d, G, Np]
        # faces
        P = [np.array([1.0] * j + [0.0] * (d - j)) for j in range(d + 1)]   # vertices of K
        self.faces = []
        for fl in range(d + 1):
            on_node, nref = self._face_eq(fl)
            fverts = [P[j] for j in range(d + 1) if j != fl]              # face fl is opposite P_fl
            W0 = fverts[0]
            M = np.array([v - W0 for v in fverts[1:]]).T                   # [d, d-1]
            fnodes = np.array([i for i, a in enumerate(self.lat) if on_node(a)], dtype=np.int64)
            fpos = {int(i): r for r, i in enumerate(fnodes)}

            def tcoord(xi):
                return np.linalg.lstsq(M, np.atleast_2d(xi).T - W0[:, None], rcond=None)[0].T   # [Q, d-1]

            zf, wf = simplex_rule(d - 1, nq)
            fx, fw, fphi, fpsi = [], [], [], []
            for sb in self.subs:
                vxi = sb["verts"] / float(m)
                for drop in range(d + 1):
                    sv = [vxi[i] for i in range(d + 1) if i != drop]
                    if not all(on_node(v * n) for v in sv):
                        continue
                    # the sub-face: nodes of the sub-simplex on the face, trace basis in face coordinates t
                    snodes = [i for i in sb["nodes"] if on_node(self.lat[i])]
                    tn = tcoord(self.xn[snodes])
                    tb = Lagrange(tn, p)
                    T0 = tcoord(sv[0])[0]
                    Tm = np.array([tcoord(v)[0] - T0 for v in sv[1:]]).T if d > 1 else np.zeros((0, 0))
                    t = T0[None, :] + zf @ Tm.T if d > 1 else np.zeros((1, 0))
                    jac = abs(np.linalg.det(Tm)) if d > 1 else 1.0
                    xi = W0[None, :] + t @ M.T
                    y = xi * m - sb["c"][None, :]
                    phi_loc, _ = sb["basis"](y)
                    ph = np.zeros((len(xi), self.Np))
                    ph[:, sb["nodes"]] = phi_loc
                    psi_loc, _ = tb(t) if d > 1 else (np.ones((1, 1)), None)
                    ps = np.zeros((len(xi), len(fnodes)))
                    ps[:, [fpos[int(i)] for i in snodes]] = psi_loc
                    fx.append(xi)
                    fw.append(wf * jac)
                    fphi.append(ph)
                    fpsi.append(ps)
            self.faces.append(dict(nodes=fnodes, M=M, W0=W0, nref=nref, xi=np.vstack(fx).T, wt=np.concatenate(fw),
                                   phi=np.vstack(fphi), psi=np.vstack(fpsi)))
        self.Nfn = len(self.faces[0]["nodes"])
        if len(self.faces[0]["wt"]) != m ** (d - 1) * len(zf):
            raise ValueError("sub-face count")

    def _face_eq(self, fl):
        """Node test (on integer lattice coordinates) and unit outward normal of face fl."""
        d, n = self.d, self.m * self.p
        if fl == 0:
            nref = np.zeros(d)
            nref[0] = 1.0
            return (lambda a: abs(a[0] - n) < 1e-9), nref
        if fl == d:
            nref = np.zeros(d)
            nref[d - 1] = -1.0
            return (lambda a: abs(a[d - 1]) < 1e-9), nref
        nref = np.zeros(d)
        nref[fl - 1], nref[fl] = -1.0, 1.0
        return (lambda a, k=fl: abs(a[k - 1] - a[k]) < 1e-9), nref / np.sqrt(2.0)


_REF = {}


def kuhn_macro(d, m, p):
    key = (d, m, p)
    if key not in _REF:
        _REF[key] = KuhnMacro(d, m, p)
    return _REF[key]


class SimplexMacroGeometry:
    """Basis values, weights and faces of the affine macro-element x = x0 + J xi, xi in K.
    Same attributes as space.MacroGeometry (faces hold a constant unit normal n)."""

    def __init__(self, ref, x0, J, h):
        d = ref.d
        self.d, self.m, self.p = d, ref.m, ref.p
        self.Np, self.Nfn = ref.Np, ref.Nfn
        self.Nth = (d + 1) * ref.Nfn
        self.h = h
        J = np.asarray(J, dtype=float)
        x0 = np.asarray(x0, dtype=float)
        Ji = np.linalg.inv(J)                                  # Ji[j, k] = dxi_j / dx_k
        det = abs(np.linalg.det(J))
        T = [ref.B0]
        for k in range(d):
            T.append(sum(Ji[j, k] * ref.Bd[j] for j in range(d)))
        self.T = np.array(T)
        self.w = ref.wq * det
        self.xq = x0[:, None] + J @ ref.xq
        self.xn = x0[:, None] + J @ ref.xn.T
        self.faces = []
        for fc in ref.faces:
            nn = Ji.T @ fc["nref"]
            JM = J @ fc["M"]
            area = np.sqrt(abs(np.linalg.det(JM.T @ JM))) if d > 1 else 1.0
            self.faces.append(dict(phi=fc["phi"], psi=fc["psi"], w=fc["wt"] * area, n=nn / np.linalg.norm(nn),
                                   x=x0[:, None] + J @ fc["xi"]))


class SimplexBoxMesh:
    """Kuhn triangulation of a box grid into simplicial macro-elements (module docstring).
    Macro e = cell * d! + (index of sigma in itertools.permutations order); cell index with
    axis 0 fastest."""

    def __init__(self, prob):
        d = prob["dim"]
        self.d = d
        self.nm = [int(x) for x in prob["nmac"][:d]]
        self.lo = np.array(prob["lo"][:d], dtype=float)
        self.hi = np.array(prob["hi"][:d], dtype=float)
        self.per = [bool(x) for x in prob["periodic"][:d]]
        self.m, self.p = prob["m"], prob["p"]
        self.ref = kuhn_macro(d, self.m, self.p)
        self.H = (self.hi - self.lo) / np.array(self.nm)
        self.perms = list(itertools.permutations(range(d)))
        ncell = int(np.prod(self.nm))
        self.E = ncell * len(self.perms)
        self.Nfn = self.ref.Nfn
        self.fnodes = [fc["nodes"] for fc in self.ref.faces]
        n = self.m * self.p
        self.N = [self.nm[k] * n for k in range(d)]         # lattice extent per axis
        # integer lattice coordinates of every macro node
        self.ilat = np.zeros((self.E, self.ref.Np, d), dtype=np.int64)
        for e in range(self.E):
            cell, sig = self.macro_cell(e)
            P = self._P(sig)
            self.ilat[e] = np.array(cell)[None, :] * n + self.ref.lat @ P.T
        # faces matched by their wrapped node sets
        keys = {}
        self.owners = []
        self.fid = np.zeros((self.E, d + 1), dtype=np.int64)
        for e in range(self.E):
            for fl in range(d + 1):
                pts = self._wrap(self.ilat[e][self.fnodes[fl]])
                key = tuple(sorted(map(tuple, pts.tolist())))
                if key not in keys:
                    keys[key] = len(self.owners)
                    self.owners.append([])
                f = keys[key]
                if len(self.owners[f]) == 2:
                    raise ValueError("face with more than two owners")
                self.owners[f].append((e, fl))
                self.fid[e, fl] = f
        self.F = len(self.owners)
        # node permutation of each owner: global face node g <- local face node perm[g]
        self.perm = np.zeros((self.E, d + 1, self.Nfn), dtype=np.int64)
        for f, own in enumerate(self.owners):
            e0, f0 = own[0]
            p0 = [tuple(x) for x in self._wrap(self.ilat[e0][self.fnodes[f0]]).tolist()]
            self.perm[e0, f0] = np.arange(self.Nfn)
            for (e1, f1) in own[1:]:
                p1 = {tuple(x): i for i, x in enumerate(self._wrap(self.ilat[e1][self.fnodes[f1]]).tolist())}
                self.perm[e1, f1] = [p1[x] for x in p0]

    def _P(self, sig):
        """x_{sigma_k} = C_{sigma_k} + H xi_k: P[sigma_k, k] = 1."""
        P = np.zeros((self.d, self.d), dtype=np.int64)
        for k, ax in enumerate(sig):
            P[ax, k] = 1
        return P

    def _wrap(self, pts):
        pts = np.array(pts)
        for k in range(self.d):
            if self.per[k]:
                pts[:, k] %= self.N[k]
        return pts

    def macro_cell(self, e):
        nperm = len(self.perms)
        c, s = divmod(e, nperm)
        cell = []
        for k in range(self.d):
            cell.append(c % self.nm[k])
            c //= self.nm[k]
        return cell, self.perms[s]

    def macro_map(self, e):
        """x0 and J of macro e (x = x0 + J xi)."""
        cell, sig = self.macro_cell(e)
        x0 = self.lo + self.H * np.array(cell)
        J = self._P(sig) * self.H[:, None]
        return x0, J

    def macro_faces(self, e):
        """Global face id and boundary side (or -1) of the local faces."""
        out = []
        for fl in range(self.d + 1):
            pts = self.ilat[e][self.fnodes[fl]]
            bside = -1
            for k in range(self.d):
                if self.per[k]:
                    continue
                if np.all(pts[:, k] == 0):
                    bside = 2 * k
                elif np.all(pts[:, k] == self.N[k]):
                    bside = 2 * k + 1
            out.append((int(self.fid[e, fl]), bside))
        return out

    def gather_map(self, e, ns):
        g = np.zeros((ns, (self.d + 1) * self.Nfn), dtype=np.int64)
        for fl in range(self.d + 1):
            f = int(self.fid[e, fl])
            inv = np.empty(self.Nfn, dtype=np.int64)
            inv[self.perm[e, fl]] = np.arange(self.Nfn)
            for s in range(ns):
                g[s, fl * self.Nfn:(fl + 1) * self.Nfn] = (f * ns + s) * self.Nfn + inv
        return g

    def face_owners(self):
        return [list(o) for o in self.owners]

    def geometry(self, e):
        x0, J = self.macro_map(e)
        return SimplexMacroGeometry(self.ref, x0, J, float(np.min(self.H)) / self.m)
