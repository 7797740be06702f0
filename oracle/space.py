"""Discrete spaces on box macro-elements and the global trace numbering.

Test infrastructure only (see ``oracle/__init__``).

Spaces (Sec. 2.2):
  * each macro-element is a box split into m^d equal sub-boxes; u and every
    component of q live in the C0 space of tensor-product degree-p Lagrange
    polynomials on the sub-boxes (continuous inside the macro-element,
    discontinuous across macro-elements);
  * the trace u^ lives on each macro-face in the C0 degree-p space of the
    m^(d-1) sub-faces, independent from one macro-face to the next.  (The trace
    space reading is the one that reproduces the paper's DOF tables.)
  * nodal basis on Gauss-Lobatto-Legendre points of each sub-interval;
  * quadrature: p+2 Gauss-Legendre points per direction on each sub-box/sub-face.

Numbering (the library's data layout, written here independently):
  * macro e = ix + nx (iy + ny iz); node a = i0 + n (i1 + n i2), n = m p + 1;
  * state u[e][s][a], gradient q[e][k][s][a];
  * faces: all x-normal faces, then y-normal, then z-normal; the k-normal faces
    at position i (0..nk, or 0..nk-1 when periodic) and tangential macro indices
    (j, l) get index i + npos_k (j + n_t1 l) inside their group;
  * face nodes lexicographic in the tangential axes (lower axis fastest);
  * trace vector uhat[f][s][j]; a macro's local trace vector is species-major
    [s][(face_local, j)] with local faces ordered (-x, +x, -y, +y, -z, +z).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gll_points(p):
    """Gauss-Lobatto-Legendre points on [-1, 1] (roots of (1-x^2) P_p'(x))."""
    if p == 1:
        return np.array([-1.0, 1.0])
    c = np.zeros(p + 1)
    c[p] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(c))))
    return np.concatenate([[-1.0], inner, [1.0]])


def lagrange(nodes, x):
    """Values L[i_x, j] and derivatives dL[i_x, j] of the Lagrange basis on ``nodes``."""
    n = len(nodes)
    x = np.asarray(x, dtype=float)
    L = np.ones((len(x), n))
    dL = np.zeros((len(x), n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            L[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
        for l in range(n):
            if l == j:
                continue
            term = np.ones(len(x)) / (nodes[j] - nodes[l])
            for k in range(n):
                if k in (j, l):
                    continue
                term *= (x - nodes[k]) / (nodes[j] - nodes[k])
            dL[:, j] += term
    return L, dL


class Macro1D:
    """1D factors of a macro-element interval [a, b] with m sub-intervals of degree p."""

    def __init__(self, a, b, m, p):
        self.m, self.p = m, p
        self.n = m * p + 1
        he = (b - a) / m
        self.he = he
        xi = gll_points(p)
        gq, gw = npleg.leggauss(p + 2)
        Lq, dLq = lagrange(xi, gq)
        nq = p + 2
        self.nq_tot = m * nq
        self.B = np.zeros((m * nq, self.n))   # basis values at quadrature points
        self.D = np.zeros((m * nq, self.n))   # physical derivatives
        self.w = np.zeros(m * nq)             # physical weights
        self.xq = np.zeros(m * nq)
        self.xn = np.zeros(self.n)
        for e in range(m):
            x0 = a + e * he
            rows = slice(e * nq, (e + 1) * nq)
            cols = slice(e * p, e * p + p + 1)
            self.B[rows, cols] = Lq
            self.D[rows, cols] = dLq * (2.0 / he)
            self.w[rows] = gw * he / 2.0
            self.xq[rows] = x0 + (gq + 1.0) * he / 2.0
            self.xn[e * p:e * p + p + 1] = x0 + (xi + 1.0) * he / 2.0
        self.xn[0], self.xn[-1] = a, b
        self.end = [np.eye(self.n)[0:1], np.eye(self.n)[self.n - 1:self.n]]


def kron_axes(mats):
    """Kronecker product of per-axis matrices, axis 0 varying fastest."""
    out = mats[-1]
    for M in reversed(mats[:-1]):
        out = np.kron(out, M)
    return out


class MacroGeometry:
    """Basis values, weights and faces of one box macro-element."""

    def __init__(self, lo, hi, m, p):
        d = len(lo)
        self.d, self.m, self.p = d, m, p
        ax = [Macro1D(lo[k], hi[k], m, p) for k in range(d)]
        self.ax = ax
        self.n1 = ax[0].n
        self.Np = self.n1 ** d
        self.h = min(ax[k].he for k in range(d))
        # volume: T[alpha] [G, Np]; alpha = 0 value, 1..d derivatives
        T = [kron_axes([a.B for a in ax])]
        for k in range(d):
            T.append(kron_axes([ax[j].D if j == k else ax[j].B for j in range(d)]))
        self.T = np.array(T)
        self.w = kron_axes([a.w[:, None] for a in ax])[:, 0]
        self.xq = np.array([kron_axes([(ax[j].xq if j == k else np.ones(ax[j].nq_tot))[:, None]
                                       for j in range(d)])[:, 0] for k in range(d)])
        self.xn = np.array([kron_axes([(ax[j].xn if j == k else np.ones(ax[j].n))[:, None]
                                       for j in range(d)])[:, 0] for k in range(d)])
        # faces, ordered (-x, +x, -y, +y, -z, +z)
        self.Nfn = self.n1 ** (d - 1)
        self.faces = []
        for k in range(d):
            tang = [j for j in range(d) if j != k]
            for side in range(2):
                phi = kron_axes([ax[j].end[side] if j == k else ax[j].B for j in range(d)])
                psi = kron_axes([ax[j].B for j in tang]) if tang else np.ones((1, 1))
                wf = kron_axes([ax[j].w[:, None] for j in tang])[:, 0] if tang else np.ones(1)
                xf = []
                for kk in range(d):
                    if kk == k:
                        xf.append(np.full(len(wf), (lo[k], hi[k])[side]))
                    else:
                        xf.append(kron_axes([(ax[j].xq if j == kk else np.ones(ax[j].nq_tot))[:, None]
                                             for j in tang])[:, 0])
                n = np.zeros(d)
                n[k] = -1.0 if side == 0 else 1.0
                self.faces.append(dict(k=k, side=side, phi=phi, psi=psi, w=wf,
                                       n=n, x=np.array(xf)))
        self.Nth = 2 * d * self.Nfn


class BoxMesh:
    """Structured box mesh of macro-elements with global trace numbering."""

    def __init__(self, prob):
        d = prob["dim"]
        self.d = d
        self.nm = list(prob["nmac"][:d])
        self.lo = np.array(prob["lo"][:d], dtype=float)
        self.hi = np.array(prob["hi"][:d], dtype=float)
        self.per = [bool(x) for x in prob["periodic"][:d]]
        self.m, self.p = prob["m"], prob["p"]
        self.E = int(np.prod(self.nm))
        self.n1 = self.m * self.p + 1
        self.Nfn = self.n1 ** (d - 1)
        # face groups per normal axis
        self.npos = [self.nm[k] if self.per[k] else self.nm[k] + 1 for k in range(d)]
        self.goff = [0] * d
        tot = 0
        for k in range(d):
            self.goff[k] = tot
            ntan = int(np.prod([self.nm[j] for j in range(d) if j != k]))
            tot += self.npos[k] * ntan
        self.F = tot
        self.dx = (self.hi - self.lo) / np.array(self.nm)

    def macro_index(self, idx):
        e = 0
        for k in reversed(range(self.d)):
            e = e * self.nm[k] + idx[k]
        return e

    def macro_coords(self, e):
        idx = []
        for k in range(self.d):
            idx.append(e % self.nm[k])
            e //= self.nm[k]
        return idx

    def macro_box(self, e):
        idx = self.macro_coords(e)
        lo = self.lo + self.dx * np.array(idx)
        return lo, lo + self.dx

    def face_index(self, k, pos, idx):
        tang = [j for j in range(self.d) if j != k]
        loc = 0
        for j in reversed(tang):
            loc = loc * self.nm[j] + idx[j]
        return self.goff[k] + pos + self.npos[k] * loc

    def macro_faces(self, e):
        """Global face id and boundary side (or -1) of local faces (-x, +x, -y, ...)."""
        idx = self.macro_coords(e)
        out = []
        for k in range(self.d):
            for side in range(2):
                pos = idx[k] + side
                bside = -1
                if pos == self.nm[k]:
                    if self.per[k]:
                        pos = 0
                    else:
                        bside = 2 * k + 1
                if pos == 0 and side == 0 and not self.per[k]:
                    bside = 2 * k
                out.append((self.face_index(k, pos, idx), bside))
        return out

    def gather_map(self, e, ns):
        """Indices into the flat global trace vector of the macro's local trace vector.

        Local order: species-major, then local face, then face node.
        """
        faces = self.macro_faces(e)
        g = np.zeros((ns, len(faces) * self.Nfn), dtype=np.int64)
        for s in range(ns):
            for fl, (f, _) in enumerate(faces):
                g[s, fl * self.Nfn:(fl + 1) * self.Nfn] = (f * ns + s) * self.Nfn + np.arange(self.Nfn)
        return g

    def face_owners(self):
        """For each face the list of (macro, local face) that touch it."""
        own = [[] for _ in range(self.F)]
        for e in range(self.E):
            for fl, (f, _) in enumerate(self.macro_faces(e)):
                own[f].append((e, fl))
        return own
