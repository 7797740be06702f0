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
        # derivatives of the macro basis at the two ends of the interval
        _, dl0 = lagrange(xi, [-1.0])
        _, dl1 = lagrange(xi, [1.0])
        self.end_d = [np.zeros((1, self.n)), np.zeros((1, self.n))]
        self.end_d[0][0, 0:p + 1] = dl0[0] * (2.0 / he)
        self.end_d[1][0, self.n - p - 1:] = dl1[0] * (2.0 / he)


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


def face_node_table(d, n1):
    """Macro node of each local face node, per local face (-x, +x, -y, ...): the face nodes are
    lexicographic in the face's tangential axes, the lower axis fastest."""
    idx = np.arange(n1 ** d).reshape([n1] * d)          # [i_{d-1}, ..., i_0]
    out = []
    for k in range(d):
        for side in range(2):
            sl = [slice(None)] * d
            sl[d - 1 - k] = 0 if side == 0 else n1 - 1
            out.append(idx[tuple(sl)].ravel())
    return out


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
        self.fnodes = face_node_table(d, self.n1)

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


class MappedMacroGeometry:
    """Basis values, weights and faces of a macro-element mapped from [0, 1]^d.

    The map is isoparametric (Sec. 2.2 spaces; the curved-macro reading): x(xi) =
    sum_a x_a phi_a(xi) with the macro's own C0 basis, so the geometry is exactly the
    interpolant of the node positions x_a.  At every quadrature point J[i][j] =
    dx_i/dxi_j, the weight is the reference weight times det J, and physical
    derivatives are d_k phi = sum_j (J^-1)[j][k] d phi / d xi_j.  On the face
    xi_k = 0 (1) the area-weighted outward normal is -(+) det J (J^-T e_k): the
    weight is its length and n its direction, one per face point.  The mass
    matrix of these weights is the per-macro A_qq = I (x) M_J of a non-affine
    macro (affine macros give back diag(J) M).  Same attributes as MacroGeometry,
    except that each face's n is [d, points].
    """

    def __init__(self, xn, m, p, h):
        xn = np.asarray(xn, dtype=float)
        d = xn.shape[0]
        self.d, self.m, self.p = d, m, p
        ax = [Macro1D(0.0, 1.0, m, p) for _ in range(d)]
        self.ax = ax
        self.n1 = ax[0].n
        self.Np = self.n1 ** d
        self.h = h
        Tr = [kron_axes([a.B for a in ax])]
        for k in range(d):
            Tr.append(kron_axes([ax[j].D if j == k else ax[j].B for j in range(d)]))
        Tr = np.array(Tr)                                        # [d+1, G, Np], reference derivatives
        J = np.einsum("ia,jga->gij", xn, Tr[1:])                 # J[g, i, j] = dx_i / dxi_j
        det = np.linalg.det(J)
        if np.any(det <= 0.0):
            raise ValueError("mapped macro-element with non-positive Jacobian")
        Ji = np.linalg.inv(J)                                    # Ji[g, j, i] = dxi_j / dx_i
        T = [Tr[0]]
        for k in range(d):
            T.append(sum(Ji[:, j, k][:, None] * Tr[1 + j] for j in range(d)))
        self.T = np.array(T)
        self.detJ = det
        self.w = kron_axes([a.w[:, None] for a in ax])[:, 0] * det
        self.xq = xn @ Tr[0].T
        self.xn = xn
        self.Nfn = self.n1 ** (d - 1)
        self.faces = []
        for k in range(d):
            tang = [j for j in range(d) if j != k]
            for side in range(2):
                phi = kron_axes([ax[j].end[side] if j == k else ax[j].B for j in range(d)])
                psi = kron_axes([ax[j].B for j in tang]) if tang else np.ones((1, 1))
                wref = kron_axes([ax[j].w[:, None] for j in tang])[:, 0] if tang else np.ones(1)
                dphi = []
                for jj in range(d):
                    mats = []
                    for j in range(d):
                        if j == k:
                            mats.append(ax[j].end_d[side] if jj == k else ax[j].end[side])
                        else:
                            mats.append(ax[j].D if jj == j else ax[j].B)
                    dphi.append(kron_axes(mats))
                Jf = np.einsum("ia,jfa->fij", xn, np.array(dphi))
                detf = np.linalg.det(Jf)
                Jif = np.linalg.inv(Jf)
                nw = (1.0 if side == 1 else -1.0) * detf[:, None] * Jif[:, k, :]   # [fp, d]
                area = np.sqrt(np.sum(nw * nw, axis=1))
                self.faces.append(dict(k=k, side=side, phi=phi, psi=psi, w=wref * area,
                                       n=(nw / area[:, None]).T.copy(), x=xn @ phi.T))
        self.Nth = 2 * d * self.Nfn


# cube-panel frames (e_n, e_1, e_2) of the cubed sphere, e_1 x e_2 = e_n, panels
# (+x, -x, +y, -y, +z, -z)
SHELL_FRAMES = (((1, 0, 0), (0, 1, 0), (0, 0, 1)),
                ((-1, 0, 0), (0, 0, 1), (0, 1, 0)),
                ((0, 1, 0), (0, 0, 1), (1, 0, 0)),
                ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
                ((0, 0, 1), (1, 0, 0), (0, 1, 0)),
                ((0, 0, -1), (0, 1, 0), (1, 0, 0)))


def shell_radius(s, r0, r1, nr, ratio):
    """Radius at radial coordinate s in [0, nr]: layer k spans [R(k), R(k+1)], the layer
    thicknesses grow by the factor ``ratio`` (uniform when ratio == 1)."""
    if ratio == 1.0:
        return r0 + (r1 - r0) * s / nr
    return r0 + (r1 - r0) * (ratio ** s - 1.0) / (ratio ** nr - 1.0)


class ShellMesh:
    """Cubed-sphere O-grid of the spherical shell r0 <= |x| <= r1 (d = 3).

    Macro e = ((panel nr + k) nq + j) nq + i, panel in SHELL_FRAMES order, (i, j) the
    equiangular cell of the panel and k the radial layer.  Macro reference axes:
    xi_0 along e_1, xi_1 along e_2, xi_2 outward.  A macro node with macro-lattice
    coordinates (t0, t1, t2) in [0, 1]^3 sits at R(k + t2) dir / |dir| with dir = e_n +
    tan(a) e_1 + tan(b) e_2, a = -pi/4 + (i + t0) pi / (2 nq), b likewise with (j, t1).
    Faces are numbered in order of first appearance over (macro, local face); a face's
    node order is that of its first owner (lexicographic in its tangential axes), the
    second owner's nodes are matched by position.  Boundary sides: 0 the inner sphere
    (xi_2 = 0 of layer 0), 1 the outer sphere.  SUPG length: the smaller of the first
    layer's radial thickness and the inner cell's arc, divided by m.
    """

    def __init__(self, prob):
        if prob["dim"] != 3:
            raise ValueError("the shell mesh is three-dimensional")
        self.d = 3
        self.nq, self.nr = int(prob["shell_n"][0]), int(prob["shell_n"][1])
        self.r0, self.r1, self.ratio = (float(x) for x in prob["shell_r"][:3])
        self.m, self.p = prob["m"], prob["p"]
        self.n1 = self.m * self.p + 1
        self.Nfn = self.n1 ** 2
        self.E = 6 * self.nq * self.nq * self.nr
        self.h = min(shell_radius(1.0, self.r0, self.r1, self.nr, self.ratio) - self.r0,
                     self.r0 * 0.5 * np.pi / self.nq) / self.m
        t = Macro1D(0.0, 1.0, self.m, self.p).xn
        self.t = t
        n1 = self.n1
        self.nodes = np.zeros((self.E, 3, n1 ** 3))
        i2, i1, i0 = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
        i0, i1, i2 = i0.ravel(), i1.ravel(), i2.ravel()       # node a = i0 + n1 (i1 + n1 i2)
        for e in range(self.E):
            i, j, k, pan = self.macro_coords(e)
            en, e1, e2 = (np.array(v, dtype=float) for v in SHELL_FRAMES[pan])
            a = -0.25 * np.pi + (i + t[i0]) * 0.5 * np.pi / self.nq
            b = -0.25 * np.pi + (j + t[i1]) * 0.5 * np.pi / self.nq
            r = shell_radius(k + t[i2], self.r0, self.r1, self.nr, self.ratio)
            dirs = en[:, None] + np.tan(a)[None, :] * e1[:, None] + np.tan(b)[None, :] * e2[:, None]
            self.nodes[e] = r[None, :] * dirs / np.linalg.norm(dirs, axis=0)[None, :]
        self.fnodes = face_node_table(3, n1)
        # faces by matching node positions
        tol = 1e-9 * self.r1
        keys = []
        for e in range(self.E):
            for fl in range(6):
                keys.append(self.nodes[e][:, self.fnodes[fl]].mean(axis=1))
        keys = np.array(keys)
        nloc = len(keys)
        fid = -np.ones(nloc, dtype=np.int64)
        self.F = 0
        self.owners = []
        for q_ in range(nloc):
            if fid[q_] >= 0:
                continue
            dist = np.max(np.abs(keys - keys[q_][None, :]), axis=1)
            same = np.nonzero(dist < tol)[0]
            if len(same) > 2:
                raise ValueError("face with more than two owners")
            fid[same] = self.F
            self.owners.append([(int(s) // 6, int(s) % 6) for s in same])
            self.F += 1
        self.fid = fid.reshape(self.E, 6)
        # node permutation of each owner: global face node g <- local face node perm[g]
        self.perm = np.zeros((self.E, 6, self.Nfn), dtype=np.int64)
        for f, own in enumerate(self.owners):
            e0, f0 = own[0]
            x0 = self.nodes[e0][:, self.fnodes[f0]]
            self.perm[e0, f0] = np.arange(self.Nfn)
            for (e1_, f1_) in own[1:]:
                x1 = self.nodes[e1_][:, self.fnodes[f1_]]
                dd = np.max(np.abs(x0[:, :, None] - x1[:, None, :]), axis=0)   # [g0, l1]
                match = np.argmin(dd, axis=1)
                if np.any(dd[np.arange(self.Nfn), match] > tol) or len(set(match.tolist())) != self.Nfn:
                    raise ValueError("face nodes of two owners do not match")
                self.perm[e1_, f1_] = match

    def macro_coords(self, e):
        i = e % self.nq
        r = e // self.nq
        j = r % self.nq
        r //= self.nq
        k = r % self.nr
        return i, j, k, r // self.nr

    def macro_faces(self, e):
        """Global face id and boundary side (0 inner, 1 outer, -1 interior) of local faces."""
        i, j, k, _ = self.macro_coords(e)
        out = []
        for fl in range(6):
            bside = -1
            if fl == 4 and k == 0:
                bside = 0
            if fl == 5 and k == self.nr - 1:
                bside = 1
            out.append((int(self.fid[e, fl]), bside))
        return out

    def gather_map(self, e, ns):
        """Indices into the flat global trace vector of the macro's local trace vector
        (local order: species, local face, the macro's own face-node order)."""
        g = np.zeros((ns, 6 * self.Nfn), dtype=np.int64)
        for fl in range(6):
            f = int(self.fid[e, fl])
            inv = np.empty(self.Nfn, dtype=np.int64)
            inv[self.perm[e, fl]] = np.arange(self.Nfn)       # local node -> global node
            for s in range(ns):
                g[s, fl * self.Nfn:(fl + 1) * self.Nfn] = (f * ns + s) * self.Nfn + inv
        return g

    def face_owners(self):
        return [list(o) for o in self.owners]
