"""Condensation, dense LU, global trace operator, Krylov solvers, Newton and DIRK.

Test infrastructure only (see ``oracle/__init__``).

Everything is the plain definition: dense matrices, numpy.linalg.solve for
A_qq^{-1} applications, an explicit row-pivoted LU written out below, explicit
loops over macro-elements.  Pinned by tests/test_oracle_pins.py.
"""
import numpy as np

from . import assemble as asm
from . import fields
from .simplex import SimplexBoxMesh
from .space import BoxMesh, MacroGeometry, MappedMacroGeometry, ShellMesh


# ---------------------------------------------------------------- dense LU (Remark, Sec. 3.3)

def lu_factor(A):
    """P A = L U with partial pivoting (first row of maximal |.| wins ties).

    Returns (LU, piv) with unit-lower L below the diagonal, U on and above it,
    and piv[i] = the original row that ends up in row i.
    """
    A = np.array(A, dtype=float, copy=True)
    n = A.shape[0]
    piv = np.arange(n)
    for k in range(n):
        r = k + int(np.argmax(np.abs(A[k:, k])))
        if A[r, k] == 0.0:
            raise np.linalg.LinAlgError("singular matrix in lu_factor at column %d" % k)
        if r != k:
            A[[k, r]] = A[[r, k]]
            piv[[k, r]] = piv[[r, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, piv


def lu_solve(LU, piv, b):
    """Solve A x = b from lu_factor's output by forward and back substitution."""
    y = np.array(b, dtype=float)[piv]
    n = LU.shape[0]
    for i in range(n):
        y[i] = y[i] - LU[i, :i] @ y[:i]
    for i in reversed(range(n)):
        y[i] = (y[i] - LU[i, i + 1:] @ y[i + 1:]) / LU[i, i]
    return y


# ---------------------------------------------------------------- problem setup

def phys_of(prob):
    return dict(gamma=prob["gamma"], Re=prob["Re"], Pr=prob["Pr"], supg=prob.get("supg", 0))


def uniform_from_par(prob):
    fp = prob["field_par"]
    d = prob["dim"]
    return fields.uniform_u(d, fp[0], fp[1:1 + d], fp[4], prob["gamma"])


class Problem:
    """Mesh, per-macro geometry factory and boundary data of one problem."""

    def __init__(self, prob):
        self.prob = prob
        self.shell = int(prob.get("mesh_kind", 0)) == 1
        self.simplex = int(prob.get("mesh_kind", 0)) == 2
        if self.shell:
            self.mesh = ShellMesh(prob)
        elif self.simplex:
            self.mesh = SimplexBoxMesh(prob)
        else:
            self.mesh = BoxMesh(prob)
        self.d = prob["dim"]
        self.ns = self.d + 2
        self.phys = phys_of(prob)
        self.m, self.p = prob["m"], prob["p"]
        g0 = self.geometry(0)
        self.Np, self.Nfn, self.Nth = g0.Np, g0.Nfn, g0.Nth
        self.F = self.mesh.F
        self.E = self.mesh.E
        self.maps = [self.mesh.gather_map(e, self.ns) for e in range(self.E)]

    def geometry(self, e):
        if self.shell:
            return MappedMacroGeometry(self.mesh.nodes[e], self.m, self.p, self.mesh.h)
        if self.simplex:
            return self.mesh.geometry(e)
        lo, hi = self.mesh.macro_box(e)
        return MacroGeometry(lo, hi, self.m, self.p)

    def source(self, geo):
        if self.prob["field"] == 1:
            return fields.mms_source(geo.xq, self.prob["field_par"], self.phys)
        if self.prob["field"] == 5:
            return fields.couette3d_source(geo.xq, self.prob["field_par"], self.phys)
        return None

    def bfaces(self, e, geo):
        """(kind, data) per local face of macro e."""
        prob = self.prob
        out = []
        for fl, (f, bside) in enumerate(self.mesh.macro_faces(e)):
            if bside < 0:
                out.append((0, None))
                continue
            kind = prob["bc"][bside]
            fc = geo.faces[fl]
            if kind == 1:
                if prob["field"] == 1:
                    uD = fields.mms_u(fc["x"], prob["field_par"], prob["gamma"])
                elif prob["field"] == 5:
                    uD = fields.couette3d_u(fc["x"], prob["field_par"], prob["gamma"])
                else:
                    uD = np.repeat(uniform_from_par(prob)[:, None], len(fc["w"]), axis=1)
                out.append((1, dict(uD=uD)))
            elif kind == 2:
                out.append((2, dict(Tw=prob["wall_T"][bside], vw=list(prob["wall_v"][bside]))))
            elif kind == 3:
                uinf = np.repeat(uniform_from_par(prob)[:, None], len(fc["w"]), axis=1)
                out.append((3, dict(uinf=uinf)))
            else:
                raise ValueError("bad bc kind %d" % kind)
        return out

    # -- state layout helpers
    def local_trace(self, e, uh_flat):
        return uh_flat[self.maps[e]]

    def zeros_state(self):
        return (np.zeros((self.E, self.ns, self.Np)), np.zeros((self.E, self.d, self.ns, self.Np)),
                np.zeros(self.F * self.ns * self.Nfn))


def initial_state(P, lift=True):
    """Initial state from the problem's closed-form field: u at the macro nodes, u^ on each face
    from its first owner's u, q = 0 or (lift) the gradient that zeroes R_Q:
    A_qq q = -(A_qu u + A_quh u^), i.e. M q_k = -(G_k u + Gh_k u^) per species."""
    prob = P.prob
    fp = prob["field_par"]
    u = np.zeros((P.E, P.ns, P.Np))
    for e in range(P.E):
        x = P.geometry(e).xn
        if prob["field"] == 1:
            u[e] = fields.mms_u(x, fp, prob["gamma"])
        elif prob["field"] == 3:
            u[e] = fields.tgv_u(x, fp[0], prob["gamma"])
        elif prob["field"] == 5:
            u[e] = fields.couette3d_u(x, fp, prob["gamma"])
        elif prob["field"] == 4:
            u[e] = fields.shell_initial_u(x, fp[0], fp[1:4], fp[4], prob["gamma"])
        else:
            u[e] = uniform_from_par(prob)[:, None]
    uh = np.zeros(P.F * P.ns * P.Nfn)
    for f, own in enumerate(P.mesh.face_owners()):
        e, fl = own[0]
        g = P.maps[e][:, fl * P.Nfn:(fl + 1) * P.Nfn]          # [s, local face node] -> trace index
        for s in range(P.ns):
            uh[g[s]] = u[e, s, P.mesh.fnodes[fl]]
    q = np.zeros((P.E, P.d, P.ns, P.Np))
    if lift:
        for e in range(P.E):
            geo = P.geometry(e)
            uhl = P.local_trace(e, uh)
            b = asm.assemble_macro(geo, P.phys, u[e], q[e], uhl, want_jac=False)
            for k in range(P.d):
                q[e, k] = -np.linalg.solve(b["M"], b["Gk"][k] @ u[e].T + b["Ghk"][k] @ uhl.T).T
    return u, q, uh


# ---------------------------------------------------------------- condensation

def condense_second_layer(geo, blk, shift=0.0):
    """Second-layer static condensation, eqs. AP12 and ASC2 (Sec. 3.3).

    S = A_uu - A_uq A_qq^{-1} A_qu          (Schur complement of A_local)
    C = -A_uuh + A_uq A_qq^{-1} A_quh       (step-1 operator of Algorithm 2)
    B = A_uhu - A_uhq A_qq^{-1} A_qu        (step-3 operator)
    D = A_uhuh - A_uhq A_qq^{-1} A_quh      (step-4 operator)
    g = -R_U + A_uq A_qq^{-1} R_Q,  h = -R_Uh + A_uhq A_qq^{-1} R_Q
    A^T_i = B S^{-1} C + D,  b^T_i = h - B S^{-1} g.
    ``shift`` adds shift * (I (x) M) to A_uu (pseudo-time term, reading of Sec. 3.1).
    """
    d = geo.d
    ns = d + 2
    Aqq, Aqu, Aqh, Auq, Ahq = asm.full_local_blocks(geo, blk)
    Auu = blk["Auu"] + shift * np.kron(np.eye(ns), blk["M"])
    RQ = blk["RQ"].reshape(-1)
    RU = blk["RU"].reshape(-1)
    RUh = blk["RUh"].reshape(-1)
    X_u = np.linalg.solve(Aqq, Aqu)
    X_h = np.linalg.solve(Aqq, Aqh)
    X_r = np.linalg.solve(Aqq, RQ)
    S = Auu - Auq @ X_u
    C = -blk["Auh"] + Auq @ X_h
    B = blk["Ahu"] - Ahq @ X_u
    D = blk["Ahh"] - Ahq @ X_h
    g = -RU + Auq @ X_r
    h = -RUh + Ahq @ X_r
    LU, piv = lu_factor(S)
    Sg = lu_solve(LU, piv, g)
    return dict(S=S, LU=LU, piv=piv, B=B, C=C, D=D, g=g, h=h, bhat=h - B @ Sg,
                X_u=X_u, X_h=X_h, X_r=X_r)


def condense_one_layer(geo, blk, shift=0.0):
    """One-layer static condensation, eqs. C46-C47 (Sec. 3.2): A^T_i and b^T_i."""
    d = geo.d
    ns = d + 2
    Aqq, Aqu, Aqh, Auq, Ahq = asm.full_local_blocks(geo, blk)
    Auu = blk["Auu"] + shift * np.kron(np.eye(ns), blk["M"])
    Aloc = np.block([[Aqq, Aqu], [Auq, Auu]])
    right = np.vstack([Aqh, blk["Auh"]])
    left = np.hstack([Ahq, blk["Ahu"]])
    R = np.concatenate([blk["RQ"].reshape(-1), blk["RU"].reshape(-1)])
    Ahat = blk["Ahh"] - left @ np.linalg.solve(Aloc, right)
    bhat = -blk["RUh"].reshape(-1) + left @ np.linalg.solve(Aloc, R)
    return Ahat, bhat


def apply_local(c, x):
    """Steps 1-4 of Algorithm 2 for one macro-element."""
    y1 = c["C"] @ x
    y2 = lu_solve(c["LU"], c["piv"], y1)
    y3 = c["B"] @ y2
    return y3 + c["D"] @ x


def apply_trace(P, cond, x):
    """Algorithm 2: y = sum_i eps_i^T (B_i S_i^{-1} C_i + D_i) eps_i x."""
    y = np.zeros_like(x)
    for e in range(P.E):
        eps = P.maps[e].reshape(-1)
        y4 = apply_local(cond[e], x[eps])
        np.add.at(y, eps, y4)
    return y


def explicit_trace_matrix(P, cond):
    """The assembled global trace matrix A^ = sum_i eps_i^T A^T_i eps_i (eq. C44)."""
    n = P.F * P.ns * P.Nfn
    A = np.zeros((n, n))
    for e in range(P.E):
        eps = P.maps[e].reshape(-1)
        Ai = cond[e]["B"] @ np.column_stack([lu_solve(cond[e]["LU"], cond[e]["piv"], cond[e]["C"][:, j])
                                             for j in range(cond[e]["C"].shape[1])]) + cond[e]["D"]
        A[np.ix_(eps, eps)] += Ai
    return A


def assemble_bhat(P, cond):
    """Lines 2-5 of Algorithm 1: b^ = sum_i eps_i^T b^T_i."""
    b = np.zeros(P.F * P.ns * P.Nfn)
    for e in range(P.E):
        np.add.at(b, P.maps[e].reshape(-1), cond[e]["bhat"])
    return b


def recover(geo, blk, c, dUh_loc):
    """Local recovery, eqs. Csc4a then Csc4b (dU first: dQ needs it)."""
    d = geo.d
    Aqq, Aqu, Aqh, Auq, Ahq = asm.full_local_blocks(geo, blk)
    dU = lu_solve(c["LU"], c["piv"], c["g"] + c["C"] @ dUh_loc)
    dQ = np.linalg.solve(Aqq, -blk["RQ"].reshape(-1) - Aqu @ dU - Aqh @ dUh_loc)
    return dU, dQ


# ---------------------------------------------------------------- preconditioner (Sec. 4.2)

def face_blocks(P, blks):
    """Block-diagonal part A_uhuh of the global system, one dense block per macro-face."""
    ns, Nfn, Nth = P.ns, P.Nfn, P.Nth
    out = np.zeros((P.F, ns * Nfn, ns * Nfn))
    for e in range(P.E):
        for fl, (f, _) in enumerate(P.mesh.macro_faces(e)):
            idx = (np.arange(ns)[:, None] * Nth + fl * Nfn + np.arange(Nfn)[None, :]).ravel()
            loc = P.maps[e][:, fl * Nfn:(fl + 1) * Nfn].ravel() - f * ns * Nfn
            out[f][np.ix_(loc, loc)] += blks[e]["Ahh"][np.ix_(idx, idx)]
    return out


def block_jacobi(P, fblocks_lu, r):
    """z = (A_uhuh)^{-1} r, face by face."""
    z = np.zeros_like(r)
    n = P.ns * P.Nfn
    for f in range(P.F):
        LU, piv = fblocks_lu[f]
        z[f * n:(f + 1) * n] = lu_solve(LU, piv, r[f * n:(f + 1) * n])
    return z


def gmres_fixed(A, Minv, b, nu):
    """nu steps of GMRES on Minv A z = Minv b from z = 0 (left preconditioning)."""
    r = Minv(b)
    beta = np.linalg.norm(r)
    n = len(b)
    z = np.zeros(n)
    if beta == 0.0:
        return z
    V = np.zeros((nu + 1, n))
    H = np.zeros((nu + 1, nu))
    V[0] = r / beta
    k_used = 0
    for j in range(nu):
        w = Minv(A(V[j]))
        for _ in range(2):
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        k_used = j + 1
        if H[j + 1, j] <= 1e-300:
            break
        V[j + 1] = w / H[j + 1, j]
    e1 = np.zeros(k_used + 1)
    e1[0] = beta
    y = np.linalg.lstsq(H[:k_used + 1, :k_used], e1, rcond=None)[0]
    return V[:k_used].T @ y


def fgmres(A, M, b, rtol=1e-10, atol=0.0, restart=30, maxit=1000):
    """Right-preconditioned flexible GMRES(restart) with CGS2 (Sec. 4.2).

    Returns x, iterations, final residual norm (of the Arnoldi recurrence).
    """
    n = len(b)
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    tol = max(rtol * bnorm, atol)
    its = 0
    r = b.copy()
    beta = bnorm
    if beta <= tol:
        return x, 0, beta
    while its < maxit:
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        gv = np.zeros(restart + 1)
        gv[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(restart):
            Z[j] = M(V[j])
            w = A(Z[j])
            for _ in range(2):
                h = V[:j + 1] @ w
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rr = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rr, H[j + 1, j] / rr
            H[j, j] = rr
            H[j + 1, j] = 0.0
            gv[j + 1] = -sn[j] * gv[j]
            gv[j] = cs[j] * gv[j]
            its += 1
            j_end = j + 1
            if abs(gv[j + 1]) <= tol or its >= maxit:
                break
        y = np.zeros(j_end)
        for i in reversed(range(j_end)):
            y[i] = (gv[i] - H[i, i + 1:j_end] @ y[i + 1:]) / H[i, i]
        x = x + Z[:j_end].T @ y
        r = b - A(x)
        beta = np.linalg.norm(r)
        if beta <= tol or its >= maxit:
            break
    return x, its, beta


def gmres_left(A, Minv, b, rtol=1e-10, atol=0.0, restart=30, maxit=1000):
    """Restarted GMRES(restart) on Minv A x = Minv b (left preconditioning, CGS2): the
    baseline solver of Sec. 4.2 with the fixed block-Jacobi preconditioner (A_uhuh)^-1.
    The stopping test is on the preconditioned residual |Minv (b - A x)|.

    Each cycle minimises |Minv (b - A x)| over x_start + the Krylov space of Minv A,
    here by a least-squares solve with the Arnoldi Hessenberg matrix.
    Returns x, iterations, final preconditioned residual norm.
    """
    n = len(b)
    x = np.zeros(n)
    r = Minv(b)
    beta = np.linalg.norm(r)
    tol = max(rtol * beta, atol)
    its = 0
    while beta > tol and its < maxit:
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        V[0] = r / beta
        k = 0
        for j in range(restart):
            w = Minv(A(V[j]))
            for _ in range(2):
                h = V[:j + 1] @ w
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            its += 1
            k = j + 1
            e1 = np.zeros(k + 1)
            e1[0] = beta
            y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[:k + 1, :k] @ y)
            if res <= tol or its >= maxit or H[j + 1, j] == 0.0:
                break
            V[j + 1] = w / H[j + 1, j]
        x = x + V[:k].T @ y
        r = Minv(b - A(x))
        beta = np.linalg.norm(r)
    return x, its, beta


# ---------------------------------------------------------------- global drivers

def global_assemble(P, u, q, uh, tt=None, want_jac=True):
    """Assemble every macro; returns per-macro blocks, geometry, and residual norms."""
    blks, geos = [], []
    RUh_g = np.zeros(P.F * P.ns * P.Nfn)
    nQ = nU = 0.0
    for e in range(P.E):
        geo = P.geometry(e)
        tte = None
        if tt is not None:
            tte = dict(coef=tt["coef"], supg_time=tt.get("supg_time", False),
                       hist=None if tt.get("hist") is None else tt["hist"][e])
        blk = asm.assemble_macro(geo, P.phys, u[e], q[e], P.local_trace(e, uh), tte,
                                 P.source(geo), P.bfaces(e, geo), want_jac=want_jac)
        np.add.at(RUh_g, P.maps[e].reshape(-1), blk["RUh"].reshape(-1))
        nQ += np.sum(blk["RQ"] ** 2)
        nU += np.sum(blk["RU"] ** 2)
        blks.append(blk)
        geos.append(geo)
    norms = dict(RQ=np.sqrt(nQ), RU=np.sqrt(nU), RUh=np.linalg.norm(RUh_g))
    norms["RF"] = np.sqrt(nQ + nU + norms["RUh"] ** 2)
    return blks, geos, norms, RUh_g


def flow_integrals(P, u, q):
    """Volume integrals behind the Taylor-Green diagnostics of Sec. 5.3, by the method's own
    volume quadrature (geo.T[0] values, geo.w physical weights) on every macro-element:

        K = int rho |v|^2 / 2,   Z = int rho (omega . omega) / 2,   V = int 1,

    with v = m / rho and omega = curl v (the scalar d_1 v_2 - d_2 v_1 in 2D).  The velocity
    gradient is taken from the HDG gradient q = grad u (eq. C5a): d_j v_i = (q[j, 1+i] -
    v_i q[j, 0]) / rho.  Eq. C5321 gives the dissipation rate eps = 2 mu Z / V; the kinetic
    energy per unit volume is K / V."""
    d = P.d
    K = Z = V = 0.0
    for e in range(P.E):
        geo = P.geometry(e)
        U = u[e] @ geo.T[0].T                                   # [ns, G]
        Q = np.einsum("jsa,ga->jsg", q[e], geo.T[0])            # [d, ns, G]
        rho = U[0]
        v = U[1:1 + d] / rho
        gv = np.array([[(Q[j, 1 + i] - v[i] * Q[j, 0]) / rho for j in range(d)]
                       for i in range(d)])                      # gv[i, j] = d_j v_i
        if d == 3:
            om = np.array([gv[2, 1] - gv[1, 2], gv[0, 2] - gv[2, 0], gv[1, 0] - gv[0, 1]])
        else:
            om = np.array([gv[1, 0] - gv[0, 1]])
        K += np.sum(geo.w * 0.5 * rho * np.sum(v * v, axis=0))
        Z += np.sum(geo.w * 0.5 * rho * np.sum(om * om, axis=0))
        V += np.sum(geo.w)
    return K, Z, V


def linear_step(P, blks, geos, shift=0.0, precond=0, rtol=1e-10, atol=0.0, restart=30,
                maxit=2000, inner=5):
    """One Newton linear solve by condensation + FGMRES + recovery (Algorithm 1)."""
    cond = [condense_second_layer(geos[e], blks[e], shift) for e in range(P.E)]
    b = assemble_bhat(P, cond)
    if precond == "direct":   # dense solve of the explicit trace system (small pins only)
        dUh = np.linalg.solve(explicit_trace_matrix(P, cond), b)
        its = 0
        return _recover_all(P, blks, geos, cond, dUh, its)
    fb = face_blocks(P, blks)
    flu = [lu_factor(fb[f]) for f in range(P.F)]
    A = lambda x: apply_trace(P, cond, x)
    M0 = lambda r: block_jacobi(P, flu, r)
    if precond == 0:
        M = M0
    else:
        M = lambda r: gmres_fixed(A, M0, r, inner)
    dUh, its, res = fgmres(A, M, b, rtol=rtol, atol=atol, restart=restart, maxit=maxit)
    return _recover_all(P, blks, geos, cond, dUh, its)


def _recover_all(P, blks, geos, cond, dUh, its):
    dU = np.zeros((P.E, P.ns, P.Np))
    dQ = np.zeros((P.E, P.d, P.ns, P.Np))
    for e in range(P.E):
        du, dq = recover(geos[e], blks[e], cond[e], dUh[P.maps[e].reshape(-1)])
        dU[e] = du.reshape(P.ns, P.Np)
        dQ[e] = dq.reshape(P.d, P.ns, P.Np)
    return dU, dQ, dUh, its, cond


def newton_ser(P, u, q, uh, rtol=1e-8, atol=1e-14, tau_init=1.0, tau_max=1e8, max_steps=200,
               lin_rtol=1e-6, precond=0, log=None):
    """Pseudo-transient continuation with SER (Sec. 3.1, eq. C31222).

    Reading of the SER update: dtau_{m+1} = min(max(dtau_m |R_U^m| / |R_U^{m+1}|, tau_init), tau_max)
    (the printed ratio is inverted with respect to Mulder and van Leer's rule; the
    floor tau_init keeps the step finite when the first R_U vanishes, e.g. for an
    exactly uniform initial state driven only by a boundary operator).
    """
    u, q, uh = u.copy(), q.copy(), uh.copy()
    blks, geos, nrm, _ = global_assemble(P, u, q, uh)
    R0 = nrm["RF"]
    dtau = tau_init
    hist = [dict(step=0, RF=nrm["RF"], RU=nrm["RU"], dtau=dtau, its=0)]
    steps = 0
    while nrm["RF"] > max(rtol * R0, atol) and steps < max_steps:
        dU, dQ, dUh, its, _ = linear_step(P, blks, geos, shift=1.0 / dtau, precond=precond,
                                          rtol=lin_rtol)
        u += dU
        q += dQ
        uh += dUh
        RU_old = nrm["RU"]
        blks, geos, nrm, _ = global_assemble(P, u, q, uh)
        steps += 1
        dtau = min(max(dtau * RU_old / max(nrm["RU"], 1e-300), tau_init), tau_max)
        hist.append(dict(step=steps, RF=nrm["RF"], RU=nrm["RU"], dtau=dtau, its=its))
        if log:
            log(hist[-1])
    return u, q, uh, hist


# ---------------------------------------------------------------- DIRK (Sec. 2.4)

def alexander_dirk3():
    """Alexander's 3-stage, 3rd-order, L-stable, stiffly accurate DIRK.

    alpha is the root of x^3 - 3x^2 + 3x/2 - 1/6 = 0 in (1/6, 1/2).
    """
    r = np.roots([1.0, -3.0, 1.5, -1.0 / 6.0])
    al = float([x.real for x in r if abs(x.imag) < 1e-12 and 1 / 6 < x.real < 0.5][0])
    b1 = -(6 * al * al - 16 * al + 1) / 4.0
    b2 = (6 * al * al - 20 * al + 5) / 4.0
    A = np.array([[al, 0, 0], [(1 - al) / 2, al, 0], [b1, b2, al]])
    b = np.array([b1, b2, al])
    c = np.array([al, (1 + al) / 2, 1.0])
    return A, b, c


def dirk_step(P, u, q, uh, dt, rtol=1e-8, atol=1e-14, max_newton=30, lin_rtol=1e-8, precond=0,
              tableau=None):
    """One time step of eq. C242 for every stage; u^{n+1} = u^{n,s} (stiffly accurate)."""
    A, b, c = alexander_dirk3() if tableau is None else tableau
    Dm = np.linalg.inv(A)
    s = len(b)
    un = u.copy()
    stages = []
    cur = (u.copy(), q.copy(), uh.copy())
    stats = []
    for i in range(s):
        coef = Dm[i, i] / dt
        hist = -coef * un
        for j in range(i):
            hist = hist + Dm[i, j] * (stages[j] - un) / dt
        tt = dict(coef=coef, hist=hist, supg_time=True)
        uu, qq, hh = (x.copy() for x in cur)
        blks, geos, nrm, _ = global_assemble(P, uu, qq, hh, tt)
        R0 = nrm["RF"]
        k = 0
        lin = 0
        while nrm["RF"] > max(rtol * R0, atol) and k < max_newton:
            dU, dQ, dUh, its, _ = linear_step(P, blks, geos, 0.0, precond=precond, rtol=lin_rtol)
            uu += dU
            qq += dQ
            hh += dUh
            blks, geos, nrm, _ = global_assemble(P, uu, qq, hh, tt)
            k += 1
            lin += its
        stats.append(dict(stage=i + 1, newton=k, fgmres=lin, RF=nrm["RF"], RF0=R0))
        stages.append(uu.copy())
        cur = (uu, qq, hh)
    return cur[0], cur[1], cur[2], stats
