"""Residuals and Newton blocks of one macro-element (eqs. C38, C31221, C312).

Test infrastructure only (see ``oracle/__init__``).

Weak form on a macro-element T with boundary dT (eq. C38 / C242):
  R_Q[k, s, a] = (q_{s,k}, phi_a)_T + (u_s, d_k phi_a)_T - <uh_s, phi_a n_k>_dT
  R_U[s, a]    = (time_s - f_s, phi_a)_T - ((F + G)_{s,k}, d_k phi_a)_T
                 + <(F^ + G^) n, phi_a>_dT + SUPG
  R_Uh[s, i]   = <(F^ + G^) n, psi_i> on interior faces, <B^, psi_i> on dOmega
(the macro's own side of each face; the global R_Uh sums the two sides).

SUPG (Sec. 2.3, defined by reference only; reading): sum over sub-elements of
((A . grad) w, tau R) with A_k = dF_k/du, scalar tau (physics.supg_tau) and the
strong residual R = [time] + sum_k d_k (F_k + G_k)(u_h, q_h) - f, where the
x-derivative is taken by the chain rule through grad u_h and grad q_h inside each
sub-element.  The time term enters R only for DIRK stages (not pseudo time).

Newton blocks (eq. C312) are the exact derivatives of these residuals, taken by
the complex step through every expression (including tau and the forward-mode
derivatives inside R), one input component at a time.

Time term: time(x) = coef u(x) + hist(x), hist a nodal field.  DIRK stage i
(eq. C242): coef = d_ii / dt, hist = -coef u^n + sum_{j<i} d_ij (u^{n,j} - u^n)/dt.
Pseudo time (reading of Sec. 3.1) is not a residual term: the Newton driver adds
(1/dtau) (I (x) M) to A_uu.

Block layout: u index (s, a) species-major, q index (k, s, a), local trace index
(s, (face, j)).  Pinned by tests/test_oracle_pins.py.
"""
import numpy as np

from . import physics as ph

H = ph.CS_H


def vol_integrand(U, GU, Q, GQ, time, f, phys, h, p, supg_time):
    """Coefficients of the volume integrand of R_U at quadrature points.

    R_U[t, a] = sum_g w_g (phi_a W_t + sum_k d_k phi_a V_tk).
    U[s], GU[s][l] = d_l u_s, Q[s][j], GQ[s][j][l] = d_l q_{s,j}; time, f: [ns].
    """
    ns = len(U)
    d = ns - 2
    F = ph.inviscid_flux(U, phys["gamma"])
    G = ph.viscous_flux(U, Q, phys)
    W = [time[t] - f[t] for t in range(ns)]
    V = [[-(F[t][k] + G[t][k]) for k in range(d)] for t in range(ns)]
    if phys.get("supg", 0):
        div, A = ph.flux_divergence_and_A(U, GU, Q, GQ, phys)
        R = [div[t] - f[t] + (time[t] if supg_time else 0.0) for t in range(ns)]
        tau = ph.supg_tau(U, h, p, phys)
        for t in range(ns):
            for k in range(d):
                V[t][k] = V[t][k] + tau * sum(A[k][s][t] * R[s] for s in range(ns))
    return W, V


def _face_eq(uh, q, u, n, bkind, bdata, phys):
    """Equation tested by the trace basis on one face (interior flux or B^)."""
    if bkind == 0:
        return ph.trace_flux(uh, q, u, n, phys)
    if bkind == 1:   # Dirichlet: B^ = uh - u_D
        return [uh[s] - bdata["uD"][s] for s in range(len(uh))]
    if bkind == 2:   # isothermal wall
        return ph.wall_operator(uh, u, bdata["Tw"], bdata["vw"], phys["gamma"])
    if bkind == 3:   # characteristic far field towards the free stream u_inf
        return ph.farfield_operator(uh, u, list(bdata["uinf"]), n, phys["gamma"])
    raise ValueError(bkind)


def _A(x):
    return np.array(x)


def assemble_macro(geo, phys, u, q, uhl, tt=None, src=None, bfaces=None, want_jac=True):
    """Residuals and Jacobian blocks of one macro-element.

    geo    -- space.MacroGeometry
    u      -- [ns, Np];  q -- [d, ns, Np];  uhl -- local trace [ns, Nth]
    tt     -- time term dict(coef, hist [ns, Np] or None, supg_time bool) or None
    src    -- source at volume points [ns, G] or None
    bfaces -- per local face: (kind, data); kind 0 interior/periodic,
              1 Dirichlet (data["uD"] [ns, nfp]), 2 wall (data Tw, vw),
              3 far field (data["uinf"] [ns, nfp])
    Complex u, q, uhl are allowed when want_jac is False (residual only).
    """
    d = geo.d
    ns = d + 2
    Np, Nfn, Nth = geo.Np, geo.Nfn, geo.Nth
    T = geo.T                              # [d+1, G, Np]
    w = geo.w
    G = len(w)
    coef = 0.0 if tt is None else tt["coef"]
    supg_time = False if tt is None else bool(tt.get("supg_time", False))
    dt_ = np.result_type(u, q, uhl)

    # fields at volume points
    U = u @ T[0].T                                                      # [ns, G]
    GU = np.array([u @ T[1 + l].T for l in range(d)]).transpose(1, 0, 2)  # [ns, l, G]
    Q = np.array([q[j] @ T[0].T for j in range(d)]).transpose(1, 0, 2)    # [ns, j, G]
    GQ = np.array([[q[j] @ T[1 + l].T for l in range(d)] for j in range(d)]).transpose(2, 0, 1, 3)  # [ns, j, l, G]
    hist = np.zeros((ns, G)) if (tt is None or tt.get("hist") is None) else tt["hist"] @ T[0].T
    f = np.zeros((ns, G)) if src is None else src

    def integrand(U_, GU_, Q_, GQ_):
        time = [coef * U_[t] + hist[t] for t in range(ns)]
        W, V = vol_integrand(list(U_), ph.to_list(GU_, 2), ph.to_list(Q_, 2), ph.to_list(GQ_, 3),
                             time, list(f), phys, geo.h, geo.p, supg_time)
        return _A(W), _A(V)

    W, V = integrand(U, GU, Q, GQ)
    RU = W @ (w[:, None] * T[0]) + sum(V[:, k] @ (w[:, None] * T[1 + k]) for k in range(d))

    # R_Q (linear): M q_k + G_k u + Gh_k uh
    M = T[0].T @ (w[:, None] * T[0])
    Gk = [T[1 + k].T @ (w[:, None] * T[0]) for k in range(d)]
    Ghk = [np.zeros((Np, Nth)) for _ in range(d)]
    for fl, fc in enumerate(geo.faces):
        sl = slice(fl * Nfn, (fl + 1) * Nfn)
        for k in range(d):
            Ghk[k][:, sl] -= fc["phi"].T @ ((fc["w"] * fc["n"][k])[:, None] * fc["psi"])
    RQ = np.array([M @ q[k].T + Gk[k] @ u.T + Ghk[k] @ uhl.T for k in range(d)]).transpose(0, 2, 1)
    out = dict(RQ=RQ, M=M, Gk=Gk, Ghk=Ghk)
    RU = RU.astype(dt_)
    RUh = np.zeros((ns, Nth), dtype=dt_)

    if want_jac:
        # pointwise kernels K[t, alpha, s, beta, g]: derivative of (W_t | V_tk) wrt
        # (u_s | d_l u_s) for Ku and (q_sj | d_l q_sj) for Kq[j]
        Ku = np.zeros((ns, d + 1, ns, d + 1, G))
        Kq = np.zeros((d, ns, d + 1, ns, d + 1, G))

        def put(K, s, beta, Wd, Vd):
            K[:, 0, s, beta] = np.imag(Wd) / H
            K[:, 1:, s, beta] = np.imag(Vd) / H

        for s in range(ns):
            X = U.astype(complex); X[s] += 1j * H
            put(Ku, s, 0, *integrand(X, GU, Q, GQ))
            for l in range(d):
                X = GU.astype(complex); X[s, l] += 1j * H
                put(Ku, s, 1 + l, *integrand(U, X, Q, GQ))
            for j in range(d):
                X = Q.astype(complex); X[s, j] += 1j * H
                put(Kq[j], s, 0, *integrand(U, GU, X, GQ))
                for l in range(d):
                    X = GQ.astype(complex); X[s, j, l] += 1j * H
                    put(Kq[j], s, 1 + l, *integrand(U, GU, Q, X))

        def contract(K):
            # A[t, a, s, b] = sum_g w_g sum_{alpha,beta} T[alpha][g,a] K[t,alpha,s,beta,g] T[beta][g,b]
            Z = np.einsum("tasbg,bgc->agtsc", K, T)                  # contract beta
            Tw = (T * w[None, :, None]).reshape((d + 1) * G, Np)      # rows (alpha, g)
            Aout = np.tensordot(Tw, Z.reshape((d + 1) * G, ns * ns * Np), axes=(0, 0))
            return Aout.reshape(Np, ns, ns, Np).transpose(1, 0, 2, 3).reshape(ns * Np, ns * Np)

        Auu = contract(Ku)
        Auq = [contract(Kq[j]) for j in range(d)]
        Auh = np.zeros((ns * Np, ns * Nth))
        Ahu = np.zeros((ns * Nth, ns * Np))
        Ahq = [np.zeros((ns * Nth, ns * Np)) for _ in range(d)]
        Ahh = np.zeros((ns * Nth, ns * Nth))

    # faces
    for fl, fc in enumerate(geo.faces):
        sl = np.arange(fl * Nfn, (fl + 1) * Nfn)
        phi, psi, wf, n = fc["phi"], fc["psi"], fc["w"], list(fc["n"])
        uf = u @ phi.T                                                  # [ns, fp]
        qf = np.array([q[j] @ phi.T for j in range(d)]).transpose(1, 0, 2)   # [ns, j, fp]
        uhf = uhl[:, sl] @ psi.T
        bkind, bdata = (0, None) if bfaces is None else bfaces[fl]

        def fhat(a, b, c):
            return _A(ph.trace_flux(list(a), ph.to_list(b, 2), list(c), n, phys))

        def feq(a, b, c):
            return _A(_face_eq(list(a), ph.to_list(b, 2), list(c), n, bkind, bdata, phys))

        RU += fhat(uhf, qf, uf) @ (wf[:, None] * phi)
        RUh[:, sl] += feq(uhf, qf, uf) @ (wf[:, None] * psi)
        if not want_jac:
            continue

        def dd(fun):
            duh, dq, du = [], [], []
            for s in range(ns):
                x = uhf.astype(complex); x[s] += 1j * H
                duh.append(np.imag(fun(x, qf, uf)) / H)
            for s in range(ns):
                row = []
                for j in range(d):
                    x = qf.astype(complex); x[s, j] += 1j * H
                    row.append(np.imag(fun(uhf, x, uf)) / H)
                dq.append(row)
            for s in range(ns):
                x = uf.astype(complex); x[s] += 1j * H
                du.append(np.imag(fun(uhf, qf, x)) / H)
            return np.array(duh), np.array(dq), np.array(du)   # [s, t, fp], [s, j, t, fp], [s, t, fp]

        Fh_uh, Fh_q, Fh_u = dd(fhat)
        E_uh, E_q, E_u = dd(feq)

        def sand(Lt, D, Rt):
            # out[t, i, s, j] = sum_fp w Lt[fp, i] D[s, t, fp] Rt[fp, j]
            return np.einsum("pi,stp,pj->tisj", wf[:, None] * Lt, D, Rt)

        cols_h = (np.arange(ns)[:, None] * Nth + sl[None, :]).ravel()
        Auu += sand(phi, Fh_u, phi).reshape(ns * Np, ns * Np)
        for j in range(d):
            Auq[j] += sand(phi, Fh_q[:, j], phi).reshape(ns * Np, ns * Np)
            Ahq[j][cols_h, :] += sand(psi, E_q[:, j], phi).reshape(ns * Nfn, ns * Np)
        Auh[:, cols_h] += sand(phi, Fh_uh, psi).reshape(ns * Np, ns * Nfn)
        Ahu[cols_h, :] += sand(psi, E_u, phi).reshape(ns * Nfn, ns * Np)
        Ahh[np.ix_(cols_h, cols_h)] += sand(psi, E_uh, psi).reshape(ns * Nfn, ns * Nfn)

    out["RUh"] = RUh
    out["RU"] = RU
    if want_jac:
        out.update(Auu=Auu, Auq=Auq, Auh=Auh, Ahu=Ahu, Ahq=Ahq, Ahh=Ahh)
    return out


def full_local_blocks(geo, blocks):
    """A_qq, A_qu, A_quh of eq. C312 as full matrices (q index (k, s, a))."""
    d = geo.d
    ns = d + 2
    I = np.eye(ns)
    Aqq = np.kron(np.eye(d * ns), blocks["M"])
    Aqu = np.vstack([np.kron(I, blocks["Gk"][k]) for k in range(d)])
    Aqh = np.vstack([np.kron(I, blocks["Ghk"][k]) for k in range(d)])
    Auq = np.hstack(blocks["Auq"])
    Ahq = np.hstack(blocks["Ahq"])
    return Aqq, Aqu, Aqh, Auq, Ahq
