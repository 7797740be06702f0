"""Pointwise physics of the nondimensional compressible Navier-Stokes system.

Test infrastructure only (see ``oracle/__init__``).

Conventions (Sec. 2.1, eqs. C4-C6):
  * state u = (rho, rho v_1..rho v_d, rho E), n_s = d + 2 components;
  * gradient q[s][k] = d u_s / d x_k;
  * acoustic scaling: gamma P = rho T, so the sound speed is c = sqrt(T);
  * P = (gamma - 1) (rho E - rho |v|^2 / 2) (perfect gas, E = e + |v|^2/2);
  * tau = (mu / Re_c) (grad v + grad v^T - (2/d) div v I), lambda = -2/d;
  * heat flux phi = -(kappa / (Re_c Pr (gamma - 1))) grad T, mu = kappa = 1.
    (The printed coefficient kappa/R is inconsistent with the printed
    thermodynamic relations; this is the reading that makes phi equal to
    -(1/(Re_c Pr)) grad h with h = c_p T the enthalpy in these units.)
  * F = [rho v, rho v (x) v + P I, rho H v], G = -[0, tau, tau v - phi].

Every function works on Python lists of "scalars": numpy arrays (real or complex,
any shape) or the forward-mode ``Dual`` below, so that the same expressions can
be differentiated twice (Dual inside, complex step outside).  |x| is written so
that its derivative is sign(x) with sign(0) = 0; likewise the speed |v| = sqrt(v.v)
has derivative v/|v| and 0 at v = 0 (sqrt0).
"""
import numpy as np

CS_H = 1e-30


class Dual:
    """Forward-mode number v + sum_i d[i] eps_i (eps_i eps_j = 0)."""
    __slots__ = ("v", "d")

    def __init__(self, v, d):
        self.v = v
        self.d = d

    def __add__(a, b):
        if isinstance(b, Dual):
            return Dual(a.v + b.v, a.d + b.d)
        return Dual(a.v + b, a.d)

    __radd__ = __add__

    def __sub__(a, b):
        if isinstance(b, Dual):
            return Dual(a.v - b.v, a.d - b.d)
        return Dual(a.v - b, a.d)

    def __rsub__(a, b):
        return Dual(b - a.v, -a.d)

    def __neg__(a):
        return Dual(-a.v, -a.d)

    def __mul__(a, b):
        if isinstance(b, Dual):
            return Dual(a.v * b.v, a.d * b.v + a.v * b.d)
        return Dual(a.v * b, a.d * b)

    __rmul__ = __mul__

    def __truediv__(a, b):
        if isinstance(b, Dual):
            return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v))
        return Dual(a.v / b, a.d / b)

    def __rtruediv__(a, b):
        return Dual(b / a.v, -b * a.d / (a.v * a.v))


def sqrt(x):
    if isinstance(x, Dual):
        s = np.sqrt(x.v)
        return Dual(s, x.d / (2.0 * s))
    return np.sqrt(x)


def sqrt0(x):
    """sqrt of a sum of squares x = v.v with derivative 0 where x vanishes: the magnitude |v|
    at v = 0 (not differentiable there) takes the derivative 0, as |x| does at x = 0.  Under
    the complex step at v = 0, x = -(h dv)^2 has a non-positive real part, and the result is 0."""
    if isinstance(x, Dual):
        s = sqrt0(x.v)
        pos = np.real(x.v) > 0.0
        return Dual(s, np.where(pos, x.d / (2.0 * np.where(pos, s, 1.0)), 0.0 * x.d))
    x = np.asarray(x)
    pos = np.real(x) > 0.0
    return np.where(pos, np.sqrt(np.where(pos, x, 1.0)), 0.0 * x)


def sign_of(x):
    v = x.v if isinstance(x, Dual) else x
    return np.sign(np.real(v))


def cabs(x):
    """|x| with derivative sign(Re x) (0 at x == 0)."""
    return x * sign_of(x)


def primitives(u, gamma):
    """rho, v[d], E, P, T from the conserved state (Sec. 2.1 thermodynamic relations)."""
    d = len(u) - 2
    rho = u[0]
    v = [u[1 + i] / rho for i in range(d)]
    E = u[d + 1] / rho
    ke = 0.5 * sum(v[i] * v[i] for i in range(d))
    P = (gamma - 1.0) * (u[d + 1] - rho * ke)
    T = gamma * P / rho
    return rho, v, E, P, T


def inviscid_flux(u, gamma):
    """F(u)[s][k] of eq. C5a."""
    d = len(u) - 2
    rho, v, E, P, T = primitives(u, gamma)
    F = [[None] * d for _ in range(d + 2)]
    for k in range(d):
        F[0][k] = u[1 + k]
        for i in range(d):
            F[1 + i][k] = u[1 + i] * v[k] + (P if i == k else 0.0)
        F[d + 1][k] = (u[d + 1] + P) * v[k]
    return F


def viscous_flux(u, q, phys):
    """G(u, q)[s][k] of eq. C5b with tau and phi of eq. C6 (mu = kappa = 1)."""
    gamma, Re, Pr = phys["gamma"], phys["Re"], phys["Pr"]
    d = len(u) - 2
    rho, v, E, P, T = primitives(u, gamma)
    # gv[i][k] = d v_i / d x_k and grad T, from q = grad u by the chain rule
    gv = [[(q[1 + i][k] - v[i] * q[0][k]) / rho for k in range(d)] for i in range(d)]
    gT = []
    for k in range(d):
        gE = (q[d + 1][k] - E * q[0][k]) / rho
        vgv = sum(v[i] * gv[i][k] for i in range(d))
        gT.append(gamma * (gamma - 1.0) * (gE - vgv))
    div = sum(gv[i][i] for i in range(d))
    G = [[0.0 * rho for _ in range(d)] for _ in range(d + 2)]
    for k in range(d):
        phi_k = -gT[k] / (Re * Pr * (gamma - 1.0))
        work = 0.0
        for i in range(d):
            tau_ik = (gv[i][k] + gv[k][i]) / Re
            if i == k:
                tau_ik = tau_ik - (2.0 / d) * div / Re
            G[1 + i][k] = -tau_ik
            work = work + tau_ik * v[i]
        G[d + 1][k] = -(work - phi_k)
    return G


def s_vis(d, phys):
    """Diagonal of S^vis (Sec. 2.3): (1/Re_c) diag(0, 1..1, 1/((gamma-1) Pr)).

    The printed factor M_inf^2 belongs to a free-stream velocity scaling; under
    the acoustic scaling used here the reference speed is c_inf (M_ref = 1).
    """
    g = phys["gamma"]
    out = [1.0 / phys["Re"]] * (d + 2)
    out[0] = 0.0
    out[d + 1] = 1.0 / ((g - 1.0) * phys["Pr"] * phys["Re"])
    return out


def trace_flux(uh, q, u, n, phys):
    """Interior numerical flux (F^ + G^) n (eq. "num fluxes", Sec. 2.3).

    (F(uh) + G(uh, q)) n + S(uh) (u - uh),  S = lambda_max I + S^vis,
    lambda_max = |v^.n| + c^ at the trace state uh (reading: the largest
    eigenvalue magnitude of dF_n/du at uh).  n is a length-d list of numbers.
    """
    d = len(uh) - 2
    gamma = phys["gamma"]
    F = inviscid_flux(uh, gamma)
    G = viscous_flux(uh, q, phys)
    rho, v, E, P, T = primitives(uh, gamma)
    vn = sum(v[k] * n[k] for k in range(d))
    lam = cabs(vn) + sqrt(T)
    sv = s_vis(d, phys)
    return [sum((F[s][k] + G[s][k]) * n[k] for k in range(d)) + (lam + sv[s]) * (u[s] - uh[s])
            for s in range(d + 2)]


def wall_operator(uh, u, wall_T, wall_v, gamma):
    """Boundary trace operator B^ for an isothermal (moving) no-slip wall.

    The paper states only that B^ imposes the boundary condition through the
    hybrid variable.  Reading: trace density follows the interior density, trace
    velocity is the wall velocity, trace temperature the wall temperature:
      B^ = (rho^ - rho, rho^ v^ - rho^ v_w, rho^ E^ - rho^ (e_w + |v_w|^2/2)),
    with e_w = T_w / (gamma (gamma - 1)).
    """
    d = len(uh) - 2
    ew = wall_T / (gamma * (gamma - 1.0))
    B = [uh[0] - u[0]]
    for i in range(d):
        B.append(uh[1 + i] - uh[0] * wall_v[i])
    B.append(uh[d + 1] - uh[0] * (ew + 0.5 * sum(w * w for w in wall_v[:d])))
    return B


def flux_jacobian_apply(uh, du, n, gamma, delta=None):
    """A_n(uh) du, or |A_n|_delta(uh) du when delta is given: the normal inviscid flux Jacobian
    A_n = dF(uh).n / du applied through its eigen-decomposition (acoustic waves v_n -/+ c with
    right eigenvectors (1, v -/+ c n, H -/+ c v_n), the remaining d waves at v_n).  A jump du
    splits into acoustic strengths a1, a5 = (dp -/+ rho c dv_n) / (2 c^2), with dp and dv_n the
    pressure and normal-velocity perturbations of du, and a remainder that moves at v_n.
    |lambda|_delta = sqrt(lambda^2 + (delta c)^2): analytic, so the complex step differentiates
    it, and nonzero where the flow is tangent to the boundary."""
    d = len(uh) - 2
    rho, v, E, P, T = primitives(uh, gamma)
    c = sqrt(T)
    H = E + P / rho
    vn = sum(v[k] * n[k] for k in range(d))
    ke = 0.5 * sum(v[k] * v[k] for k in range(d))
    dp = (gamma - 1.0) * (du[d + 1] - sum(v[k] * du[1 + k] for k in range(d)) + ke * du[0])
    dvn = (sum(du[1 + k] * n[k] for k in range(d)) - vn * du[0]) / rho
    a1 = (dp - rho * c * dvn) / (2.0 * c * c)
    a5 = (dp + rho * c * dvn) / (2.0 * c * c)
    r1 = [1.0] + [v[k] - c * n[k] for k in range(d)] + [H - c * vn]
    r5 = [1.0] + [v[k] + c * n[k] for k in range(d)] + [H + c * vn]
    if delta is None:
        l1, l2, l5 = vn - c, vn, vn + c
    else:
        dc2 = (delta * c) * (delta * c)
        l1, l2, l5 = sqrt((vn - c) * (vn - c) + dc2), sqrt(vn * vn + dc2), sqrt((vn + c) * (vn + c) + dc2)
    return [l2 * du[s] + (l1 - l2) * a1 * r1[s] + (l5 - l2) * a5 * r5[s] for s in range(d + 2)]


FARFIELD_DELTA = 0.05


def farfield_operator(uh, u, uinf, n, gamma, delta=FARFIELD_DELTA):
    """Characteristic far-field trace operator (reading of B^ in Sec. 2.3, which gives no formula):
    B^ = A_n^+(uh) (u - uh) - A_n^-(uh) (u_inf - uh), A_n^+- = (A_n +- |A_n|_delta) / 2: outgoing
    characteristics of uh follow the interior state, incoming ones the free stream."""
    d = len(uh) - 2
    du_i = [u[s] - uh[s] for s in range(d + 2)]
    du_o = [uinf[s] - uh[s] for s in range(d + 2)]
    Ai, Ao = flux_jacobian_apply(uh, du_i, n, gamma), flux_jacobian_apply(uh, du_o, n, gamma)
    Bi, Bo = flux_jacobian_apply(uh, du_i, n, gamma, delta), flux_jacobian_apply(uh, du_o, n, gamma, delta)
    return [0.5 * (Ai[s] + Bi[s]) - 0.5 * (Ao[s] - Bo[s]) for s in range(d + 2)]


def supg_tau(u, h, p, phys):
    """Scalar SUPG coefficient (reading of Sec. 2.3, which defines tau only by reference).

    tau = ((2 (|v| + c) p / h)^2 + (4 p^2 nu / h^2)^2)^(-1/2),  nu = 1 / (Re_c rho);
    |v| through sqrt0 (derivative 0 at v = 0, e.g. a gas at rest).
    """
    rho, v, E, P, T = primitives(u, phys["gamma"])
    d = len(v)
    speed = sqrt0(sum(v[i] * v[i] for i in range(d))) + sqrt(T)
    a = 2.0 * p / h * speed
    b = 4.0 * p * p / (phys["Re"] * h * h) / rho
    return 1.0 / sqrt(a * a + b * b)


def flux_divergence_and_A(u, gu, q, gq, phys):
    """Strong-form pieces at a point, by forward-mode derivatives of the fluxes.

    Returns (div, A) where
      div[s] = sum_l d/dx_l (F + G)_{s,l}(u(x), q(x)) by the chain rule
               (directional derivative of column l along (d_l u, d_l q)),
      A[k][t][s] = d F_{t,k} / d u_s (inviscid flux Jacobian).
    gu[s][l] = d_l u_s, gq[s][j][l] = d_l q_{s,j}.  Works for complex inputs.
    """
    ns = len(u)
    d = ns - 2
    nd = ns + d
    z = 0.0 * (u[0] + q[0][0])

    def seed(val, dirs):
        D = np.zeros((nd,) + np.shape(val), dtype=np.result_type(val, z, *[w for _, w in dirs]))
        for i, w in dirs:
            D[i] = D[i] + w
        return Dual(val + z, D)

    ud = [seed(u[s], [(s, 1.0)] + [(ns + l, gu[s][l]) for l in range(d)]) for s in range(ns)]
    qd = [[seed(q[s][j], [(ns + l, gq[s][j][l]) for l in range(d)]) for j in range(d)] for s in range(ns)]
    F = inviscid_flux(ud, phys["gamma"])
    G = viscous_flux(ud, qd, phys)
    div = [sum(F[s][l].d[ns + l] + G[s][l].d[ns + l] for l in range(d)) for s in range(ns)]
    A = [[[F[t][k].d[s] for s in range(ns)] for t in range(ns)] for k in range(d)]
    return div, A


def to_list(x, depth):
    """Split the leading ``depth`` axes of an array into nested lists."""
    if depth == 0:
        return x
    return [to_list(x[i], depth - 1) for i in range(x.shape[0])]


def to_array(x):
    return np.array(x)
