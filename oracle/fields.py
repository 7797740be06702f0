"""Closed-form fields: manufactured solution, Couette profile, Taylor-Green vortex.

Test infrastructure only (see ``oracle/__init__``).

Each field returns conserved variables u(x) [n_s, ...] for coordinates x [d, ...]
(complex x allowed: every expression is analytic), and where needed the
gradient q(x) [n_s, d, ...] written out by hand from the primitive fields.
"""
import numpy as np

from . import physics


def conserved(rho, v, P, gamma):
    d = len(v)
    u = [rho] + [rho * v[k] for k in range(d)]
    u.append(P / (gamma - 1.0) + 0.5 * rho * sum(v[k] * v[k] for k in range(d)))
    return np.array(u)


def conserved_grad(rho, grho, v, gv, P, gP, gamma):
    """d u_s / d x_j from primitive values and gradients (product rule)."""
    d = len(v)
    q = []
    q.append([grho[j] for j in range(d)])
    for k in range(d):
        q.append([grho[j] * v[k] + rho * gv[k][j] for j in range(d)])
    ke = 0.5 * sum(v[k] * v[k] for k in range(d))
    q.append([gP[j] / (gamma - 1.0) + grho[j] * ke + rho * sum(v[k] * gv[k][j] for k in range(d))
              for j in range(d)])
    return np.array(q)


# ---- manufactured solution (config "3D MMS cube" and its 2D analogue) -------------
# rho = 1 + A prod_k sin(pi x_k); v_k = V sin(2 pi x_k) (k even) / V cos(2 pi x_k) (k odd);
# P = 1/gamma + Pa cos(pi sum_k x_k)

def mms_primitives(x, par, gamma):
    A, V, Pa = par[0], par[1], par[2]
    d = x.shape[0]
    s = [np.sin(np.pi * x[k]) for k in range(d)]
    c = [np.cos(np.pi * x[k]) for k in range(d)]
    prod = 1.0
    for k in range(d):
        prod = prod * s[k]
    rho = 1.0 + A * prod
    grho = []
    for j in range(d):
        g = A * np.pi * c[j]
        for k in range(d):
            if k != j:
                g = g * s[k]
        grho.append(g)
    v, gv = [], []
    for k in range(d):
        if k % 2 == 0:
            v.append(V * np.sin(2 * np.pi * x[k]))
            dk = V * 2 * np.pi * np.cos(2 * np.pi * x[k])
        else:
            v.append(V * np.cos(2 * np.pi * x[k]))
            dk = -V * 2 * np.pi * np.sin(2 * np.pi * x[k])
        gv.append([dk if j == k else 0.0 * dk for j in range(d)])
    sx = sum(x[k] for k in range(d))
    P = 1.0 / gamma + Pa * np.cos(np.pi * sx)
    gP = [-Pa * np.pi * np.sin(np.pi * sx) for _ in range(d)]
    return rho, grho, v, gv, P, gP


def mms_u(x, par, gamma):
    rho, grho, v, gv, P, gP = mms_primitives(x, par, gamma)
    return conserved(rho, v, P, gamma)


def mms_q(x, par, gamma):
    rho, grho, v, gv, P, gP = mms_primitives(x, par, gamma)
    return conserved_grad(rho, grho, v, gv, P, gP, gamma)


def flux_source(x, ufun, qfun, phys):
    """f = div(F + G)(u_ex, grad u_ex): the source that makes the closed-form u_ex a steady
    solution.  The divergence is taken by the complex step in each coordinate direction."""
    d = x.shape[0]
    gamma = phys["gamma"]
    f = 0.0
    for k in range(d):
        xp = x.astype(complex)
        xp[k] = xp[k] + 1j * physics.CS_H
        u = ufun(xp)
        q = qfun(xp)
        Fi = physics.inviscid_flux(u, gamma)
        Gv = physics.viscous_flux(u, q, phys)
        f = f + np.imag(np.array([Fi[s][k] + Gv[s][k] for s in range(len(Fi))])) / physics.CS_H
    return f


def mms_source(x, par, phys):
    """The manufactured solution's source (flux_source of mms_u)."""
    g = phys["gamma"]
    return flux_source(x, lambda y: mms_u(y, par, g), lambda y: mms_q(y, par, g), phys)


# ---- compressible Couette flow with a source term (Sec. 5.1, eq. CF0) -------------
# Reading in acoustic units (c = 1 at T = 1): v_1 = M x_2 log(1 + x_2), v_2 = v_3 = 0,
# T = a + x_2 (b - a) + K x_2 (1 - x_2), P = 1/gamma (so rho = 1/T); par = (M, a, b, K).
# The paper's printed source term is garbled; the source here is the divergence of the
# fluxes of this state (flux_source), which is what the paper says it is.

def couette3d_primitives(x, par, gamma):
    M, a, b, K = par[0], par[1], par[2], par[3]
    d = x.shape[0]
    y = x[1]
    T = a + y * (b - a) + K * y * (1.0 - y)
    dT = (b - a) + K * (1.0 - 2.0 * y)
    rho = 1.0 / T
    grho = [0.0 * y for _ in range(d)]
    grho[1] = -dT / (T * T)
    v = [M * y * np.log(1.0 + y)] + [0.0 * y for _ in range(d - 1)]
    gv = [[0.0 * y for _ in range(d)] for _ in range(d)]
    gv[0][1] = M * (np.log(1.0 + y) + y / (1.0 + y))
    P = 1.0 / gamma + 0.0 * y
    gP = [0.0 * y for _ in range(d)]
    return rho, grho, v, gv, P, gP


def couette3d_u(x, par, gamma):
    rho, grho, v, gv, P, gP = couette3d_primitives(x, par, gamma)
    return conserved(rho, v, P, gamma)


def couette3d_q(x, par, gamma):
    rho, grho, v, gv, P, gP = couette3d_primitives(x, par, gamma)
    return conserved_grad(rho, grho, v, gv, P, gP, gamma)


def couette3d_source(x, par, phys):
    g = phys["gamma"]
    return flux_source(x, lambda y: couette3d_u(y, par, g), lambda y: couette3d_q(y, par, g), phys)


# ---- Couette flow between isothermal walls (config "2D Couette") ------------------

def couette_exact(y, uw, Tw, P0, phys):
    """Steady Couette profile with constant mu, kappa in these units.

    x-momentum: tau_xy constant -> v_1 = u_w y.  Energy: tau_xy v_1 - phi_y constant
    with phi = -(1/(Re Pr (gamma-1))) dT/dy -> T = T_w + (Pr (gamma-1)/2) u_w^2 y (1-y).
    Pressure constant, rho = gamma P0 / T.
    Returns rho, v1, T.
    """
    g, Pr = phys["gamma"], phys["Pr"]
    T = Tw + 0.5 * Pr * (g - 1.0) * uw * uw * y * (1.0 - y)
    return g * P0 / T, uw * y, T


# ---- Taylor-Green vortex initial condition (Sec. 5.3, eq. TGV0) -------------------

def tgv_u(x, V0, gamma):
    """Isothermal TGV initial state with L = rho0 = 1, P0 = 1/gamma."""
    P0 = 1.0 / gamma
    v1 = V0 * np.sin(x[0]) * np.cos(x[1]) * np.cos(x[2])
    v2 = -V0 * np.cos(x[0]) * np.sin(x[1]) * np.cos(x[2])
    v3 = 0.0 * x[0]
    P = P0 + (V0 * V0 / 16.0) * (np.cos(2 * x[0]) + np.cos(2 * x[1])) * (np.cos(2 * x[2]) + 2.0)
    rho = P / P0
    return conserved(rho, [v1, v2, v3], P, gamma)


def uniform_u(d, rho, v, T, gamma):
    """Constant conserved state from rho, v, T (gamma P = rho T)."""
    P = rho * T / gamma
    return conserved(rho, list(v[:d]), P, gamma)


# ---- flow past a sphere: initial state (input recipe, not from the paper) ----------

SHELL_BLEND = (0.6, 1.0)


def shell_initial_u(x, rho, v, T, gamma):
    """Free stream (rho, v, T) with the velocity scaled by a smooth step of r = |x|: zero
    for r <= 0.6, one for r >= 1, 3 s^2 - 2 s^3 of s = (r - 0.6) / 0.4 between."""
    r = np.sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2])
    s = np.clip((r - SHELL_BLEND[0]) / (SHELL_BLEND[1] - SHELL_BLEND[0]), 0.0, 1.0)
    beta = s * s * (3.0 - 2.0 * s)
    P = rho * T / gamma
    return conserved(rho + 0.0 * r, [v[k] * beta for k in range(3)], P + 0.0 * r, gamma)
