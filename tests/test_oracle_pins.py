"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests uses a GPU.  Each pin targets a part of the oracle where a
plausible mistake (dropped term, wrong sign, transposed block, wrong index) would
show: closed forms, exact identities between the paper's own alternative
formulas, brute force on tiny inputs, the paper's printed DOF tables, and
convergence rates.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import assemble as asm
from oracle import fields, physics as ph, simplex as sx, solve, space

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- spaces (Sec. 2.2)

def test_gll_points_closed_form():
    assert np.allclose(space.gll_points(1), [-1, 1])
    assert np.allclose(space.gll_points(2), [-1, 0, 1])
    assert np.allclose(space.gll_points(3), [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1])
    assert np.allclose(space.gll_points(4), [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1])


def test_lagrange_reproduces_polynomials():
    nodes = space.gll_points(3)
    x = np.linspace(-1, 1, 7)
    L, dL = space.lagrange(nodes, x)
    assert np.allclose(space.lagrange(nodes, nodes)[0], np.eye(4))
    f = lambda t: 2 * t ** 3 - t ** 2 + 0.5
    df = lambda t: 6 * t ** 2 - 2 * t
    assert np.allclose(L @ f(nodes), f(x), atol=1e-14)
    assert np.allclose(dL @ f(nodes), df(x), atol=1e-13)


def test_macro_geometry_exact_integrals():
    # box [0.2, 0.7] x [0.1, 0.4], m = 2, p = 2: integrals of polynomials of degree <= 2p+3
    g = space.MacroGeometry([0.2, 0.1], [0.7, 0.4], 2, 2)
    x, y = g.xq
    assert np.isclose(g.w.sum(), 0.5 * 0.3)
    exact = (0.7 ** 4 - 0.2 ** 4) / 4 * (0.4 ** 3 - 0.1 ** 3) / 3
    assert np.isclose(g.w @ (x ** 3 * y ** 2), exact, rtol=1e-14)
    # C0 nodal interpolation of a Q2 function is exact and its gradient too
    f = lambda X, Y: X ** 2 * Y - 3 * X * Y ** 2 + Y
    fn = f(*g.xn)
    assert np.allclose(g.T[0] @ fn, f(x, y), atol=1e-14)
    assert np.allclose(g.T[1] @ fn, 2 * x * y - 3 * y ** 2, atol=1e-13)
    assert np.allclose(g.T[2] @ fn, x ** 2 - 6 * x * y + 1, atol=1e-13)


def _simplex_nodes(n, d=3):
    from math import comb
    return comb(n + d, d)


def _tri_nodes(n):
    return (n + 1) * (n + 2) // 2


def test_dof_tables_of_the_paper():
    """The paper's DOF tables follow from: u and q C0 on each macro-element with
    (d+1)(d+2) unknowns per node, trace C0 per macro-face, independent across faces,
    n_s = 5 unknowns per trace node (Tables 1, 3, 6-8, 10)."""
    gold = json.load(open(os.path.join(GOLD, "dof_tables.json")))
    per_node = 4 * 5      # (d+1)(d+2), d = 3
    t1 = gold["table1_couette_768_elements_p3"]
    for r in t1["rows"]:
        mp = r["m"] * t1["p"]
        assert per_node * _simplex_nodes(mp) == r["local"]
        assert r["local"] * r["n_macro"] == r["total_local"]
        faces = (4 * r["n_macro"] + r["boundary_triangles"]) // 2
        assert 5 * faces * _tri_nodes(mp) == r["global"]
        assert r["n_macro"] * r["m"] ** 3 == 768
    t3 = gold["table3_couette_fixed_local"]
    for r in t3["rows"]:
        assert per_node * _simplex_nodes(t3["mp"]) == r["local"]
        assert r["local"] * r["n_macro"] == r["total_local"]
        faces = (4 * r["n_macro"] + r["boundary_triangles"]) // 2
        assert 5 * faces * _tri_nodes(t3["mp"]) == r["global"]
    t6 = gold["table6_sphere_p3"]
    bnd = []
    for r in t6["rows"]:
        mp = r["m"] * t6["p"]
        assert per_node * _simplex_nodes(mp) * r["n_macro"] == r["total_local"]
        nf, rem = divmod(r["global"], 5 * _tri_nodes(mp))
        assert rem == 0
        bnd.append(2 * nf - 4 * r["n_macro"])
    assert bnd[0] == 4 * bnd[1]          # each macro boundary triangle holds 4 element triangles
    t8 = gold["table8_tgv_mp8_periodic"]
    for r in t8["rows"]:
        assert per_node * _simplex_nodes(t8["mp"]) * r["n_macro"] == r["total_local"]
        assert 5 * (2 * r["n_macro"]) * _tri_nodes(t8["mp"]) == r["global"]


@pytest.mark.parametrize("d,m,p", [(2, 2, 2), (3, 2, 1), (2, 3, 3)])
def test_box_node_and_face_counts_brute_force(d, m, p):
    pr = W.mms(dim=d, nmac=3, m=m, p=p)
    P = solve.Problem(pr)
    g = P.geometry(4)
    pts = {tuple(np.round(x, 12)) for x in g.xn.T}
    assert len(pts) == P.Np == (m * p + 1) ** d
    # faces: enumerate unique (axis, position, tangential box) from every macro's boundary
    faces = set()
    for e in range(P.E):
        lo, hi = P.mesh.macro_box(e)
        for k in range(d):
            for side in range(2):
                key = [k, round((lo, hi)[side][k], 12)]
                key += [round(lo[j], 12) for j in range(d) if j != k]
                faces.add(tuple(key))
    assert len(faces) == P.F
    own = P.mesh.face_owners()
    assert sum(len(o) for o in own) == 2 * d * P.E


# ---------------------------------------------------------------- pointwise physics (Sec. 2.1)

@pytest.mark.parametrize("d", [2, 3])
def test_inviscid_flux_eigenvalues(d):
    rng = np.random.default_rng(3)
    g = 1.4
    for _ in range(5):
        rho, T = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
        v = rng.uniform(-0.5, 0.5, d)
        u = fields.uniform_u(d, rho, v, T, g)
        n = rng.normal(size=d)
        n /= np.linalg.norm(n)
        An = np.zeros((d + 2, d + 2))
        for s in range(d + 2):
            up = u.astype(complex)
            up[s] += 1j * ph.CS_H
            F = ph.inviscid_flux(list(up), g)
            An[:, s] = [np.imag(sum(F[t][k] * n[k] for k in range(d))) / ph.CS_H for t in range(d + 2)]
        ev = np.sort(np.linalg.eigvals(An).real)
        vn, c = v @ n, np.sqrt(T)
        assert np.allclose(ev, np.sort([vn - c] + [vn] * d + [vn + c]), atol=1e-12)


def test_viscous_flux_closed_forms():
    """Shear flow v = (a y, 0, 0) with constant rho, and a linear temperature."""
    g, Re, Pr = 1.4, 50.0, 0.72
    phys = dict(gamma=g, Re=Re, Pr=Pr)
    a, rho, T0, bT = 0.3, 1.3, 1.1, 0.2
    x = np.array([0.4, 0.25, 0.7])
    # primitives and gradients
    v = [a * x[1], 0.0, 0.0]
    gv = [[0.0, a, 0.0], [0.0] * 3, [0.0] * 3]
    T = T0 + bT * x[0]
    P = rho * T / g
    gP = [rho * bT / g, 0.0, 0.0]
    u = fields.conserved(rho, v, P, g)
    q = fields.conserved_grad(rho, [0.0] * 3, v, gv, P, gP, g)
    G = np.array(ph.viscous_flux(list(u), ph.to_list(np.array(q), 2), phys))
    tau_xy = a / Re
    assert np.isclose(G[1, 1], -tau_xy) and np.isclose(G[2, 0], -tau_xy)
    assert np.isclose(G[1, 0], 0.0, atol=1e-15) and np.isclose(G[3, 2], 0.0, atol=1e-15)
    kcoef = 1.0 / (Re * Pr * (g - 1.0))
    assert np.isclose(G[4, 0], -(0.0 - (-kcoef * bT)))             # -(tau v - phi)_x
    assert np.isclose(G[4, 1], -(tau_xy * v[0]))


@pytest.mark.parametrize("d", [2, 3])
def test_supg_tau_at_rest_has_zero_momentum_derivative(d):
    """A gas at rest (v = 0) sits on the kink of |v| in tau: the derivative of tau along every
    momentum direction is taken as 0 there (the sign(0) = 0 convention of |x|).  It equals the
    central difference (|eps| - |-eps|) / (2 eps) = 0, the complex step of the oracle returns
    it, the value is the closed form with |v| = 0, and away from rest the complex step still
    matches the central difference."""
    gamma, h, p = 1.4, 0.3, 2
    phys = dict(gamma=gamma, Re=80.0)
    rho, P = 1.1, 0.9
    for v in (np.zeros(d), 0.2 * np.ones(d)):
        u = np.array([rho] + list(rho * v) + [P / (gamma - 1.0) + 0.5 * rho * float(v @ v)])
        for k in range(d):
            uc = u.astype(complex)
            uc[1 + k] += 1j * ph.CS_H
            dcs = np.imag(ph.supg_tau(list(uc), h, p, phys)) / ph.CS_H
            eps = 1e-7
            up, um = u.copy(), u.copy()
            up[1 + k] += eps
            um[1 + k] -= eps
            dfd = (ph.supg_tau(list(up), h, p, phys) - ph.supg_tau(list(um), h, p, phys)) / (2.0 * eps)
            assert abs(dcs - dfd) <= 1e-6 * max(abs(dfd), 1e-3)
            if not v.any():
                assert dcs == 0.0
    c = np.sqrt(gamma * P / rho)
    tau0 = ph.supg_tau([rho] + [0.0] * d + [P / (gamma - 1.0)], h, p, phys)
    assert np.isclose(tau0, 1.0 / np.hypot(2.0 * p / h * c, 4.0 * p * p / (phys["Re"] * h * h * rho)), rtol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_supg_tau_limits(d):
    """The SUPG coefficient (a reading: Sec. 2.3 defines it by reference) blends the two
    textbook element time scales: h / (2 p (|v| + c)) when advection dominates and
    Re rho h^2 / (4 p^2) when diffusion does, with c the ideal-gas sound speed
    sqrt(gamma P / rho) of the conserved state.  It decreases with p, grows with h and
    is never above either time scale."""
    rng = np.random.default_rng(3 + d)
    gamma = 1.4
    rho = 0.8 + 0.4 * rng.random()
    v = rng.standard_normal(d) * 0.3
    P = 0.5 + rng.random()
    rhoE = P / (gamma - 1.0) + 0.5 * rho * float(v @ v)
    u = [rho] + list(rho * v) + [rhoE]
    c = np.sqrt(gamma * P / rho)
    h, p = 0.37, 2
    t_adv = h / (2.0 * p * (np.linalg.norm(v) + c))
    big = dict(gamma=gamma, Re=1e14)
    assert np.isclose(ph.supg_tau(u, h, p, big), t_adv, rtol=1e-9)
    small = dict(gamma=gamma, Re=1e-14)
    t_dif = small["Re"] * rho * h * h / (4.0 * p * p)
    assert np.isclose(ph.supg_tau(u, h, p, small), t_dif, rtol=1e-9)
    mid = dict(gamma=gamma, Re=50.0)
    tau = ph.supg_tau(u, h, p, mid)
    assert tau <= t_adv and tau <= mid["Re"] * rho * h * h / (4.0 * p * p)
    assert ph.supg_tau(u, h, p + 1, mid) < tau < ph.supg_tau(u, 2.0 * h, p, mid)


@pytest.mark.parametrize("d", [2, 3])
def test_numerical_flux_consistency_and_dissipation(d):
    """Numerical flux of Sec. 2.3, (F + G)(u^) n + S (u - u^): at u = u^ it is the physical
    flux; for a jump it adds S (u - u^) with the dissipative sign, whose inviscid part is
    the largest |eigenvalue| of dF_n/du at u^ (found numerically, by complex-step columns)
    and whose viscous part is the viscous flux's own coefficients: 0 for density, the
    shear coefficient 1/Re for momentum, the heat-conduction coefficient for energy."""
    rng = np.random.default_rng(11 + d)
    g, Re, Pr = 1.4, 40.0, 0.72
    phys = dict(gamma=g, Re=Re, Pr=Pr)
    rho, T = rng.uniform(0.6, 1.5), rng.uniform(0.6, 1.5)
    uh = fields.uniform_u(d, rho, rng.uniform(-0.4, 0.4, d), T, g)
    q = rng.normal(size=(d + 2, d)) * 0.1
    n = rng.normal(size=d)
    n /= np.linalg.norm(n)
    nl, ql = list(n), ph.to_list(q, 2)
    F = np.array(ph.inviscid_flux(list(uh), g))
    G = np.array(ph.viscous_flux(list(uh), ql, phys))
    phys_flux = (F + G) @ n
    assert np.allclose(ph.trace_flux(list(uh), ql, list(uh), nl, phys), phys_flux, atol=1e-14)
    An = np.zeros((d + 2, d + 2))
    for c in range(d + 2):
        up = uh.astype(complex)
        up[c] += 1j * ph.CS_H
        Fc = ph.inviscid_flux(list(up), g)
        An[:, c] = [np.imag(sum(Fc[t][k] * n[k] for k in range(d))) / ph.CS_H for t in range(d + 2)]
    lam = np.abs(np.linalg.eigvals(An)).max()
    visc = np.array([0.0] + [1.0 / Re] * d + [1.0 / (Re * Pr * (g - 1.0))])
    for s in range(d + 2):
        du = np.zeros(d + 2)
        du[s] = 1e-3 * (1 + s)
        jump = np.array(ph.trace_flux(list(uh), ql, list(uh + du), nl, phys)) - phys_flux
        expect = np.zeros(d + 2)
        expect[s] = (lam + visc[s]) * du[s]
        assert np.allclose(jump, expect, rtol=1e-10, atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_farfield_operator_against_eigendecomposition(d):
    """The closed-form A_n and |A_n|_delta of the far-field operator against the flux Jacobian
    taken by the complex step of F(u).n and decomposed by numpy.linalg.eig (independent of the
    closed form), and the operator's defining properties: zero when u = uh = u_inf, and for a
    constant coefficient state the trace it defines takes the outgoing characteristics of u and
    the incoming ones of u_inf (the solution of B^ = 0 with A_n frozen is
    |A|^-1 (A^+ u - A^- u_inf))."""
    g = 1.4
    rng = np.random.default_rng(d)
    rho, v, T = 1.1, rng.uniform(-0.3, 0.3, d), 0.9
    uh = fields.uniform_u(d, rho, v, T, g)
    n = rng.normal(size=d)
    n = n / np.linalg.norm(n)
    A = np.zeros((d + 2, d + 2))
    for j in range(d + 2):
        x = [complex(a) for a in uh]
        x[j] += 1j * ph.CS_H
        F = ph.inviscid_flux(x, g)
        A[:, j] = [np.imag(sum(F[s][k] * n[k] for k in range(d))) / ph.CS_H for s in range(d + 2)]
    lam, V = np.linalg.eig(A)
    lam, V = lam.real, V.real
    c = np.sqrt(T)
    absA = V @ np.diag(np.sqrt(lam ** 2 + (ph.FARFIELD_DELTA * c) ** 2)) @ np.linalg.inv(V)
    du = rng.normal(size=d + 2)
    assert np.allclose(ph.flux_jacobian_apply(list(uh), list(du), list(n), g), A @ du, rtol=1e-12, atol=1e-12)
    assert np.allclose(ph.flux_jacobian_apply(list(uh), list(du), list(n), g, ph.FARFIELD_DELTA), absA @ du,
                       rtol=1e-12, atol=1e-12)
    assert np.allclose(ph.farfield_operator(list(uh), list(uh), list(uh), list(n), g), 0.0, atol=1e-15)
    uin = uh + 0.01 * rng.normal(size=d + 2)
    uinf = uh + 0.01 * rng.normal(size=d + 2)
    Ap, Am = 0.5 * (A + absA), 0.5 * (A - absA)
    ut = np.linalg.solve(absA, Ap @ uin - Am @ uinf)
    B = lambda w: np.array([a + b for a, b in zip(Ap @ (uin - w), -(Am @ (uinf - w)))])
    assert np.allclose(B(ut), 0.0, atol=1e-14)
    assert np.allclose(ph.farfield_operator(list(uh), list(uin), list(uinf), list(n), g),
                       Ap @ (uin - uh) - Am @ (uinf - uh), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_wall_operator_vanishes_on_the_wall_state(d):
    """B^ of an isothermal moving wall is zero exactly when the trace state has the
    interior density, the wall velocity and the wall temperature (ideal gas with
    gamma P = rho T), and not otherwise."""
    rng = np.random.default_rng(5 + d)
    g = 1.4
    u = fields.uniform_u(d, 1.1, rng.uniform(-0.3, 0.3, d), 0.9, g)
    wall_v = list(rng.uniform(-0.2, 0.2, d)) + [0.0] * (3 - d)
    wall_T = 1.3
    uh = fields.uniform_u(d, u[0], np.array(wall_v[:d]), wall_T, g)
    assert np.allclose(ph.wall_operator(list(uh), list(u), wall_T, wall_v, g), 0.0, atol=1e-14)
    for s in range(d + 2):
        up = uh.copy()
        up[s] += 1e-3
        assert np.abs(ph.wall_operator(list(up), list(u), wall_T, wall_v, g)).max() > 1e-5


# ---------------------------------------------------------------- residual and Jacobian

def _uniform_state(P, u0):
    u = np.repeat(u0[None, :, None], P.E, 0).repeat(P.Np, 2)
    q = np.zeros((P.E, P.d, P.ns, P.Np))
    uh = np.tile(np.repeat(u0[:, None], P.Nfn, 1).reshape(-1), P.F)
    return u, q, uh


@pytest.mark.parametrize("d,p", [(2, 2), (3, 1)])
def test_free_stream_preservation(d, p):
    pr = W.periodic_uniform(dim=d, nmac=2, m=2, p=p)
    P = solve.Problem(pr)
    u, q, uh = _uniform_state(P, solve.uniform_from_par(pr))
    _, _, nrm, _ = solve.global_assemble(P, u, q, uh, want_jac=False)
    assert nrm["RF"] < 1e-13
    # the same state with Dirichlet data equal to it on every boundary
    pr2 = dict(pr, periodic=[0, 0, 0], bc=[W.BC_DIRICHLET] * 6)
    P2 = solve.Problem(pr2)
    u, q, uh = _uniform_state(P2, solve.uniform_from_par(pr2))
    _, _, nrm, _ = solve.global_assemble(P2, u, q, uh, want_jac=False)
    assert nrm["RF"] < 1e-13


def _whole_residual_jacobian(P, geo, e, ue, qe, uhl, tt, src, bf, cols=None):
    def res(uu, qq, hh):
        b = asm.assemble_macro(geo, P.phys, uu, qq, hh, tt, src, bf, want_jac=False)
        return np.concatenate([b["RU"].ravel(), b["RUh"].ravel()])
    parts = [ue, qe, uhl]
    sizes = [x.size for x in parts]
    ncol = sum(sizes)
    cols = range(ncol) if cols is None else cols
    out = {}
    for c in cols:
        which = 0 if c < sizes[0] else (1 if c < sizes[0] + sizes[1] else 2)
        off = c - sum(sizes[:which])
        args = [x.astype(complex) for x in parts]
        flat = args[which].reshape(-1)
        flat[off] += 1j * ph.CS_H
        out[c] = np.imag(res(*args)) / ph.CS_H
    return out


@pytest.mark.parametrize("case", ["mms2d", "couette2d", "mms3d", "sphere", "simplex2d", "simplex3d"])
def test_jacobian_equals_complex_step_of_residual(case):
    """Every Newton block of eq. C312 equals the derivative of the residual (SUPG on,
    DIRK time term on), random state: catches any dropped or mis-signed term."""
    if case == "mms2d":
        pr, e, cols = W.mms(dim=2, nmac=2, m=2, p=2), 3, None
    elif case == "couette2d":
        pr, e, cols = W.couette2d(nmac=2, m=2, p=2), 1, None
    elif case == "mms3d":
        pr, e = W.mms(dim=3, nmac=2, m=2, p=1), 5
        cols = list(np.random.default_rng(0).choice(135 + 405 + 270, 36, replace=False))
    elif case == "sphere":   # curved macro touching the wall and the far field
        pr, e = W.sphere(nq=2, nr=1, m=1, p=2), 5
        cols = list(np.random.default_rng(0).choice(135 + 405 + 270, 36, replace=False))
    elif case == "simplex2d":   # P_2 on a twice-refined triangle at the Dirichlet boundary
        pr, e, cols = _simplex(W.mms(dim=2, nmac=2, m=2, p=2)), 1, None
    else:   # P_1 on a twice-refined tetrahedron (Nu 50, Nq 150, Nt 120)
        pr, e = _simplex(W.mms(dim=3, nmac=1, m=2, p=1)), 2
        cols = list(np.random.default_rng(0).choice(50 + 150 + 120, 36, replace=False))
    P = solve.Problem(pr)
    u, q, uh = W.random_state(pr, 7)
    geo = P.geometry(e)
    bf, src = P.bfaces(e, geo), P.source(geo)
    ue, qe, uhl = u[e], q[e], P.local_trace(e, uh)
    tt = dict(coef=0.7, hist=0.05 * np.ones_like(ue), supg_time=True)
    blk = asm.assemble_macro(geo, P.phys, ue, qe, uhl, tt, src, bf)
    Ja = np.block([[blk["Auu"], np.hstack(blk["Auq"]), blk["Auh"]],
                   [blk["Ahu"], np.hstack(blk["Ahq"]), blk["Ahh"]]])
    Jc = _whole_residual_jacobian(P, geo, e, ue, qe, uhl, tt, src, bf, cols)
    scale = np.abs(Ja).max()
    for c, col in Jc.items():
        assert np.abs(col - Ja[:, c]).max() <= 1e-12 * scale, c
    # R_Q is linear: its blocks are the mass, lifting and face matrices
    Aqq, Aqu, Aqh, _, _ = asm.full_local_blocks(geo, blk)
    RQ = Aqq @ qe.reshape(-1) + Aqu @ ue.reshape(-1) + Aqh @ uhl.reshape(-1)
    assert np.allclose(RQ, blk["RQ"].reshape(-1), atol=1e-14)


# ---------------------------------------------------------------- condensation (Sec. 3.2-3.3)

@pytest.fixture(scope="module")
def small2d():
    pr = W.mms(dim=2, nmac=2, m=2, p=2)
    P = solve.Problem(pr)
    u, q, uh = W.random_state(pr, 11)
    blks, geos, nrm, _ = solve.global_assemble(P, u, q, uh)
    cond = [solve.condense_second_layer(geos[e], blks[e], shift=0.3) for e in range(P.E)]
    return P, blks, geos, cond


def test_one_layer_equals_second_layer(small2d):
    P, blks, geos, cond = small2d
    for e in range(P.E):
        A1, b1 = solve.condense_one_layer(geos[e], blks[e], shift=0.3)
        c = cond[e]
        SinvC = np.linalg.solve(c["S"], c["C"])
        A2 = c["B"] @ SinvC + c["D"]
        assert np.abs(A1 - A2).max() <= 1e-11 * np.abs(A1).max()
        assert np.abs(b1 - c["bhat"]).max() <= 1e-11 * max(np.abs(b1).max(), 1e-300)


def test_algorithm2_equals_explicit_matrix(small2d):
    P, blks, geos, cond = small2d
    A = solve.explicit_trace_matrix(P, cond)
    x = W.random_vector(A.shape[0], 5)
    assert np.allclose(solve.apply_trace(P, cond, x), A @ x, rtol=1e-12, atol=1e-13 * np.abs(A).max())


def _monolithic(P, blks, geos, shift):
    """The global block system of eq. C312 assembled densely (all macros)."""
    ns, Np, d = P.ns, P.Np, P.d
    nQ, nU = d * ns * Np, ns * Np
    nloc = nQ + nU
    nT = P.F * ns * P.Nfn
    N = P.E * nloc + nT
    A = np.zeros((N, N))
    r = np.zeros(N)
    for e in range(P.E):
        Aqq, Aqu, Aqh, Auq, Ahq = asm.full_local_blocks(geos[e], blks[e])
        Auu = blks[e]["Auu"] + shift * np.kron(np.eye(ns), blks[e]["M"])
        o = e * nloc
        eps = P.E * nloc + P.maps[e].reshape(-1)
        A[o:o + nQ, o:o + nQ] = Aqq
        A[o:o + nQ, o + nQ:o + nloc] = Aqu
        A[o + nQ:o + nloc, o:o + nQ] = Auq
        A[o + nQ:o + nloc, o + nQ:o + nloc] = Auu
        A[np.ix_(np.arange(o, o + nQ), eps)] += Aqh
        A[np.ix_(np.arange(o + nQ, o + nloc), eps)] += blks[e]["Auh"]
        A[np.ix_(eps, np.arange(o, o + nQ))] += Ahq
        A[np.ix_(eps, np.arange(o + nQ, o + nloc))] += blks[e]["Ahu"]
        A[np.ix_(eps, eps)] += blks[e]["Ahh"]
        r[o:o + nQ] = blks[e]["RQ"].reshape(-1)
        r[o + nQ:o + nloc] = blks[e]["RU"].reshape(-1)
        np.add.at(r, eps, blks[e]["RUh"].reshape(-1))
    return A, r


def test_condense_solve_recover_equals_monolithic(small2d):
    P, blks, geos, cond = small2d
    A, r = _monolithic(P, blks, geos, 0.3)
    x = np.linalg.solve(A, -r)
    dU, dQ, dUh, its, _ = solve.linear_step(P, blks, geos, shift=0.3, precond="direct")
    nloc = P.d * P.ns * P.Np + P.ns * P.Np
    assert np.allclose(dUh, x[P.E * nloc:], rtol=1e-9, atol=1e-11)
    for e in range(P.E):
        o = e * nloc
        assert np.allclose(dQ[e].reshape(-1), x[o:o + P.d * P.ns * P.Np], atol=1e-9)
        assert np.allclose(dU[e].reshape(-1), x[o + P.d * P.ns * P.Np:o + nloc], atol=1e-10)


@pytest.mark.parametrize("case", ["mms2d", "mms3d", "tgv3d_periodic", "sphere"])
def test_face_blocks_are_the_diagonal_of_the_assembled_trace_block(case):
    """Block-Jacobi preconditioner (Sec. 4.2): the face blocks equal the diagonal blocks
    of the global A_uhuh assembled independently through the gather maps (which carry
    each owner's face-node order), the global A_uhuh has no coupling between different
    faces (HDG traces interact only through the element unknowns), and the
    preconditioner applies the exact inverse of each block."""
    pr = {"mms2d": lambda: W.mms(dim=2, nmac=3, m=2, p=2), "mms3d": lambda: W.mms(dim=3, nmac=2, m=1, p=1),
          "tgv3d_periodic": lambda: W.tgv(nmac=2, m=1, p=1),
          "sphere": lambda: W.sphere(nq=2, nr=1, m=1, p=1)}[case]()
    P = solve.Problem(pr)
    u, q, uh = W.random_state(pr, 3)
    blks, _, _, _ = solve.global_assemble(P, u, q, uh)
    n, nb = P.F * P.ns * P.Nfn, P.ns * P.Nfn
    G = np.zeros((n, n))
    for e in range(P.E):
        m = P.maps[e].reshape(-1)
        G[np.ix_(m, m)] += blks[e]["Ahh"]
    fb = solve.face_blocks(P, blks)
    off = G.copy()
    for f in range(P.F):
        assert np.array_equal(fb[f], G[f * nb:(f + 1) * nb, f * nb:(f + 1) * nb])
        off[f * nb:(f + 1) * nb, f * nb:(f + 1) * nb] = 0.0
    assert not off.any()
    r = W.random_vector(n, 4)
    z = solve.block_jacobi(P, [solve.lu_factor(fb[f]) for f in range(P.F)], r)
    assert np.allclose(G @ z, r, rtol=0, atol=1e-10 * np.abs(r).max())


def test_inner_gmres_minimises_the_residual_over_the_krylov_space():
    """The fixed-step inner GMRES of the multi-level preconditioner (Sec. 4.2): after nu
    steps its iterate minimises |M^-1 (b - A z)| over the Krylov space K_nu(M^-1 A,
    M^-1 b) (checked against a brute-force least-squares fit on an explicit, orthonormalised
    Krylov basis), the minimum never grows with nu, and at nu = n it is the exact solution."""
    rng = np.random.default_rng(8)
    n = 12
    A = np.eye(n) * 3 + rng.standard_normal((n, n))
    Md = np.diag(2 + rng.random(n))
    Minv = lambda v: np.linalg.solve(Md, v)
    b = rng.standard_normal(n)
    B = np.linalg.solve(Md, A)
    c = Minv(b)
    prev = np.inf
    for nu in range(1, n + 1):
        z = solve.gmres_fixed(lambda v: A @ v, Minv, b, nu)
        K = np.stack([np.linalg.matrix_power(B, k) @ c for k in range(nu)], 1)
        Q, _ = np.linalg.qr(K)
        coef = np.linalg.lstsq(B @ Q, c, rcond=None)[0]
        best = np.linalg.norm(c - B @ (Q @ coef))
        res = np.linalg.norm(c - B @ z)
        assert abs(res - best) <= 1e-9 * np.linalg.norm(c)
        assert res <= prev + 1e-12
        prev = res
    assert np.allclose(z, np.linalg.solve(A, b), rtol=0, atol=1e-9 * np.abs(np.linalg.solve(A, b)).max())


def test_fgmres_equals_dense_solve(small2d):
    P, blks, geos, cond = small2d
    A = solve.explicit_trace_matrix(P, cond)
    b = solve.assemble_bhat(P, cond)
    fb = solve.face_blocks(P, blks)
    flu = [solve.lu_factor(fb[f]) for f in range(P.F)]
    M0 = lambda r: solve.block_jacobi(P, flu, r)
    for M in (M0, lambda r: solve.gmres_fixed(lambda x: A @ x, M0, r, 5)):
        x, its, res = solve.fgmres(lambda x: solve.apply_trace(P, cond, x), M, b, rtol=1e-13, restart=20)
        assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-11)


def test_gmres_left_equals_dense_solve_and_minimises_the_preconditioned_residual(small2d):
    """Sec. 4.2 baseline (GMRES left-preconditioned by the face blocks): converges to the
    dense solve of the explicit trace matrix, and after k steps of one cycle its iterate
    minimises |Minv (b - A x)| over span{Minv b, (Minv A) Minv b, ...} (brute-force
    least squares on the explicit Krylov basis)."""
    P, blks, geos, cond = small2d
    A = solve.explicit_trace_matrix(P, cond)
    b = solve.assemble_bhat(P, cond)
    fb = solve.face_blocks(P, blks)
    flu = [solve.lu_factor(fb[f]) for f in range(P.F)]
    Minv = lambda r: solve.block_jacobi(P, flu, r)
    x, its, res = solve.gmres_left(lambda v: A @ v, Minv, b, rtol=1e-13, restart=40, maxit=2000)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd) and its > 0
    k = 6
    xk, _, _ = solve.gmres_left(lambda v: A @ v, Minv, b, rtol=0.0, restart=k, maxit=k)
    Mb = Minv(b)
    K = [Mb]
    for _ in range(k - 1):
        K.append(Minv(A @ K[-1]))
    Kb = np.array(K).T
    MA = np.array([Minv(A @ Kb[:, i]) for i in range(k)]).T
    c = np.linalg.lstsq(MA, Mb, rcond=None)[0]
    xb = Kb @ c
    assert np.linalg.norm(xk - xb) <= 1e-7 * np.linalg.norm(xb)


def test_lu_factor_against_definition_and_scipy():
    rng = np.random.default_rng(2)
    for n in (1, 7, 64, 130):
        A = rng.normal(size=(n, n))
        LU, piv = solve.lu_factor(A)
        L = np.tril(LU, -1) + np.eye(n)
        U = np.triu(LU)
        assert np.abs(A[piv] - L @ U).max() <= 20 * n * 2.2e-16 * np.abs(A).max()
        assert np.all(np.abs(L) <= 1.0 + 1e-15)                       # partial pivoting bound
        b = rng.normal(size=n)
        assert np.allclose(solve.lu_solve(LU, piv, b), scipy.linalg.solve(A, b), rtol=1e-9)
    # tie rule: first maximal row wins
    A = np.array([[1.0, 2.0], [-1.0, 3.0]])
    LU, piv = solve.lu_factor(A)
    assert list(piv) == [0, 1]


# ---------------------------------------------------------------- time integration (Sec. 2.4)

def test_dirk3_order_conditions_and_stiff_accuracy():
    A, b, c = solve.alexander_dirk3()
    al = A[0, 0]
    assert abs(al ** 3 - 3 * al ** 2 + 1.5 * al - 1 / 6) < 1e-14
    assert np.isclose(b.sum(), 1) and np.isclose(b @ c, 0.5)
    assert np.isclose(b @ c ** 2, 1 / 3) and np.isclose(b @ (A @ c), 1 / 6)
    assert np.allclose(A.sum(1), c)
    assert np.allclose(A[-1], b) and c[-1] == 1.0                    # stiffly accurate: u^{n+1} = u^{n,s}
    # L-stability: R(z) = 1 + z b^T (I - z A)^{-1} 1 -> 0 as z -> -inf
    z = -1e8
    R = 1 + z * b @ np.linalg.solve(np.eye(3) - z * A, np.ones(3))
    assert abs(R) < 1e-6


def test_dirk_step_conserves_mass_momentum_energy():
    """Periodic box: the trace equations make the fluxes conservative, so the totals
    (integrals of u) are constant through each DIRK stage (eq. C242)."""
    pr = W.periodic_uniform(dim=2, nmac=2, m=2, p=2, v=(0.1, 0.05, 0))
    P = solve.Problem(pr)
    u, q, uh = _uniform_state(P, solve.uniform_from_par(pr))
    du, duh = W.perturbation(pr, 3, amp=2e-3)
    u = u + du
    uh = uh + duh
    def totals(u):
        return sum(P.geometry(e).w @ (u[e] @ P.geometry(e).T[0].T).T for e in range(P.E))
    t0 = totals(u)
    u1, q1, uh1, stats = solve.dirk_step(P, u, q, uh, dt=0.05, rtol=1e-13, precond="direct")
    assert np.allclose(totals(u1), t0, rtol=0, atol=1e-12)
    assert all(s["RF"] <= 1e-11 for s in stats)


def test_dirk_step_self_convergence_rate_three():
    """Sec. 2.4, eq. C242 with Alexander's DIRK(3,3): on a smooth periodic 2D flow the
    time-discretisation error of the whole HDG step (stage history term, stage
    solves, u^{n+1} = u^{n,3}) falls at rate 3.  Successive differences of the state at
    t = 0.04 from 1, 2, 4, 8 steps on one fixed mesh cancel the spatial error.  A wrong
    sign or index in the history term makes the scheme inconsistent or first order,
    which this rate exposes (conservation alone does not: any time term conserves).
    SUPG is off: its |v| is not smooth at the stagnation points of this flow."""
    pr = W.periodic_uniform(dim=2, nmac=2, m=2, p=1, v=(0.0, 0.0, 0), supg=0)
    P = solve.Problem(pr)
    V = 0.1

    def ufun(x):
        v1 = V * np.sin(2 * np.pi * x[0]) * np.cos(2 * np.pi * x[1])
        v2 = -V * np.cos(2 * np.pi * x[0]) * np.sin(2 * np.pi * x[1])
        return fields.conserved(1.0 + 0 * x[0], [v1, v2], 1 / 1.4 + 0 * x[0], 1.4)

    u0, q0, uh0 = _init_from_field(P, ufun, None)
    T = 0.04
    ends = []
    for n in (1, 2, 4, 8):
        u, q, uh = u0.copy(), q0.copy(), uh0.copy()
        for _ in range(n):
            u, q, uh, _ = solve.dirk_step(P, u, q, uh, dt=T / n, rtol=1e-12, precond="direct")
        ends.append(u)
    diff = [np.linalg.norm(a - b) for a, b in zip(ends[:-1], ends[1:])]
    rates = [np.log2(diff[i] / diff[i + 1]) for i in range(2)]
    assert all(2.7 < r < 3.3 for r in rates), (diff, rates)


def test_tgv_initial_state_closed_form():
    """Sec. 5.3, eq. TGV0: the initial velocity is divergence-free, the printed pressure
    is the incompressible pressure of that velocity (Laplacian of P equals minus
    sum_ij d_i v_j d_j v_i with rho_0 = 1), the state is isothermal (P / rho = P_0 /
    rho_0, i.e. rho = gamma P with P_0 = 1/gamma) and 2 pi periodic.  Derivatives by the
    complex step (first) and central differences (second), not from the formula."""
    g, V0 = 1.4, 0.1
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 2 * np.pi, size=(3, 40))

    def prim(xx):
        u = fields.tgv_u(xx, V0, g)
        rho = u[0]
        v = u[1:4] / rho
        P = (g - 1) * (u[4] - 0.5 * rho * (v * v).sum(0))
        return rho, v, P

    rho, v, P = prim(x)
    h = 1e-30
    dv = np.zeros((3, 3, x.shape[1]))          # dv[i][j] = d v_j / d x_i
    for i in range(3):
        xc = x.astype(complex)
        xc[i] += 1j * h
        dv[i] = np.imag(prim(xc)[1]) / h
    assert np.abs(np.trace(dv)).max() < 1e-15
    lapP = 0.0
    hf = 1e-3
    for i in range(3):
        e = np.zeros((3, 1))
        e[i] = hf
        lapP = lapP + (prim(x + e)[2] - 2 * P + prim(x - e)[2]) / hf ** 2
    rhs = -np.einsum("ijn,jin->n", dv, dv)
    assert np.allclose(lapP, rhs, rtol=0, atol=1e-6 * V0 ** 2)
    assert np.allclose(rho, g * P, rtol=1e-14)
    assert np.isclose(prim(np.zeros((3, 1)) + np.array([[np.pi / 2], [0.0], [0.0]]))[1][0, 0], V0)
    for k in range(3):
        s = np.zeros((3, 1))
        s[k] = 2 * np.pi
        assert np.allclose(fields.tgv_u(x + s, V0, g), fields.tgv_u(x, V0, g), atol=1e-14)
    # mean density rho_0 = 1: the pressure fluctuation has zero mean over the period
    n = 24
    t = np.arange(n) * 2 * np.pi / n
    X = np.array(np.meshgrid(t, t, t, indexing="ij")).reshape(3, -1)
    assert abs(prim(X)[0].mean() - 1.0) < 1e-14


# ---------------------------------------------------------------- Taylor-Green diagnostics (eq. C5321)

def _box_moment(lo, hi, powers):
    """int over the box of prod_k x_k^a_k, in closed form."""
    out = 1.0
    for a, b, n in zip(lo, hi, powers):
        out *= (b ** (n + 1) - a ** (n + 1)) / (n + 1)
    return out


def _linear_flow_state(P, rho_c, rho_g, A, b):
    """u at the nodes and the exact q = grad u for rho = rho_c + rho_g . x, v = A x + b
    (energy component and its gradient zero: the diagnostics do not read them)."""
    d = P.d
    u = np.zeros((P.E, P.ns, P.Np))
    q = np.zeros((P.E, d, P.ns, P.Np))
    for e in range(P.E):
        x = P.geometry(e).xn
        rho = rho_c + rho_g @ x
        v = A @ x + b[:, None]
        u[e, 0] = rho
        u[e, 1:1 + d] = rho * v
        for j in range(d):
            q[e, j, 0] = rho_g[j]
            q[e, j, 1:1 + d] = rho_g[j] * v + rho * A[:, j][:, None]   # d_j (rho v_i)
    return u, q


@pytest.mark.parametrize("d", [2, 3])
def test_flow_integrals_of_linear_velocity_fields(d):
    """Polynomial states the p = 2 space holds exactly, integrals in closed form.
    (a) rho constant, v = A x + b: K = rho/2 int |A x + b|^2 (box moments), Z = rho/2 |curl A|^2
    |Omega|.  (b) rho linear (m = rho v quadratic): the velocity gradient d_j v_i = A_ij is
    recovered exactly from q = grad u only with the - v_i d_j rho term, so Z = |curl A|^2 / 2
    int rho = |curl A|^2 / 2 rho(centre) |Omega|.  A is not symmetric (curl A != 0)."""
    pr = W.mms(dim=d, nmac=2, m=2, p=2)
    P = solve.Problem(pr)
    lo, hi = pr["lo"][:d], pr["hi"][:d]
    vol = _box_moment(lo, hi, [0] * d)
    rng = np.random.default_rng(17 + d)
    A = rng.uniform(-1, 1, size=(d, d))
    b = rng.uniform(-1, 1, size=d)
    if d == 3:
        curl = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    else:
        curl = np.array([A[1, 0] - A[0, 1]])
    # (a)
    rho0 = 1.3
    u, q = _linear_flow_state(P, rho0, np.zeros(d), A, b)
    K, Z, V = solve.flow_integrals(P, u, q)
    Kx = 0.0
    for i in range(d):
        for j in range(d):
            for k in range(d):
                pw = [0] * d
                pw[j] += 1
                pw[k] += 1
                Kx += A[i, j] * A[i, k] * _box_moment(lo, hi, pw)
            pw = [0] * d
            pw[j] = 1
            Kx += 2.0 * b[i] * A[i, j] * _box_moment(lo, hi, pw)
        Kx += b[i] * b[i] * vol
    Kx *= 0.5 * rho0
    assert abs(V - vol) < 1e-14 * vol
    assert abs(K - Kx) < 1e-13 * abs(Kx), (K, Kx)
    assert abs(Z - 0.5 * rho0 * curl @ curl * vol) < 1e-13 * Z
    # (b)
    rg = np.array([0.1, -0.07, 0.05][:d])
    u, q = _linear_flow_state(P, 1.0, rg, A, b)
    K, Z, V = solve.flow_integrals(P, u, q)
    centre = 0.5 * (np.array(lo) + np.array(hi))
    assert abs(Z - 0.5 * curl @ curl * (1.0 + rg @ centre) * vol) < 1e-13 * Z
    # without the density-gradient term the recovered gradient (hence Z) is wrong
    q_bad = q.copy()
    q_bad[:, :, 0] = 0.0
    assert abs(solve.flow_integrals(P, u, q_bad)[1] - Z) > 1e-4 * Z


def test_flow_integrals_rigid_rotation_on_the_curved_shell():
    """On the isoparametric shell a rigid rotation v = W x (W skew, angular velocity w) lies in
    the mapped space, so curl v = 2 w at every point: Z / V = 2 rho |w|^2 to rounding; and
    K = rho |w|^2 / 3 int r^2 converges to its closed form 4 pi rho |w|^2 (r1^5 - r0^5) / 15."""
    r0, r1, rho0 = 0.5, 1.0, 1.1
    w = np.array([0.3, -0.2, 0.5])
    W_ = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    Kx = 4.0 * np.pi * rho0 * (w @ w) * (r1 ** 5 - r0 ** 5) / 15.0
    errs = []
    for nq in (2, 4):
        P = solve.Problem(W.sphere(nq=nq, nr=1, m=1, p=2, r0=r0, r1=r1, ratio=1.0))
        u, q = _linear_flow_state(P, rho0, np.zeros(3), W_, np.zeros(3))
        K, Z, V = solve.flow_integrals(P, u, q)
        assert abs(Z / V - 2.0 * rho0 * (w @ w)) < 1e-13
        errs.append(abs(K / Kx - 1.0))
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 8.0, errs


def test_flow_integrals_of_the_tgv_initial_state_converge():
    """Sec. 5.3 (eq. C5321 at t = 0): the integrals of the lifted initial state (nodal
    interpolation, q from R_Q = 0) converge to those of the closed-form field, K / V -> mean
    of rho |v|^2 / 2 and Z / V -> mean of rho |omega|^2 / 2 with the hand-derived vorticity
    omega = V0 (-cos x sin y sin z, -sin x cos y sin z, 2 sin x sin y cos z).  The exact means
    come from the trapezoidal rule on a 24^3 periodic grid (exact for these trigonometric
    polynomials); their incompressible limits are 1/8 and 3/8 of V0^2.  Observed rate about 4."""
    g, V0 = 1.4, 0.1
    n = 24
    t = np.arange(n) * 2 * np.pi / n
    X = np.array(np.meshgrid(t, t, t, indexing="ij")).reshape(3, -1)
    ue = fields.tgv_u(X, V0, g)
    rho = ue[0]
    v = ue[1:4] / rho
    x, y, z = X
    om = V0 * np.array([-np.cos(x) * np.sin(y) * np.sin(z), -np.sin(x) * np.cos(y) * np.sin(z),
                        2 * np.sin(x) * np.sin(y) * np.cos(z)])
    Kx = (0.5 * rho * (v * v).sum(0)).mean()
    Zx = (0.5 * rho * (om * om).sum(0)).mean()
    assert abs(Kx / V0 ** 2 - 0.125) < 1e-3 and abs(Zx / V0 ** 2 - 0.375) < 1e-3
    errs = []
    for nm in (2, 4):
        P = solve.Problem(W.tgv(nmac=nm, Re=100.0))
        u, q, _ = solve.initial_state(P, lift=True)
        K, Z, V = solve.flow_integrals(P, u, q)
        assert abs(V / (2 * np.pi) ** 3 - 1.0) < 1e-13
        errs.append((abs(K / V / Kx - 1.0), abs(Z / V / Zx - 1.0)))
    assert errs[1][0] < 3e-3 and errs[1][1] < 3e-3, errs
    for i in range(2):
        assert errs[0][i] / errs[1][i] > 8.0, errs


# ---------------------------------------------------------------- convergence rates

def _init_from_field(P, ufun, qfun):
    u = np.zeros((P.E, P.ns, P.Np))
    q = np.zeros((P.E, P.d, P.ns, P.Np))
    uh = np.zeros(P.F * P.ns * P.Nfn)
    for e in range(P.E):
        g = P.geometry(e)
        u[e] = ufun(g.xn)
        if qfun is not None:
            q[e] = qfun(g.xn).transpose(1, 0, 2)
        for fl, (f, _) in enumerate(P.mesh.macro_faces(e)):
            fc = g.faces[fl]
            idx = P.maps[e][:, fl * P.Nfn:(fl + 1) * P.Nfn]
            uh[idx] = np.linalg.lstsq(fc["psi"], (u[e] @ fc["phi"].T).T, rcond=None)[0].T
    return u, q, uh


def _couette_error(n, p):
    pr = W.couette2d(nmac=n, p=p)
    P = solve.Problem(pr)
    u0 = solve.uniform_from_par(pr)
    u, q, uh = _uniform_state(P, u0)
    du, duh = W.perturbation(pr, 0)
    u, q, uh, hist = solve.newton_ser(P, u + du, q, uh + duh, rtol=1e-11, precond="direct")
    mass = sum(P.geometry(e).w @ (u[e, 0] @ P.geometry(e).T[0].T) for e in range(P.E))
    yq, wq = np.polynomial.legendre.leggauss(40)
    yq, wq = (yq + 1) / 2, wq / 2
    rho1 = fields.couette_exact(yq, pr["Mw"], 1.0, 1.0, P.phys)[0]
    P0 = mass / (wq @ rho1)
    err = 0.0
    for e in range(P.E):
        g = P.geometry(e)
        rho, v, E, Pr_, T = ph.primitives(list(u[e] @ g.T[0].T), 1.4)
        T_ex = fields.couette_exact(g.xq[1], pr["Mw"], 1.0, P0, P.phys)[2]
        err += g.w @ (T - T_ex) ** 2
    return np.sqrt(err), hist


def test_newton_converges_quadratically():
    """With the pseudo-time term switched off (dtau -> infinity) the SER iteration is
    Newton's method on the fully coupled residual; with the exact Jacobian blocks, the
    two-layer condensation, a direct trace solve and the recovery all consistent, the
    convergence is quadratic: order estimates log(r_{k+1}/r_k) / log(r_k/r_{k-1}) near
    2 above the round-off floor.  A dropped or mis-signed Jacobian term, or an
    inconsistent condensation/recovery, degrades this to linear convergence."""
    pr = W.mms(dim=2, nmac=2, m=2, p=2, vel=0.1)
    P = solve.Problem(pr)
    par = pr["field_par"]
    u, q, uh = _init_from_field(P, lambda x: fields.mms_u(x, par, 1.4), lambda x: fields.mms_q(x, par, 1.4))
    rng = np.random.default_rng(0)
    u = u * (1 + 0.02 * rng.standard_normal(u.shape))
    uh = uh * (1 + 0.02 * rng.standard_normal(uh.shape))
    _, _, _, hist = solve.newton_ser(P, u, q, uh, rtol=1e-13, tau_init=1e12, tau_max=1e12, precond="direct")
    r = np.array([h["RF"] for h in hist])
    assert r[-1] <= 1e-13 * r[0] and len(r) <= 7
    live = r[r > 1e-12 * r[0]]
    orders = np.log(live[2:] / live[1:-1]) / np.log(live[1:-1] / live[:-2])
    assert len(orders) >= 2 and orders[-1] > 1.7 and orders[-2] > 1.15   # first step pre-asymptotic


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2])
def test_couette_temperature_converges_at_rate_p_plus_1(p):
    e1, h1 = _couette_error(2, p)
    e2, h2 = _couette_error(4, p)
    assert h1[-1]["RF"] <= 1e-11 * h1[0]["RF"] and h2[-1]["RF"] <= 1e-11 * h2[0]["RF"]
    assert np.log2(e1 / e2) >= p + 1 - 0.3


def _mms_error(n, p):
    pr = W.mms(dim=2, nmac=n, m=2, p=p, vel=0.1)
    P = solve.Problem(pr)
    par = pr["field_par"]
    u, q, uh = _init_from_field(P, lambda x: fields.mms_u(x, par, 1.4), lambda x: fields.mms_q(x, par, 1.4))
    u, q, uh, hist = solve.newton_ser(P, u, q, uh, rtol=1e-10, precond="direct")
    err = 0.0
    for e in range(P.E):
        g = P.geometry(e)
        err += g.w @ np.sum((u[e] @ g.T[0].T - fields.mms_u(g.xq, par, 1.4)) ** 2, 0)
    return np.sqrt(err), hist


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2])
def test_manufactured_solution_converges_at_rate_p_plus_1(p):
    e1, h1 = _mms_error(2, p)
    e2, h2 = _mms_error(4, p)
    assert h2[-1]["RF"] <= 1e-10 * h2[0]["RF"]
    assert np.log2(e1 / e2) >= p + 1 - 0.3


# ---------------------------------------------------------------- simplicial macro-elements (Sec. 2.2)

def _simplex(pr):
    pr = dict(pr)
    pr["mesh_kind"] = W.MESH_SIMPLEX
    return pr


@pytest.mark.parametrize("d", [2, 3])
def test_simplex_macro_subdivision_and_nodes_brute_force(d):
    """The m-refined Kuhn macro K = {1 >= xi_1 >= ... >= xi_d >= 0}: its m^d sub-simplices tile K
    (each of 300 random points of K lies in exactly one, tested by the sub-simplex's own
    inequalities), each carries the C(p + d, d) nodes of P_p, their union is the C(m p + d, d)
    lattice points of K, and each face holds C(m p + d - 1, d - 1) of them."""
    from math import comb
    rng = np.random.default_rng(3 + d)
    for m, p in ((1, 2), (2, 1), (2, 2), (3, 1), (2, 3)):
        K = sx.KuhnMacro(d, m, p, tables=False)
        assert len(K.subs) == m ** d
        assert K.Np == comb(m * p + d, d) and K.Nfn == comb(m * p + d - 1, d - 1)
        union = set()
        for sb in K.subs:
            assert len(sb["nodes"]) == comb(p + d, d)
            union |= set(sb["nodes"].tolist())
        assert union == set(range(K.Np))
        for fn in K.face_nodes:
            assert len(fn) == K.Nfn
        X = -np.sort(-rng.uniform(size=(300, d)), axis=1)
        for x in X:
            hits = 0
            for sb in K.subs:
                u = (m * x - sb["c"])[list(sb["pi"])]
                if u[0] <= 1.0 and u[-1] >= 0.0 and np.all(np.diff(u) <= 0.0):
                    hits += 1
            assert hits == 1


def test_simplex_spaces_reproduce_the_papers_dof_tables():
    """The paper's tetrahedral DOF tables, now from the constructed spaces (not a formula):
    (d + 1)(d + 2) = 20 unknowns per node of KuhnMacro(3, m, p), 5 per node of a face, and
    n_macro m^3 = 768 elements in Table 1; the m p = 8 counts of Tables 3, 8 and 10 come out
    the same for (m, p) = (8, 1), (4, 2), (2, 4); the sphere's Table 6 for m = 1, 2."""
    gold = json.load(open(os.path.join(GOLD, "dof_tables.json")))
    t1 = gold["table1_couette_768_elements_p3"]
    for r in t1["rows"]:
        K = sx.KuhnMacro(3, r["m"], t1["p"], tables=False)
        assert 20 * K.Np == r["local"]
        assert r["n_macro"] * len(K.subs) == 768
        faces = (4 * r["n_macro"] + r["boundary_triangles"]) // 2
        assert 5 * faces * K.Nfn == r["global"]
    t3 = gold["table3_couette_fixed_local"]
    for m, p in ((8, 1), (4, 2), (2, 4)):
        K = sx.KuhnMacro(3, m, p, tables=False)
        for r in t3["rows"]:
            assert 20 * K.Np == r["local"]
            faces = (4 * r["n_macro"] + r["boundary_triangles"]) // 2
            assert 5 * faces * K.Nfn == r["global"]
        t8 = gold["table8_tgv_mp8_periodic"]
        for r in t8["rows"]:      # periodic: every face has two owners, F = 2 E
            assert 20 * K.Np * r["n_macro"] == r["total_local"]
            assert 5 * 2 * r["n_macro"] * K.Nfn == r["global"]
    t6 = gold["table6_sphere_p3"]
    for r in t6["rows"]:
        K = sx.KuhnMacro(3, r["m"], t6["p"], tables=False)
        assert 20 * K.Np * r["n_macro"] == r["total_local"]
        assert r["global"] % (5 * K.Nfn) == 0


@pytest.mark.parametrize("d", [2, 3])
def test_simplex_quadrature_basis_and_faces(d):
    """Reference tables of KuhnMacro(d, 2, 2): the volume rule integrates every monomial of
    degree <= 2 p + 3 exactly (iterated integrals over K by sympy); the basis and its
    derivatives reproduce a random polynomial of degree p; on each face the volume basis and
    the trace basis reproduce it too, the face points satisfy the face's equation, and with
    x = xi the face weights add up to the face areas 1/(d-1)!, sqrt(2)/(d-1)!, ... and the
    area-weighted normals to zero."""
    import sympy
    from math import factorial
    m, p = 2, 2
    K = sx.KuhnMacro(d, m, p)
    xs = sympy.symbols("x1:%d" % (d + 1))
    for alpha in sx.monomials(d, 2 * p + 3):
        expr = sympy.Integer(1)
        for k in range(d):
            expr = expr * xs[k] ** alpha[k]
        for k in reversed(range(d)):
            expr = sympy.integrate(expr, (xs[k], 0, xs[k - 1] if k > 0 else 1))
        num = np.sum(K.wq * np.prod(K.xq ** np.array(alpha)[:, None], axis=0))
        assert abs(num - float(expr)) < 1e-14, alpha
    rng = np.random.default_rng(d)
    coef = {a: rng.uniform(-1, 1) for a in sx.monomials(d, p)}

    def poly(x):          # x [d, n] -> values [n], gradient [d, n]
        v = np.zeros(x.shape[1])
        g = np.zeros_like(x)
        for a, c in coef.items():
            v += c * np.prod(x ** np.array(a)[:, None], axis=0)
            for l in range(d):
                if a[l]:
                    b = list(a)
                    b[l] -= 1
                    g[l] += c * a[l] * np.prod(x ** np.array(b)[:, None], axis=0)
        return v, g

    nodal, _ = poly(K.xn.T)
    v, g = poly(K.xq)
    assert np.abs(K.B0 @ nodal - v).max() < 1e-12
    for l in range(d):
        assert np.abs(K.Bd[l] @ nodal - g[l]).max() < 1e-11
    geo = sx.SimplexMacroGeometry(K, np.zeros(d), np.eye(d), 1.0)
    areas = [1.0 / factorial(d - 1)] + [np.sqrt(2.0) / factorial(d - 1)] * (d - 1) + [1.0 / factorial(d - 1)]
    total = np.zeros(d)
    for fl, (fc, gf) in enumerate(zip(K.faces, geo.faces)):
        vf, _ = poly(fc["xi"])
        assert np.abs(fc["phi"] @ nodal - vf).max() < 1e-12
        assert np.abs(fc["psi"] @ nodal[fc["nodes"]] - vf).max() < 1e-12
        xi = fc["xi"]
        eq = xi[0] - 1.0 if fl == 0 else (xi[d - 1] if fl == d else xi[fl - 1] - xi[fl])
        assert np.abs(eq).max() < 1e-14
        assert abs(gf["w"].sum() - areas[fl]) < 1e-13
        total += gf["w"].sum() * gf["n"]
    assert np.abs(total).max() < 1e-14


@pytest.mark.parametrize("d,per", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_simplex_mesh_owners_and_matching(d, per):
    """Kuhn triangulation of a 2^d box grid: E and F as counted in workloads.sizes; every
    face has two owners except on the non-periodic boundary planes, where it has one and a
    boundary side; both owners' gather maps send the nodes at the same position (periodic
    axes wrapped) to the same trace unknown."""
    pr = _simplex(W.mms(dim=d, nmac=2, m=2, p=2))
    pr["periodic"] = [per] * 3
    P = solve.Problem(pr)
    z = W.sizes(pr)
    assert (P.E, P.F, P.Np, P.Nfn) == (z["E"], z["F"], z["Np"], z["Nfn"])
    L = np.array(pr["hi"][:d]) - np.array(pr["lo"][:d])
    for f, own in enumerate(P.mesh.face_owners()):
        bs = [P.mesh.macro_faces(e)[fl][1] for e, fl in own]
        if len(own) == 1:
            assert not per and bs[0] >= 0
            continue
        assert bs == [-1, -1]
        pos = []
        for e, fl in own:
            x = P.geometry(e).xn[:, P.mesh.fnodes[fl]]
            if per:
                x = np.mod(x + 1e-9, L[:, None]) - 1e-9
            gi = P.maps[e][0, fl * P.Nfn:(fl + 1) * P.Nfn]
            pos.append({int(i): tuple(np.round(x[:, k], 9)) for k, i in enumerate(gi)})
        assert pos[0] == pos[1]


@pytest.mark.parametrize("d", [2, 3])
def test_free_stream_preservation_on_simplicial_meshes(d):
    """A uniform state (q = 0, u^ = u) on periodic and on Dirichlet simplicial meshes gives
    R = 0 to rounding (SUPG on): watertight faces, consistent normals and weights."""
    pr = _simplex(W.periodic_uniform(dim=d, nmac=2, m=2, p=2 if d == 2 else 1))
    P = solve.Problem(pr)
    u0 = solve.uniform_from_par(pr)
    u, q, _ = _uniform_state(P, u0)
    _, _, nrm, _ = solve.global_assemble(P, u, q, _uniform_trace(P, u0), want_jac=False)
    assert nrm["RF"] < 1e-13, nrm
    pr2 = dict(pr)
    pr2["periodic"] = [0, 0, 0]
    pr2["bc"] = [W.BC_DIRICHLET] * 6
    P2 = solve.Problem(pr2)
    u, q, _ = _uniform_state(P2, u0)
    _, _, nrm, _ = solve.global_assemble(P2, u, q, _uniform_trace(P2, u0), want_jac=False)
    assert nrm["RF"] < 1e-13, nrm


@pytest.mark.parametrize("p", [1, 2])
def test_simplex_lifting_reproduces_gradients_of_linear_fields(p):
    """R_Q = 0 on a tetrahedral macro: q_k = -M^-1 (G_k u + Gh_k u^) returns the exact
    gradient of a linear field given at the nodes and on the faces (every macro of the
    triangulated cell, all d! orientations)."""
    P = solve.Problem(_simplex(W.mms(dim=3, nmac=1, m=2, p=p)))
    rng = np.random.default_rng(p)
    for e in range(P.E):
        geo = P.geometry(e)
        c, g = rng.uniform(-1, 1), rng.uniform(-1, 1, size=3)
        u = c + g @ geo.xn
        uh = np.concatenate([c + g @ geo.xn[:, P.mesh.fnodes[fl]] for fl in range(4)])
        with np.errstate(invalid="ignore"):
            blk = asm.assemble_macro(geo, P.phys, np.repeat(u[None], P.ns, 0), np.zeros((3, P.ns, P.Np)),
                                     np.repeat(uh[None], P.ns, 0), want_jac=False)
        for k in range(3):
            qk = -np.linalg.solve(blk["M"], blk["Gk"][k] @ u + blk["Ghk"][k] @ uh)
            assert np.abs(qk - g[k]).max() < 1e-12


def test_simplex_condense_solve_recover_equals_monolithic():
    """Second-layer condensation, trace solve and recovery on a triangulated mesh equal the
    monolithic solve of the whole system of eq. C312."""
    pr = _simplex(W.mms(dim=2, nmac=2, m=2, p=2))
    P = solve.Problem(pr)
    u, q, uh = W.random_state(pr, 13)
    blks, geos, _, _ = solve.global_assemble(P, u, q, uh)
    A, r = _monolithic(P, blks, geos, 0.3)
    x = np.linalg.solve(A, -r)
    dU, dQ, dUh, its, _ = solve.linear_step(P, blks, geos, shift=0.3, precond="direct")
    nloc = P.d * P.ns * P.Np + P.ns * P.Np
    assert np.allclose(dUh, x[P.E * nloc:], rtol=1e-9, atol=1e-11)
    for e in range(P.E):
        o = e * nloc
        assert np.allclose(dQ[e].reshape(-1), x[o:o + P.d * P.ns * P.Np], atol=1e-9)
        assert np.allclose(dU[e].reshape(-1), x[o + P.d * P.ns * P.Np:o + nloc], atol=1e-10)


def _simplex_mms_error(n, p):
    pr = _simplex(W.mms(dim=2, nmac=n, m=2, p=p, vel=0.1))
    P = solve.Problem(pr)
    par = pr["field_par"]
    u, q, uh = _init_from_field(P, lambda x: fields.mms_u(x, par, 1.4), lambda x: fields.mms_q(x, par, 1.4))
    u, q, uh, hist = solve.newton_ser(P, u, q, uh, rtol=1e-10, precond="direct")
    err = 0.0
    for e in range(P.E):
        g = P.geometry(e)
        err += g.w @ np.sum((u[e] @ g.T[0].T - fields.mms_u(g.xq, par, 1.4)) ** 2, 0)
    return np.sqrt(err), hist


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2])
def test_simplex_manufactured_solution_converges_at_rate_p_plus_1(p):
    """The steady 2D manufactured solution on twice-refined triangular macro-elements
    (Kuhn triangulation of 2^2 and 4^2 cells): the L2 error falls at rate p + 1 (observed
    2.18 and 2.97)."""
    e1, h1 = _simplex_mms_error(2, p)
    e2, h2 = _simplex_mms_error(4, p)
    assert h2[-1]["RF"] <= 1e-10 * h2[0]["RF"]
    assert np.log2(e1 / e2) >= p + 1 - 0.3


@pytest.mark.slow
def test_simplex_couette3d_with_source_converges():
    """The paper's 3D Couette flow with a source (Sec. 5.1) on tetrahedral macro-elements
    (Kuhn triangulation of 1^3 and 2^3 cells, m = 1, p = 2), steady-solved from the closed
    form plus a seeded 1e-3 perturbation: every conserved variable's L2 error falls at a rate
    near p + 1 on these coarse meshes (observed 2.47 to 2.91)."""
    def run(n):
        pr = _simplex(W.couette3d(nmac=n, m=1, p=2))
        P = solve.Problem(pr)
        par, g_ = pr["field_par"], pr["gamma"]
        u, q, uh = _init_from_field(P, lambda x: fields.couette3d_u(x, par, g_),
                                    lambda x: fields.couette3d_q(x, par, g_))
        du, duh = W.perturbation(pr, 0)
        u, q, uh, hist = solve.newton_ser(P, u + du, q, uh + duh, rtol=1e-10, atol=1e-13, precond="direct")
        assert hist[-1]["RF"] <= 1e-10 * hist[0]["RF"] or hist[-1]["RF"] <= 1e-13
        err = np.zeros(P.ns)
        for e in range(P.E):
            g = P.geometry(e)
            err += g.w @ ((u[e] @ g.T[0].T - fields.couette3d_u(g.xq, par, g_)) ** 2).T
        return np.sqrt(err)
    rates = np.log2(run(1) / run(2))
    assert np.all(rates >= 2.3), rates


# ---------------------------------------------------------------- MLP correction (oracle side)

def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import mlp
    nin, hid, nout = 8, 6, 8
    rng = np.random.default_rng(4)
    p = rng.normal(size=mlp.n_params(nin, hid, nout)) * 0.5
    X = rng.normal(size=(5, nin))
    T = rng.normal(size=(5, nout))
    loss, g = mlp.loss_and_grad(p, X, T, nin, hid, nout)
    h = 1e-6
    for i in rng.choice(len(p), 25, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, T, nin, hid, nout)[0] - mlp.loss_and_grad(pm, X, T, nin, hid, nout)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i]))
    # bf16 rounding: 8 significant bits, round to nearest even
    assert mlp.bf16_round(np.float32(1.0 + 2 ** -9))[()] == 1.0
    assert mlp.bf16_round(np.float32(1.0 + 3 * 2 ** -9))[()] == 1.0 + 2 ** -7


# ---------------------------------------------------------------- curved macros on the cubed sphere

def _uniform_trace(P, u0):
    uh = np.zeros(P.F * P.ns * P.Nfn)
    for f in range(P.F):
        for s in range(P.ns):
            uh[(f * P.ns + s) * P.Nfn:(f * P.ns + s + 1) * P.Nfn] = u0[s]
    return uh


def test_shell_mesh_counts_owners_and_node_matching():
    """Cubed-sphere O-grid: E = 6 nq^2 nr macros, 6 nq^2 (nr + 1) radial plus 12 nq^2 nr
    angular faces (brute-force count of distinct faces by position); inner and outer
    spheres have one owner per face, every other face two, and the two owners' gather maps
    send nodes at the same position to the same trace unknown (also across cube-panel
    edges, where the two owners' face axes are permuted or reversed)."""
    pr = W.sphere(nq=2, nr=2, m=1, p=2)
    P = solve.Problem(pr)
    assert P.E == 48 and P.F == 6 * 4 * 3 + 12 * 4 * 2 == W.sizes(pr)["F"]
    own = P.mesh.face_owners()
    nb = [0, 0]
    for f, o in enumerate(own):
        sides = [P.mesh.macro_faces(e)[fl][1] for e, fl in o]
        if len(o) == 1:
            assert sides[0] in (0, 1)
            nb[sides[0]] += 1
        else:
            assert len(o) == 2 and sides == [-1, -1]
    assert nb == [24, 24]
    pos = {}
    for e in range(P.E):
        g = P.maps[e][0]
        for fl in range(6):
            for j in range(P.Nfn):
                x = P.mesh.nodes[e][:, P.mesh.fnodes[fl][j]]
                key = int(g[fl * P.Nfn + j])
                if key in pos:
                    assert np.abs(pos[key] - x).max() < 1e-12
                else:
                    pos[key] = x
    assert len(pos) == P.F * P.Nfn
    # the nodes of the inner and outer layers lie on the spheres
    r = np.linalg.norm(P.mesh.nodes, axis=1)
    assert np.abs(r.min() - 0.5) < 1e-14 and np.abs(r.max() - 10.0) < 1e-12


def test_mapped_geometry_volume_and_area_converge():
    """Isoparametric curved macros: the shell volume 4/3 pi (r1^3 - r0^3) and the inner
    sphere's area 4 pi r0^2 from the quadrature weights converge under refinement of the
    angular cells at least at rate 3 (degree-2 interpolation of the sphere), and the two
    owners of every interior face see opposite area-weighted normals (watertight map)."""
    r0, r1 = 0.5, 1.0
    errs = []
    for nq in (2, 4):
        P = solve.Problem(W.sphere(nq=nq, nr=1, m=1, p=2, r0=r0, r1=r1, ratio=1.0))
        geos = [P.geometry(e) for e in range(P.E)]
        vol = sum(g.w.sum() for g in geos)
        area = sum(geos[e].faces[4]["w"].sum() for e in range(P.E))
        errs.append((abs(vol / (4.0 / 3.0 * np.pi * (r1 ** 3 - r0 ** 3)) - 1.0),
                     abs(area / (4.0 * np.pi * r0 * r0) - 1.0)))
        for o in P.mesh.face_owners():
            if len(o) == 2:
                nw = [(geos[e].faces[fl]["w"][None, :] * geos[e].faces[fl]["n"]).sum(axis=1) for e, fl in o]
                assert np.abs(nw[0] + nw[1]).max() < 1e-13
    for i in range(2):
        assert errs[0][i] < 5e-3 and errs[1][i] < errs[0][i] / 8.0, errs


@pytest.mark.parametrize("inner", [1, 3])
def test_free_stream_preservation_on_the_sphere_mesh(inner):
    """A uniform state (q = 0, u^ = u) on the curved shell mesh with Dirichlet or far-field
    data equal to that state gives R_Q = R_U = R_Uh = 0 to rounding (SUPG on): the discrete
    divergence theorem holds on the curved macros (the quadrature integrates the mapped
    integrands of degree 3p exactly) and the far-field operator vanishes at u = u^ = u_inf."""
    pr = W.sphere(nq=2, nr=1, m=1, p=2, inner=inner, outer=3)
    pr["field_par"] = [1.2, 0.3, -0.1, 0.2, 1.1, 0.0, 0.0, 0.0]
    P = solve.Problem(pr)
    u0 = solve.uniform_from_par(pr)
    u = np.repeat(np.repeat(u0[None, :, None], P.E, 0), P.Np, 2)
    q = np.zeros((P.E, 3, P.ns, P.Np))
    _, _, nrm, _ = solve.global_assemble(P, u, q, _uniform_trace(P, u0), want_jac=False)
    assert nrm["RF"] < 1e-12, nrm


def test_mapped_lifting_reproduces_gradients_of_linear_fields():
    """R_Q = 0 on a curved macro (p = 1, where the quadrature is exact for the mapped
    integrands): q_k = -M_J^-1 (G_k u + Gh_k u^) returns the exact constant gradient of
    any linear field u = c + g.x given at the nodes and on the faces (x is in the
    isoparametric space, so is u): pins J^-1 in the volume terms, the normals and weights of
    the faces and the per-macro mass matrix."""
    P = solve.Problem(W.sphere(nq=2, nr=2, m=2, p=1))
    rng = np.random.default_rng(5)
    for e in (0, 13, 47):
        geo = P.geometry(e)
        c, g = rng.uniform(-1, 1), rng.uniform(-1, 1, size=3)
        u = c + g @ geo.xn
        uh = np.concatenate([c + g @ geo.xn[:, P.mesh.fnodes[fl]] for fl in range(6)])
        with np.errstate(invalid="ignore"):   # the residual of this non-physical state is unused
            blk = asm.assemble_macro(geo, P.phys, np.repeat(u[None], P.ns, 0), np.zeros((3, P.ns, P.Np)),
                                     np.repeat(uh[None], P.ns, 0), want_jac=False)
        for k in range(3):
            qk = -np.linalg.solve(blk["M"], blk["Gk"][k] @ u + blk["Ghk"][k] @ uh)
            assert np.abs(qk - g[k]).max() < 1e-12


def test_couette3d_closed_form_gradient_and_walls():
    """Compressible Couette flow with a source (Sec. 5.1): the closed-form gradient used for the
    source equals the complex-step derivative of the closed-form state; the state is a shear
    flow (only v_1, depending on x_2 only, zero at x_2 = 0), at constant pressure 1/gamma, with
    T(0) = alpha and T(1) = beta."""
    pr = W.couette3d()
    par, g = pr["field_par"], pr["gamma"]
    rng = np.random.default_rng(4)
    x = rng.uniform(0.0, 1.0, size=(3, 7))
    q = np.array(fields.couette3d_q(x, par, g))        # [s][k]
    for k in range(3):
        xc = x.astype(complex)
        xc[k] += 1j * ph.CS_H
        dk = np.imag(np.array(fields.couette3d_u(xc, par, g))) / ph.CS_H
        assert np.abs(dk - q[:, k]).max() < 1e-13
    u = np.array(fields.couette3d_u(x, par, g))
    rho, v, E, P, T = ph.primitives(list(u), g)
    assert np.allclose(P, 1.0 / g, rtol=1e-14) and np.abs(v[1]).max() == 0.0 and np.abs(v[2]).max() == 0.0
    ends = np.array([[0.3, 0.3], [0.0, 1.0], [0.6, 0.6]])
    ue = np.array(fields.couette3d_u(ends, par, g))
    _, ve, _, _, Te = ph.primitives(list(ue), g)
    assert abs(ve[0][0]) < 1e-16 and np.allclose(Te, [par[1], par[2]], rtol=1e-14)
