"""Curved macro-elements on the cubed-sphere shell (flow past a sphere): parity of the CUDA
path (through the C ABI) with the FP64 oracle.

The oracle builds its own mesh, isoparametric geometry, face matching and far-field operator
(oracle/space.py, oracle/physics.py); the library builds its own (csrc/shell.cu,
csrc/physics.cuh).  The same seeded states go to both.  Tolerances as for the box meshes:
blocks and residuals 1e-11 relative to the largest entry, the FP64 linear step 1e-10
relative L2, the FP64 DIRK end state 1e-10 relative L2 (both solved to stagnation).
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import assemble as asm
from oracle import solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as m
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for gpu tests")
    return m


def to_dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def rel2(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# inner isothermal wall, outer characteristic far field, SUPG on
CASES = {
    "p2_m1": (lambda: W.sphere(nq=2, nr=1, m=1, p=2, r1=2.0), [0, 5, 23]),      # 24 macros touching both spheres
    "p1_m2": (lambda: W.sphere(nq=2, nr=2, m=2, p=1), [0, 9, 30, 47]),          # interior radial faces
    "p2_m2": (lambda: W.sphere(nq=1, nr=1, m=2, p=2, r1=2.0), [0, 3]),          # the sphere workload's macro (Nu 625)
    "p2_m2_stretched": (lambda: W.sphere(nq=1, nr=1, m=2, p=2), [1, 4]),       # one layer 0.5 <= r <= 10
}
FP64 = dict(precision=0, precond=1, apply_mode=0)
GOLD = os.path.join(os.path.dirname(__file__), "golden", "dirk_sphere_2x1_p2.npz")


@pytest.mark.parametrize("case", sorted(CASES))
def test_sphere_assembly_blocks_and_residuals(lib, case):
    mk, macros = CASES[case]
    pr = mk()
    P = solve.Problem(pr)
    u, q, uh = W.random_state(pr, 31)
    hist = 0.05 * np.ones_like(u)
    ctx = lib.Context(pr, FP64)
    assert ctx.info["n_macro"] == P.E and ctx.info["n_face"] == P.F
    norms = ctx.assemble(to_dev(u), to_dev(q), to_dev(uh), coef=0.4, hist=to_dev(hist), supg_time=1)
    tt = dict(coef=0.4, hist=hist, supg_time=True)
    _, _, onrm, _ = solve.global_assemble(P, u, q, uh, tt, want_jac=False)
    assert np.allclose(norms, [onrm["RQ"], onrm["RU"], onrm["RUh"], onrm["RF"]], rtol=1e-11)
    Nu, Nt = P.ns * P.Np, P.ns * P.Nth
    for e in macros:
        geo = P.geometry(e)
        b = asm.assemble_macro(geo, P.phys, u[e], q[e], P.local_trace(e, uh),
                               dict(coef=0.4, hist=hist[e], supg_time=True), None, P.bfaces(e, geo))
        assert rel(ctx.get_block(0, e).reshape(Nu, Nu), b["Auu"]) < 1e-11
        for k in range(3):
            assert rel(ctx.get_block(1 + k, e).reshape(Nu, Nu), b["Auq"][k]) < 1e-11
            assert rel(ctx.get_block(6 + k, e).reshape(Nt, Nu), b["Ahq"][k]) < 1e-11
        assert rel(ctx.get_block(4, e).reshape(Nu, Nt), b["Auh"]) < 1e-11
        assert rel(ctx.get_block(5, e).reshape(Nt, Nu), b["Ahu"]) < 1e-11
        assert rel(ctx.get_block(9, e).reshape(Nt, Nt), b["Ahh"]) < 1e-11
        assert rel(ctx.get_block(10, e), b["RQ"].reshape(-1)) < 1e-11
        assert rel(ctx.get_block(11, e), b["RU"].reshape(-1)) < 1e-11
        assert rel(ctx.get_block(12, e), b["RUh"].reshape(-1)) < 1e-11
    ctx.close()


def test_sphere_assembly_at_rest(lib):
    """Zero momentum at every node (a gas at rest near the sphere, as in the first layers of the
    blended initial state): the SUPG coefficient sits on the kink of |v|; its derivative there is
    0 on both sides, the blocks are finite and equal to the oracle's."""
    pr = W.sphere(nq=2, nr=1, m=1, p=2, r1=2.0)
    P = solve.Problem(pr)
    u, q, uh = W.random_state(pr, 33)
    u[:, 1:4, :] = 0.0
    ctx = lib.Context(pr, FP64)
    norms = ctx.assemble(to_dev(u), to_dev(q), to_dev(uh))
    _, _, onrm, _ = solve.global_assemble(P, u, q, uh, want_jac=False)
    assert np.allclose(norms, [onrm["RQ"], onrm["RU"], onrm["RUh"], onrm["RF"]], rtol=1e-11)
    Nu = P.ns * P.Np
    for e in (0, 13):
        geo = P.geometry(e)
        b = asm.assemble_macro(geo, P.phys, u[e], q[e], P.local_trace(e, uh), None, None, P.bfaces(e, geo))
        A = ctx.get_block(0, e).reshape(Nu, Nu)
        assert np.isfinite(A).all()
        assert rel(A, b["Auu"]) < 1e-11
        for k in range(3):
            assert rel(ctx.get_block(1 + k, e).reshape(Nu, Nu), b["Auq"][k]) < 1e-11
    ctx.close()


@pytest.mark.parametrize("inner", [W.BC_DIRICHLET, W.BC_FARFIELD])
def test_sphere_free_stream_preservation(lib, inner):
    """A uniform state with q = 0 and u^ = u, and Dirichlet / far-field data equal to it,
    has zero residual on the curved mesh (discrete divergence theorem on the mapped macros)."""
    pr = W.sphere(nq=2, nr=2, m=2, p=2, inner=inner)
    pr["field"] = W.FIELD_UNIFORM
    pr["field_par"] = [1.2, 0.3, -0.1, 0.2, 1.1, 0.0, 0.0, 0.0]
    ctx = lib.Context(pr, FP64)
    u, q, uh = ctx.init_state(None, None, lift=True)
    norms = ctx.assemble(u, q, uh)
    print("free stream on the sphere mesh: |R| =", norms)
    assert norms[3] < 1e-11
    assert q.abs().max().item() < 1e-11
    ctx.close()


def test_sphere_initial_state_matches_oracle(lib):
    """The blended free stream at the nodes, the first owner's trace and the lifted gradient
    (R_Q = 0 with the per-macro M_J) on a mesh whose faces cross cube-panel edges."""
    pr = W.sphere(nq=2, nr=2, m=2, p=2, r0=0.5, r1=2.0)
    P = solve.Problem(pr)
    ou, oq, ouh = solve.initial_state(P, lift=True)
    ctx = lib.Context(pr, FP64)
    u, q, uh = ctx.init_state(None, None, lift=True)
    eu, eq, eh = rel2(u.cpu().numpy(), ou), rel2(q.cpu().numpy(), oq), rel2(uh.cpu().numpy(), ouh)
    print("sphere initial state rel L2: u %.2e q %.2e uh %.2e" % (eu, eq, eh))
    assert eu <= 1e-14 and eh <= 1e-14 and eq <= 1e-11
    ctx.close()


_lin = {}


def _oracle_linear(case):
    """Newton linearisation about the blended free stream plus a seeded U(-0.01, 0.01)
    perturbation of u and u^ (wall and far field active).  (A fully random state, as used for
    the blocks, makes the block-Jacobi-preconditioned trace system of this mesh strongly
    indefinite: FGMRES stalls there, while the oracle's dense solve does not.)"""
    if case not in _lin:
        pr = CASES[case][0]()
        P = solve.Problem(pr)
        u, q, uh = solve.initial_state(P, lift=True)
        du, duh = W.perturbation(pr, 41, amp=1e-2)
        u, uh = u + du, uh + duh
        blks, geos, _, _ = solve.global_assemble(P, u, q, uh)
        dU, dQ, dUh, _, _ = solve.linear_step(P, blks, geos, shift=0.5, precond="direct")
        _lin[case] = (pr, (u, q, uh), (dU, dQ, dUh))
    return _lin[case]


MIXED = dict(precision=1, precond=1, apply_mode=1, tc_mode=4, refine_iters=2, precond_bf16=1)


@pytest.mark.parametrize("case", ["p2_m1", "p2_m2"])
def test_sphere_newton_linear_step_mixed(lib, case):
    """The mixed form on curved macros (FP32 blocks, per-macro FP32 liftings, tcgen05 product
    for A^T_i, FP64 refinement and Krylov vectors): the linear step is the FP64 step of a
    perturbed matrix, held to 64 cond(S) 2^-24 and never looser than 1e-4."""
    pr, (u, q, uh), (dU, dQ, dUh) = _oracle_linear(case)
    P = solve.Problem(pr)
    geo = P.geometry(0)
    c0 = solve.condense_second_layer(geo, asm.assemble_macro(geo, P.phys, u[0], q[0], P.local_trace(0, uh),
                                                             None, None, P.bfaces(0, geo)), shift=0.5)
    condS = np.linalg.cond(c0["S"])
    ctx = lib.Context(pr, dict(MIXED, lin_rtol=1e-6, lin_atol=0.0, restart=60, max_iters=3000))
    ctx.assemble(to_dev(u), to_dev(q), to_dev(uh))
    b = ctx.condense(shift=0.5)
    duh, st = ctx.linear_solve(b)
    du, dq = ctx.recover(duh)
    e = [rel2(duh.cpu().numpy(), dUh), rel2(du.cpu().numpy(), dU), rel2(dq.cpu().numpy(), dQ)]
    print("sphere %s mixed linear step rel L2 (dUh, dU, dQ) = %s, FGMRES its %d, cond(S) %.2e"
          % (case, ["%.2e" % x for x in e], st["fgmres_iters"], condS))
    assert max(e) <= min(64 * condS * 2.0 ** -24, 1e-4)
    ctx.close()


@pytest.mark.parametrize("apply_mode", [0, 1, 2])
@pytest.mark.parametrize("case", ["p2_m1", "p2_m2"])
def test_sphere_newton_linear_step(lib, case, apply_mode):
    """Condensation with the per-macro liftings, factorisation, FGMRES on the trace system
    (Algorithm 2, the stored A^T_i, and the row-compressed Algorithm 2) and recovery."""
    pr, (u, q, uh), (dU, dQ, dUh) = _oracle_linear(case)
    ctx = lib.Context(pr, dict(FP64, apply_mode=apply_mode, lin_rtol=1e-13, lin_atol=0.0, restart=60,
                               max_iters=3000))
    ctx.assemble(to_dev(u), to_dev(q), to_dev(uh))
    b = ctx.condense(shift=0.5)
    duh, st = ctx.linear_solve(b)
    du, dq = ctx.recover(duh)
    e = [rel2(duh.cpu().numpy(), dUh), rel2(du.cpu().numpy(), dU), rel2(dq.cpu().numpy(), dQ)]
    print("sphere %s apply_mode %d linear step rel L2 (dUh, dU, dQ) = %s, FGMRES its %d, |r|/|b| %.2e"
          % (case, apply_mode, ["%.2e" % x for x in e], st["fgmres_iters"], st["res"] / b.norm().item()))
    assert max(e) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sphere_dirk_step_matches_oracle(lib, prec):
    """One DIRK3 step (3 stages, Newton to 1e-12) from the blended free stream, wall and far
    field active, against the oracle's values in tests/golden/dirk_sphere_2x1_p2.npz (written by
    tests/golden/make_dirk_sphere.py): end state within 1e-10, increment within 1e-8 (relative
    L2)."""
    if not os.path.exists(GOLD):
        pytest.fail("missing %s: run tests/golden/make_dirk_sphere.py" % GOLD)
    g = np.load(GOLD)
    pr = W.sphere(nq=2, nr=1, m=1, p=2, r0=0.5, r1=2.0)
    u0, q0, uh0, ou, ouh = g["u0"], g["q0"], g["uh0"], g["u1"], g["uh1"]
    dt = float(g["dt"])
    base = FP64 if prec == "fp64" else MIXED
    ctx = lib.Context(pr, dict(base, newton_rtol=1e-12, newton_atol=0.0, lin_rtol=1e-12, restart=60,
                               max_iters=4000, max_newton=40))
    u, q, uh = to_dev(u0), to_dev(q0), to_dev(uh0)
    for stage in (1, 2, 3):
        st = ctx.dirk_stage(stage, dt, u, q, uh)
        assert st["res"] <= 1e-12 * st["res0"]
    gu, guh = u.cpu().numpy(), uh.cpu().numpy()
    e_state = max(rel2(gu, ou), rel2(guh, ouh))
    e_inc = rel2(gu - u0, ou - u0)
    print("sphere %s DIRK step rel L2: state %.2e, increment %.2e, oracle Newton %s"
          % (prec, e_state, e_inc, list(g["newton"])))
    if prec == "fp64":
        assert e_state <= 1e-10 and e_inc <= 1e-8
    else:
        assert e_state <= 1e-8 and e_inc <= 1e-6
    ctx.close()


def test_sphere_rejects_unsupported_options(lib):
    pr = W.sphere(nq=1, nr=1, m=2, p=2)
    for bad in (dict(precision=1, tc_mode=2), dict(condense_layers=1)):
        with pytest.raises(lib.MehdgError):
            lib.Context(pr, bad)
    pr = W.sphere(nq=1, nr=1, m=2, p=3)     # m p = 6: M_J^-1 would not fit in shared memory
    with pytest.raises(lib.MehdgError):
        lib.Context(pr, FP64)
