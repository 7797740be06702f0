"""Simplicial macro-elements (P_p on m-refined simplices, the paper's element type): parity of
the CUDA path (through the C ABI) with the FP64 oracle.

The oracle builds its own reference simplex, quadrature, mesh and face matching
(oracle/simplex.py); the library its own (csrc/simplex.cu, table-driven kernels in
csrc/assemble.cu).  The same seeded states go to both.  Tolerances as for the box meshes:
blocks and residuals 1e-11 relative to the largest entry, the linear step 1e-10 relative L2,
the DIRK end state 1e-10 relative L2.
"""
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


def simplex(pr):
    pr = dict(pr)
    pr["mesh_kind"] = W.MESH_SIMPLEX
    return pr


CASES = {
    "2d_p2_m2_dirichlet": (lambda: simplex(W.mms(dim=2, nmac=2, m=2, p=2)), [0, 3, 7]),
    "2d_p3_m1_wall": (lambda: simplex(W.couette2d(nmac=2, m=1, p=3)), [0, 5]),
    "3d_p1_m2_dirichlet": (lambda: simplex(W.mms(dim=3, nmac=1, m=2, p=1)), [0, 2, 5]),
    "3d_p2_m1_periodic": (lambda: simplex(W.periodic_uniform(dim=3, nmac=2, m=1, p=2)), [0, 17, 47]),
}
FP64 = dict(precision=0, precond=1, apply_mode=0)


@pytest.mark.parametrize("case", sorted(CASES))
def test_simplex_assembly_blocks_and_residuals(lib, case):
    mk, macros = CASES[case]
    pr = mk()
    P = solve.Problem(pr)
    u, q, uh = W.random_state(pr, 23)
    hist = 0.05 * np.ones_like(u)
    ctx = lib.Context(pr, FP64)
    assert ctx.info["n_macro"] == P.E and ctx.info["n_face"] == P.F and ctx.info["Nth"] == P.Nth
    norms = ctx.assemble(to_dev(u), to_dev(q), to_dev(uh), coef=0.4, hist=to_dev(hist), supg_time=1)
    tt = dict(coef=0.4, hist=hist, supg_time=True)
    _, _, onrm, _ = solve.global_assemble(P, u, q, uh, tt, want_jac=False)
    print(case, "GPU norms", norms, "oracle", [onrm["RQ"], onrm["RU"], onrm["RUh"], onrm["RF"]])
    Nu, Nt, d = P.ns * P.Np, P.ns * P.Nth, P.d
    errs = []
    for e in macros:
        geo = P.geometry(e)
        b = asm.assemble_macro(geo, P.phys, u[e], q[e], P.local_trace(e, uh),
                               dict(coef=0.4, hist=hist[e], supg_time=True), P.source(geo), P.bfaces(e, geo))
        errs.append([rel(ctx.get_block(0, e).reshape(Nu, Nu), b["Auu"]),
                     max(rel(ctx.get_block(1 + k, e).reshape(Nu, Nu), b["Auq"][k]) for k in range(d)),
                     rel(ctx.get_block(4, e).reshape(Nu, Nt), b["Auh"]),
                     rel(ctx.get_block(5, e).reshape(Nt, Nu), b["Ahu"]),
                     max(rel(ctx.get_block(6 + k, e).reshape(Nt, Nu), b["Ahq"][k]) for k in range(d)),
                     rel(ctx.get_block(9, e).reshape(Nt, Nt), b["Ahh"]),
                     rel(ctx.get_block(10, e), b["RQ"].reshape(-1)),
                     rel(ctx.get_block(11, e), b["RU"].reshape(-1)),
                     rel(ctx.get_block(12, e), b["RUh"].reshape(-1))])
    print(case, "block errors (Auu, Auq, Auh, Ahu, Ahq, Ahh, RQ, RU, RUh) per macro:",
          [["%.1e" % x for x in r] for r in errs])
    assert np.allclose(norms, [onrm["RQ"], onrm["RU"], onrm["RUh"], onrm["RF"]], rtol=1e-11)
    assert max(max(r) for r in errs) < 1e-11
    ctx.close()


def test_simplex_free_stream_preservation(lib):
    """A uniform state on a periodic tetrahedral mesh gives R = 0 to rounding."""
    pr = simplex(W.periodic_uniform(dim=3, nmac=2, m=2, p=1))
    ctx = lib.Context(pr, FP64)
    u, q, uh = ctx.init_state(None, None, lift=False)
    norms = ctx.assemble(u, q, uh)
    print("simplex free stream |R|", norms)
    assert norms[3] < 1e-13
    ctx.close()


def test_simplex_initial_state_matches_oracle(lib):
    """The closed form at the nodes, the first owner's trace and the lifted gradient."""
    pr = simplex(W.mms(dim=2, nmac=2, m=2, p=2))
    P = solve.Problem(pr)
    ou, oq, ouh = solve.initial_state(P, lift=True)
    ctx = lib.Context(pr, FP64)
    u, q, uh = ctx.init_state(None, None, lift=True)
    eu, eq, eh = rel2(u.cpu().numpy(), ou), rel2(q.cpu().numpy(), oq), rel2(uh.cpu().numpy(), ouh)
    print("simplex initial state rel L2: u %.2e q %.2e uh %.2e" % (eu, eq, eh))
    assert eu <= 1e-14 and eh <= 1e-14 and eq <= 1e-11
    ctx.close()


@pytest.mark.parametrize("case", ["2d_p2_m2_dirichlet", "3d_p1_m2_dirichlet"])
def test_simplex_newton_linear_step(lib, case):
    """Condensation with the per-macro liftings, factorisation, FGMRES with the multi-level
    preconditioner on the trace system (Algorithm 2) and recovery, against the oracle's dense
    solve, about the closed form plus a seeded 1e-2 perturbation."""
    pr = CASES[case][0]()
    P = solve.Problem(pr)
    u, q, uh = solve.initial_state(P, lift=True)
    du, duh = W.perturbation(pr, 43, amp=1e-2)
    u, uh = u + du, uh + duh
    blks, geos, _, _ = solve.global_assemble(P, u, q, uh)
    dU, dQ, dUh, _, _ = solve.linear_step(P, blks, geos, shift=0.5, precond="direct")
    ctx = lib.Context(pr, dict(FP64, lin_rtol=1e-13, lin_atol=0.0, restart=60, max_iters=3000))
    ctx.assemble(to_dev(u), to_dev(q), to_dev(uh))
    b = ctx.condense(shift=0.5)
    x, st = ctx.linear_solve(b)
    gu, gq = ctx.recover(x)
    e = [rel2(x.cpu().numpy(), dUh), rel2(gu.cpu().numpy(), dU), rel2(gq.cpu().numpy(), dQ)]
    print("simplex %s linear step rel L2 (dUh, dU, dQ) = %s, FGMRES its %d" % (case, ["%.2e" % v for v in e],
                                                                              st["fgmres_iters"]))
    assert max(e) <= 1e-10
    ctx.close()


def test_simplex_dirk_step_matches_oracle(lib):
    """One DIRK3 step (three stages, Newton to 1e-12) of the 2D manufactured-solution problem on
    triangular macro-elements from the closed form plus a seeded perturbation."""
    from oracle import fields
    pr = CASES["2d_p2_m2_dirichlet"][0]()
    P = solve.Problem(pr)
    du, duh = W.perturbation(pr, 45, amp=1e-3)
    # the initial state rule of mehdg_init_state (lift off) with the oracle's spaces
    u0 = np.array([fields.mms_u(P.geometry(e).xn, pr["field_par"], pr["gamma"]) for e in range(P.E)]) + du
    uh0 = np.zeros(P.F * P.ns * P.Nfn)
    for f, own in enumerate(P.mesh.face_owners()):
        e, fl = own[0]
        for s in range(P.ns):
            uh0[(f * P.ns + s) * P.Nfn:(f * P.ns + s + 1) * P.Nfn] = u0[e, s, P.mesh.fnodes[fl]]
    uh0 = uh0 + duh
    q0 = np.zeros((P.E, P.d, P.ns, P.Np))
    ou, oq, ouh = solve.dirk_step(P, u0, q0, uh0, 0.05, rtol=1e-12, atol=1e-14, lin_rtol=1e-13,
                                  precond="direct")[:3]
    ctx = lib.Context(pr, dict(FP64, newton_rtol=1e-12, newton_atol=1e-14, lin_rtol=1e-13, restart=60,
                               max_iters=3000, max_newton=30))
    u, q, uh = ctx.init_state(to_dev(du), to_dev(duh), lift=False)
    assert rel2(u.cpu().numpy(), u0) < 1e-14 and rel2(uh.cpu().numpy(), uh0) < 1e-14
    for stage in (1, 2, 3):
        ctx.dirk_stage(stage, 0.05, u, q, uh)
    eu, eh = rel2(u.cpu().numpy(), ou), rel2(uh.cpu().numpy(), ouh)
    print("simplex DIRK step rel L2: u %.2e uh %.2e" % (eu, eh))
    assert eu <= 1e-10 and eh <= 1e-10
    ctx.close()
