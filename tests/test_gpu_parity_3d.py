"""3D end-to-end parity of the CUDA path (through the C ABI) with the FP64 oracle.

Cases: the Taylor-Green vortex (Sec. 5.3, periodic) and the manufactured solution
(Dirichlet) on 2^3 macro-elements of 2^3 hexes, p = 2, i.e. the macro-element of
the 3D configurations (Nu = 625, Nt = 750) on the smallest mesh with interior
faces in every direction.  Compared in relative L2 over the whole vector:

- the initial state of mehdg_init_state for the TGV field with the lifted gradient
  (q solving R_Q = 0) against the oracle's;
- one Newton linear step (eq. C312 by second-layer condensation, FGMRES to 1e-13,
  recovery, Algorithm 1) from an identical state: dUh, dU, dQ within 1e-10 on the
  FP64 path.  On the mixed path the Jacobian blocks themselves are assembled and
  condensed in FP32, so its linear step is the FP64 step of a perturbed matrix: it
  is held to the FP32 level of that perturbation, cond(S)-scaled (see below), and
  the FP64 Newton residual removes the difference at convergence;
- one DIRK3 step (eq. C242) of the TGV, every stage to |R_F| <= 1e-12 |R_F^0|:
  end state within 1e-10 (FP64) and 1e-8 (mixed) of the oracle's, and the step's
  increment u^{n+1} - u^n within 1e-8 (FP64) and 1e-6 (mixed) of the oracle's.
  The oracle's values come from tests/golden/make_dirk3d_tgv.py (oracle only).
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLD = os.path.join(os.path.dirname(__file__), "golden", "dirk3d_tgv_2cubed_p2.npz")


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


def rel2(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


FP64 = dict(precision=0, precond=1, apply_mode=0)
FP64SP = dict(precision=0, precond=1, apply_mode=2)      # row-compressed Algorithm 2 (the bench's FP64 form)
MIXED = dict(precision=1, precond=1, apply_mode=1, precond_bf16=1, refine_iters=1, tc_mode=4)   # the bench's mixed form
CASES3D = {"tgv": lambda: W.tgv(nmac=2, m=2, p=2), "mms": lambda: W.mms(dim=3, nmac=2, m=2, p=2)}
SHIFT = 0.5
_oracle_cache = {}


def _oracle_linear_step(case):
    if case not in _oracle_cache:
        pr = CASES3D[case]()
        P = solve.Problem(pr)
        u, q, uh = W.random_state(pr, 21)
        blks, geos, _, _ = solve.global_assemble(P, u, q, uh)
        dU, dQ, dUh, _, cond = solve.linear_step(P, blks, geos, shift=SHIFT, precond="direct")
        condS = max(np.linalg.cond(cond[e]["S"]) for e in (0, P.E - 1))
        _oracle_cache[case] = (pr, P, (u, q, uh), (dU, dQ, dUh), condS)
    return _oracle_cache[case]


@pytest.mark.parametrize("prec", ["fp64", "fp64sp", "mixed"])
@pytest.mark.parametrize("case", sorted(CASES3D))
def test_newton_linear_step_3d(lib, case, prec):
    pr, P, (u, q, uh), (dU, dQ, dUh), condS = _oracle_linear_step(case)
    # FGMRES to 1e-13 on the FP64 operator; the mixed path's outer operator is the FP32-stored
    # A^T_i (FP64 accumulation), whose rounding puts the reachable residual near 1e-7
    base = {"fp64": FP64, "fp64sp": FP64SP, "mixed": MIXED}[prec]
    opts = dict(base, lin_rtol=1e-6 if prec == "mixed" else 1e-13, lin_atol=0.0, restart=60, max_iters=4000)
    ctx = lib.Context(pr, opts)
    ctx.assemble(to_dev(u), to_dev(q), to_dev(uh))
    b = ctx.condense(shift=SHIFT)
    duh, st = ctx.linear_solve(b)
    du, dq = ctx.recover(duh)
    e = [rel2(duh.cpu().numpy(), dUh), rel2(du.cpu().numpy(), dU), rel2(dq.cpu().numpy(), dQ)]
    print("%s %s linear step rel L2 (dUh, dU, dQ) = %s, FGMRES its %d, cond(S) %.2e"
          % (case, prec, ["%.2e" % x for x in e], st["fgmres_iters"], condS))
    if prec != "mixed":
        assert max(e) <= 1e-10
    else:
        # FP32 blocks: relative perturbation ~ 2^-24 per entry, amplified by the local
        # solves (cond(S)) and by the trace system; bound 64 cond(S) 2^-24, and never
        # looser than 1e-4
        assert max(e) <= min(64 * condS * 2.0 ** -24, 1e-4)
    ctx.close()


def _gold():
    if not os.path.exists(GOLD):
        pytest.fail("missing %s: run tests/golden/make_dirk3d_tgv.py" % GOLD)
    return np.load(GOLD)


def test_init_state_tgv_lifted_matches_oracle(lib):
    g = _gold()
    pr = W.tgv(nmac=2, m=2, p=2)
    ctx = lib.Context(pr, FP64)
    u, q, uh = ctx.init_state(None, None, lift=True)
    eu, eq, eh = rel2(u.cpu().numpy(), g["u0"]), rel2(q.cpu().numpy(), g["q0"]), rel2(uh.cpu().numpy(), g["uh0"])
    print("TGV lifted initial state rel L2: u %.2e q %.2e uh %.2e" % (eu, eq, eh))
    assert eu <= 1e-14 and eh <= 1e-14 and eq <= 1e-12
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp64sp", "mixed"])
def test_dirk_step_3d_tgv_matches_oracle(lib, prec):
    g = _gold()
    pr = W.tgv(nmac=2, m=2, p=2)
    base = {"fp64": FP64, "fp64sp": FP64SP, "mixed": MIXED}[prec]
    opts = dict(base, newton_rtol=1e-12, newton_atol=0.0, lin_rtol=1e-12,
                restart=60, max_iters=4000, max_newton=40)
    ctx = lib.Context(pr, opts)
    u, q, uh = to_dev(g["u0"]), to_dev(g["q0"]), to_dev(g["uh0"])
    for stage in (1, 2, 3):
        st = ctx.dirk_stage(stage, float(g["dt"]), u, q, uh)
        assert st["res"] <= 1e-12 * st["res0"]
    gu, guh = u.cpu().numpy(), uh.cpu().numpy()
    e_state = max(rel2(gu, g["u1"]), rel2(guh, g["uh1"]))
    e_inc = rel2(gu - g["u0"], g["u1"] - g["u0"])
    print("%s DIRK step rel L2: state %.2e, increment %.2e" % (prec, e_state, e_inc))
    if prec != "mixed":
        assert e_state <= 1e-10 and e_inc <= 1e-8
    else:
        assert e_state <= 1e-8 and e_inc <= 1e-6
    ctx.close()


def test_newton_step_calls_compose_the_dirk_stage(lib):
    """mehdg_stage_begin + mehdg_newton_step (until converged) + mehdg_stage_end give the
    same DIRK step as three mehdg_dirk_stage calls."""
    g = _gold()
    pr = W.tgv(nmac=2, m=2, p=2)
    opts = dict(FP64, newton_rtol=1e-10, lin_rtol=1e-12, restart=60, max_iters=4000)
    outs = []
    for mode in ("stage", "step"):
        ctx = lib.Context(pr, opts)
        u, q, uh = to_dev(g["u0"]), to_dev(g["q0"]), to_dev(g["uh0"])
        n = 0
        for stage in (1, 2, 3):
            if mode == "stage":
                n += ctx.dirk_stage(stage, float(g["dt"]), u, q, uh)["newton_steps"]
            else:
                st = ctx.stage_begin(stage, float(g["dt"]), u, q, uh)
                while not st["converged"]:
                    st = ctx.newton_step(u, q, uh)
                    n += 1
                ctx.stage_end(u)
        outs.append((u.cpu().numpy(), n))
        ctx.close()
    assert outs[0][1] == outs[1][1]
    assert rel2(outs[1][0], outs[0][0]) <= 1e-14
