"""Parity at the full size of the steady MMS cube (3D, 8^3 macro-elements of 2^3 hexes,
p = 2: 512 macros, Nu = 625, Nt = 750, 216,000 trace unknowns) with the options and
launch configuration of the default bench line (mixed precision, stored A^T_i, the
multi-level preconditioner with BF16 inner copies, one refinement sweep).

The oracle needs about 3.5 s per macro-element, so it is run on sampled macros (a
corner, an interior macro, the opposite corner); the rest is checked through properties
that hold at any size:

* blocks and local residuals of the sampled macros against the oracle's assembly
  (FP32 blocks within FP32 rounding, FP64 residuals to FP64 accuracy, the same bounds as
  the small mixed-precision tests);
* the explicit local operators A^T_i and local condensed right-hand sides of the sampled
  macros against the oracle's one- and second-layer condensation (FP32 blocks through
  S^-1: 7.7e-6 observed on the same macro type, bound 1e-3);
* the full-size trace apply at the trace unknowns of each sampled macro against a plain
  numpy sum of the stored operators of every macro touching them (face reduction and
  FP32 products, bound 1e-4);
* FGMRES: the true residual of its solution, recomputed with the apply, meets the
  requested relative tolerance;
* recovery of the sampled macros against the oracle's eq. Csc4, and the residual of the
  refined local solve with the unfactored S below the FP32 level.
"""
import numpy as np
import pytest

import workloads as W
from oracle import assemble as asm
from oracle import solve

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SAMPLED = (0, 219, 511)   # corner (three boundary faces), interior (3, 3, 3), opposite corner
SHIFT = 0.3
LIN_RTOL = 1e-3


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


def test_full_size_mixed_path_sampled_against_oracle(lib):
    pr = W.mms(dim=3, nmac=8, m=2, p=2)
    P = solve.Problem(pr)
    assert P.E == 512
    Nu, Nt = P.ns * P.Np, P.ns * P.Nth
    ntr = P.F * P.ns * P.Nfn
    assert (Nu, Nt, ntr) == (625, 750, 216000)
    opts = dict(precision=1, apply_mode=1, precond=1, precond_bf16=1, refine_iters=1, inner_iters=10,
                restart=60, lin_rtol=LIN_RTOL, max_iters=3000)
    u, q, uh = W.random_state(pr, 5)
    ctx = lib.Context(pr, opts)
    try:
        ctx.assemble(to_dev(u), to_dev(q), to_dev(uh))
        maps = [P.maps[e].reshape(-1) for e in range(P.E)]

        # ---- sampled blocks and residuals (oracle assembly of those macros only)
        geos, blks = {}, {}
        for e in SAMPLED:
            geo = P.geometry(e)
            b = asm.assemble_macro(geo, P.phys, u[e], q[e], P.local_trace(e, uh), None, P.source(geo),
                                   P.bfaces(e, geo))
            geos[e], blks[e] = geo, b
            assert rel(ctx.get_block(0, e).reshape(Nu, Nu), b["Auu"]) < 3e-6
            assert rel(ctx.get_block(9, e).reshape(Nt, Nt), b["Ahh"]) < 3e-6
            assert rel(ctx.get_block(10, e), b["RQ"].reshape(-1)) < 1e-10
            assert rel(ctx.get_block(11, e), b["RU"].reshape(-1)) < 1e-10
            assert rel(ctx.get_block(12, e), b["RUh"].reshape(-1)) < 1e-10

        # ---- condensation: A^T_i and the local condensed right-hand side
        bhat = ctx.condense(shift=SHIFT)
        cond = {}
        for e in SAMPLED:
            A1, _ = solve.condense_one_layer(geos[e], blks[e], shift=SHIFT)
            cond[e] = solve.condense_second_layer(geos[e], blks[e], shift=SHIFT)
            assert rel(ctx.get_block(9, e).reshape(Nt, Nt), A1) < 1e-3
            assert rel(ctx.get_block(16, e), cond[e]["bhat"]) < 1e-3

        # ---- full-size trace apply, checked at the unknowns of each sampled macro
        x = W.random_vector(ntr, 9)
        y = ctx.apply(to_dev(x)).cpu().numpy()
        for e in SAMPLED:
            touching = [f for f in range(P.E) if np.isin(maps[f], maps[e]).any()]
            assert e in touching and 2 <= len(touching) <= 7
            yref = np.zeros(ntr)
            for f in touching:
                Af = ctx.get_block(9, f).reshape(Nt, Nt)
                yref[maps[f]] += Af @ x[maps[f]]
            assert rel(y[maps[e]], yref[maps[e]]) < 1e-4

        # ---- FGMRES with the multi-level preconditioner (BF16 inner copies)
        duh, st = ctx.linear_solve(bhat)
        assert st["fgmres_iters"] > 0
        r = bhat - ctx.apply(duh)
        assert float(r.norm() / bhat.norm()) <= LIN_RTOL * (1 + 1e-6)

        # ---- recovery (eq. Csc4) of the sampled macros
        duh_h = duh.cpu().numpy()
        du, dq = ctx.recover(duh)
        du, dq = du.cpu().numpy(), dq.cpu().numpy()
        for e in SAMPLED:
            ou, oq = solve.recover(geos[e], blks[e], cond[e], duh_h[maps[e]])
            assert rel(du[e].reshape(-1), ou) < 1e-3
            assert rel(dq[e].reshape(-1), oq) < 1e-3
            S0 = ctx.get_block(17, e).reshape(Nu, Nu)
            C = ctx.get_block(4, e).reshape(Nu, Nt)
            rhs = ctx.get_block(13, e) + C @ duh_h[maps[e]]
            res = np.linalg.norm(rhs - S0 @ du[e].reshape(-1)) / np.linalg.norm(rhs)
            # the FP32 LU solve alone leaves a relative residual near n u32 ~ 1e-6 to 1e-5;
            # one sweep with the FP64 residual gains a factor of about kappa(S) u32
            assert res < 1e-7
    finally:
        ctx.close()


def _sampled_blocks(ctx, P, u, q, uh, sampled, tol_blk, tol_res):
    Nu, Nt = P.ns * P.Np, P.ns * P.Nth
    out = {}
    for e in sampled:
        geo = P.geometry(e)
        b = asm.assemble_macro(geo, P.phys, u[e], q[e], P.local_trace(e, uh), None, P.source(geo), P.bfaces(e, geo))
        out[e] = (geo, b)
        assert rel(ctx.get_block(0, e).reshape(Nu, Nu), b["Auu"]) < tol_blk
        assert rel(ctx.get_block(1, e).reshape(Nu, Nu), b["Auq"][0]) < tol_blk
        assert rel(ctx.get_block(9, e).reshape(Nt, Nt), b["Ahh"]) < tol_blk
        assert rel(ctx.get_block(10, e), b["RQ"].reshape(-1)) < tol_res
        assert rel(ctx.get_block(11, e), b["RU"].reshape(-1)) < tol_res
        assert rel(ctx.get_block(12, e), b["RUh"].reshape(-1)) < tol_res
    return out


def test_full_size_tgv_fp64_sampled_against_oracle(lib):
    """The headline configuration (16^3 TGV, 4096 macros, the bench's plain FP64 options with
    the row-compressed Algorithm-2 apply): blocks, residuals and the condensed operators S, B,
    C, D, g, h, b^ of sampled macros (a corner, an interior macro, the opposite corner; the
    mesh is periodic, so every macro is interior) against the oracle at 1e-11 / 1e-10."""
    pr = W.tgv(nmac=16)
    P = solve.Problem(pr)
    assert P.E == 4096
    Nu, Nt = P.ns * P.Np, P.ns * P.Nth
    opts = dict(precision=0, apply_mode=2, precond=1, inner_iters=10, restart=60, lin_rtol=LIN_RTOL, max_iters=3000)
    u, q, uh = W.random_state(pr, 17)
    ctx = lib.Context(pr, opts)
    try:
        ctx.assemble(to_dev(u), to_dev(q), to_dev(uh))
        sampled = (0, 2184, 4095)
        ob = _sampled_blocks(ctx, P, u, q, uh, sampled, 1e-11, 1e-11)
        ctx.condense(shift=SHIFT)
        for e in sampled:
            c = solve.condense_second_layer(ob[e][0], ob[e][1], shift=SHIFT)
            assert rel(ctx.get_block(4, e).reshape(Nu, Nt), c["C"]) < 1e-11
            assert rel(ctx.get_block(5, e).reshape(Nt, Nu), c["B"]) < 1e-11
            assert rel(ctx.get_block(9, e).reshape(Nt, Nt), c["D"]) < 1e-11
            assert rel(ctx.get_block(13, e), c["g"]) < 1e-11
            assert rel(ctx.get_block(14, e), c["h"]) < 1e-11
            assert np.array_equal(ctx.get_block(15, e).astype(int), c["piv"])
            assert rel(ctx.get_block(0, e).reshape(Nu, Nu), c["LU"]) < 1e-10
            assert rel(ctx.get_block(16, e), c["bhat"]) < 1e-10
    finally:
        ctx.close()


def test_full_size_sphere_mixed_sampled_against_oracle(lib):
    """The sphere configuration at full size (6 x 8^2 x 16 = 6144 curved macros, the mixed form
    that fits it): FP32 blocks of sampled macros (at the wall on a cube-panel corner, in the
    middle of the shell, at the far field) within the FP32 level, their FP64 residuals to 1e-10,
    and the local condensed right-hand side through the FP32 local factors within 1e-3."""
    pr = W.sphere()
    P = solve.Problem(pr)
    assert P.E == 6144
    opts = dict(precision=1, apply_mode=1, precond=1, precond_bf16=1, refine_iters=1, tc_mode=4, inner_iters=10,
                restart=60, lin_rtol=LIN_RTOL, max_iters=3000)
    u, q, uh = W.random_state(pr, 19)
    ctx = lib.Context(pr, opts)
    try:
        ctx.assemble(to_dev(u), to_dev(q), to_dev(uh))
        sampled = (0, 2524, 6143)
        ob = _sampled_blocks(ctx, P, u, q, uh, sampled, 3e-6, 1e-10)
        ctx.condense(shift=SHIFT)
        for e in sampled:
            c = solve.condense_second_layer(ob[e][0], ob[e][1], shift=SHIFT)
            assert rel(ctx.get_block(16, e), c["bhat"]) < 1e-3
    finally:
        ctx.close()
