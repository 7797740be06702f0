"""Batches of independent problems of uneven size (the batching form of the hot path).

* The persistent work-queue LU (mehdg_lu_queue) on matrices of uneven size, every panel
  width: the pivot sequence of the oracle's LU and its factors (FP64 within 1e-10 relative;
  FP32 through P A = L U within a multiple of n u_32 |A|), and SINGULAR on a zero column.
* The batch's steady solve (lockstep Newton rounds, graph replays, one queued LU per round):
  every problem's end state zeroes the oracle's residual to the solve's tolerance, and equals
  the state the same problem reaches alone (mehdg_dirk_stage, stage 0).
"""
import numpy as np
import pytest

import workloads as W
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


def rel2(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("nb", [8, 16, 32])
def test_lu_queue_matches_oracle_fp64(lib, nb):
    rng = np.random.default_rng(nb)
    sizes = [40, 625, 135, 300, 17, 625, 33]      # uneven, ragged panels, tails
    mats = [rng.uniform(-1, 1, size=(n, n)) for n in sizes]
    dev = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in mats]
    perms = lib.lu_queue(dev, nb=nb)
    for a, d, p in zip(mats, dev, perms):
        LU, piv = solve.lu_factor(a)
        assert np.array_equal(p.cpu().numpy(), piv)
        g = d.cpu().numpy()
        assert np.abs(g - LU).max() <= 1e-10 * np.abs(LU).max()


def test_lu_queue_fp32_reconstructs(lib):
    rng = np.random.default_rng(3)
    sizes = [625, 135, 1715, 300]
    mats = [rng.uniform(-1, 1, size=(n, n)).astype(np.float32) for n in sizes]
    dev = [torch.tensor(a, device="cuda") for a in mats]
    perms = lib.lu_queue(dev, nb=16)
    for a, d, p in zip(mats, dev, perms):
        n = a.shape[0]
        g = d.cpu().numpy().astype(np.float64)
        L = np.tril(g, -1) + np.eye(n)
        U = np.triu(g)
        PA = a.astype(np.float64)[p.cpu().numpy()]
        err = np.abs(PA - L @ U).max() / np.abs(a).max()
        assert err <= 8 * n * 2.0 ** -24, (n, err)


def test_lu_queue_reports_singular(lib):
    a = torch.rand(64, 64, dtype=torch.float64, device="cuda")
    b = torch.rand(100, 100, dtype=torch.float64, device="cuda")
    b[:, 7] = 0.0
    with pytest.raises(lib.MehdgError, match="SINGULAR"):
        lib.lu_queue([a, b], nb=16)


# uneven: 3D p = 1 and p = 2, 2D p = 3 and p = 2 (velocity amplitude 0.1: the single-problem
# Newton iteration converges from the perturbed field on these coarse meshes)
PROBLEMS = [lambda: W.mms(dim=3, nmac=2, m=2, p=1, vel=0.1), lambda: W.mms(dim=3, nmac=2, m=2, p=2, vel=0.1),
            lambda: W.mms(dim=2, nmac=3, m=2, p=3, vel=0.1), lambda: W.mms(dim=2, nmac=2, m=2, p=2, vel=0.1)]
FP64 = dict(precision=0, precond=1, apply_mode=0, newton_rtol=1e-11, newton_atol=0.0, lin_rtol=1e-10,
            restart=60, max_iters=4000, max_newton=60)
MIXED = dict(precision=1, precond=1, apply_mode=1, tc_mode=4, precond_bf16=1, refine_iters=2, newton_rtol=1e-11,
             newton_atol=0.0, lin_rtol=1e-10, restart=60, max_iters=4000, max_newton=60)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_steady_solve_matches_oracle_and_single_solves(lib, prec):
    opts = FP64 if prec == "fp64" else MIXED
    probs = [mk() for mk in PROBLEMS]
    batch = lib.Batch(probs, opts)
    tiles = batch.tiles()
    assert {t[0] for t in tiles} == {c.info["Nu"] for c in batch.contexts}
    for n, fp64, nb, ms in tiles:
        assert nb in ms and ms[nb] == min(ms.values())
    states, singles = [], []
    for i, (pr, c) in enumerate(zip(probs, batch.contexts)):
        du, duh = W.perturbation(pr, 500 + i, amp=1e-2)
        du, duh = torch.tensor(du, device="cuda"), torch.tensor(duh, device="cuda")
        states.append(c.init_state(du, duh, lift=True))
        one = lib.Context(pr, opts)
        s = one.init_state(du, duh, lift=True)
        st = one.dirk_stage(0, 0.0, *s)
        assert st["res"] <= 1e-11 * st["res0"]
        singles.append([x.cpu().numpy() for x in s])
        one.close()
    stats, rounds = batch.steady_solve(states)
    print("%s batch: rounds %d, graph replays %d, Newton steps %s, tiles %s"
          % (prec, rounds, batch.graph_replays(), [s["newton_steps"] for s in stats], tiles))
    assert batch.graph_replays() > 0
    for i, (pr, s, st) in enumerate(zip(probs, states, stats)):
        assert st["converged"] and st["res"] <= 1e-11 * st["res0"]
        gu, gq, guh = (x.cpu().numpy() for x in s)
        P = solve.Problem(pr)
        du, duh = W.perturbation(pr, 500 + i, amp=1e-2)
        u0, q0, uh0 = solve.initial_state(P, lift=True)
        _, _, n0, _ = solve.global_assemble(P, u0 + du, q0, uh0 + duh, want_jac=False)
        _, _, n1, _ = solve.global_assemble(P, gu, gq, guh, want_jac=False)
        e_single = max(rel2(gu, singles[i][0]), rel2(guh, singles[i][2]))
        print("  problem %d (E %d, Nu %d): oracle residual %.2e of the initial, vs single solve %.2e"
              % (i, P.E, P.ns * P.Np, n1["RF"] / n0["RF"], e_single))
        assert n1["RF"] <= 1e-10 * n0["RF"]
        assert e_single <= 1e-9
    batch.close()


def test_batch_retries_a_step_that_leaves_the_physical_states(lib):
    """Velocity amplitude 0.3 on the 2 x 2 macro mesh: the second pseudo-time Newton step of the
    plain iteration reaches negative pressures (the oracle's newton_ser and mehdg_dirk_stage
    both end there with a non-finite residual).  The batch undoes that step, retries it with a
    ten times smaller pseudo-time step, and converges; its end state zeroes the oracle's
    residual."""
    pr = W.mms(dim=2, nmac=2, m=2, p=2)
    opts = dict(FP64, newton_rtol=1e-10)
    batch = lib.Batch([pr], opts)
    c = batch.contexts[0]
    du, duh = W.perturbation(pr, 503, amp=1e-3)
    s = c.init_state(torch.tensor(du, device="cuda"), torch.tensor(duh, device="cuda"), lift=True)
    stats, rounds = batch.steady_solve([s])
    print("retry batch:", stats[0], rounds)
    assert stats[0]["converged"] and stats[0]["status"] & 4
    P = solve.Problem(pr)
    u0, q0, uh0 = solve.initial_state(P, lift=True)
    _, _, n0, _ = solve.global_assemble(P, u0 + du, q0, uh0 + duh, want_jac=False)
    gu, gq, guh = (x.cpu().numpy() for x in s)
    _, _, n1, _ = solve.global_assemble(P, gu, gq, guh, want_jac=False)
    assert n1["RF"] <= 1e-9 * n0["RF"]
    batch.close()
