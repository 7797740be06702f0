"""Edge cases and argument checks of the C ABI on the GPU: invalid problems and calls
are refused with an error status (no context, no launch), a zero right-hand side gives
the zero solution without iterations, and the trace apply is linear."""
import ctypes

import numpy as np
import pytest

import workloads as W

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


@pytest.mark.parametrize("change", [dict(p=4), dict(m=0), dict(p=0), dict(gamma=1.0), dict(Re=0.0)])
def test_invalid_problems_are_refused(lib, change):
    pr = W.mms(dim=2, nmac=2, m=2, p=2)
    pr.update(change)
    with pytest.raises(lib.MehdgError):
        lib.Context(pr)


def test_invalid_mesh_sizes_are_refused(lib):
    pr = W.mms(dim=2, nmac=2, m=2, p=2)
    pr["nmac"][0] = 0
    with pytest.raises(lib.MehdgError):
        lib.Context(pr)


def test_explicit_operator_too_large_for_shared_memory_is_refused(lib):
    # 3D p = 3 macro-elements (Nu = 1715) need the Algorithm-2 apply in FP32
    with pytest.raises(lib.MehdgError):
        lib.Context(W.mms(dim=3, nmac=1, m=2, p=3), dict(precision=1, apply_mode=1))


def test_call_order_and_argument_checks(lib):
    pr = W.mms(dim=2, nmac=2, m=2, p=2)
    ctx = lib.Context(pr)
    n = ctx.info["n_trace"]
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.MehdgError):
        ctx.apply(x)                               # before mehdg_condense_factor
    u, q, uh = W.random_state(pr, 3)
    ctx.assemble(*[torch.as_tensor(a, device="cuda") for a in (u, q, uh)])
    ctx.condense(shift=0.5)
    f = ctx.lib.mehdg_apply_trace
    assert f(ctx.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr())) == -1   # x aliases y
    assert f(ctx.h, None, ctypes.c_void_p(x.data_ptr())) == -1
    with pytest.raises(lib.MehdgError):
        ctx.set_precond(7)
    with pytest.raises(lib.MehdgError):
        ctx.set_precond(2)                         # needs mehdg_mlp_setup
    with pytest.raises(lib.MehdgError):
        ctx.precondition(2, x)
    ctx.close()


@pytest.mark.parametrize("precision,apply_mode", [(0, 0), (1, 1)])
def test_zero_rhs_and_linearity(lib, precision, apply_mode):
    pr = W.mms(dim=3, nmac=2, m=2, p=1)
    ctx = lib.Context(pr, dict(precision=precision, apply_mode=apply_mode, precond=1, lin_rtol=1e-8))
    u, q, uh = W.random_state(pr, 4)
    ctx.assemble(*[torch.as_tensor(a, device="cuda") for a in (u, q, uh)])
    ctx.condense(shift=0.2)
    n = ctx.info["n_trace"]
    zero = torch.zeros(n, dtype=torch.float64, device="cuda")
    x, st = ctx.linear_solve(zero)
    assert st["fgmres_iters"] == 0 and float(x.abs().max()) == 0.0
    a = torch.as_tensor(W.random_vector(n, 1), device="cuda")
    b = torch.as_tensor(W.random_vector(n, 2), device="cuda")
    lhs = ctx.apply(2.0 * a - 3.0 * b).cpu().numpy()
    rhs = (2.0 * ctx.apply(a) - 3.0 * ctx.apply(b)).cpu().numpy()
    tol = 1e-13 if precision == 0 else 1e-5    # FP32 blocks: rounding of the products
    assert np.abs(lhs - rhs).max() <= tol * np.abs(rhs).max()
    ctx.close()


# ---------------------------------------------------------------- error statuses reached from the host

def test_nan_in_the_state_returns_nan_status(lib):
    """A non-finite entry in a host-prepared state: the stage's first residual is not
    finite and the nonlinear solve returns MEHDG_ERR_NAN without touching the solver."""
    pr = W.mms(dim=2, nmac=2, m=2, p=2)
    ctx = lib.Context(pr)
    u, q, uh = ctx.init_state(None, None)
    u[1, 0, 3] = float("nan")
    c = ctypes.c_void_p
    rc = ctx.lib.mehdg_dirk_stage(ctx.h, 0, 0.0, c(u.data_ptr()), c(q.data_ptr()), c(uh.data_ptr()), None)
    assert rc == -7 and b"non-finite" in ctx.lib.mehdg_last_error(ctx.h)
    st = lib.SolveStats()
    assert ctx.lib.mehdg_stage_begin(ctx.h, 1, 0.1, c(u.data_ptr()), c(q.data_ptr()), c(uh.data_ptr()),
                                     ctypes.byref(st)) == -7
    ctx.close()


def test_iteration_caps_return_not_converged(lib):
    """FGMRES capped at one iteration and Newton capped at one step return
    MEHDG_ERR_NOT_CONVERGED, leaving the last iterate in place (finite)."""
    pr = W.mms(dim=2, nmac=2, m=2, p=2)
    du, duh = W.perturbation(pr, 0, amp=1e-2)
    ctx = lib.Context(pr, dict(max_iters=1, lin_rtol=1e-12, precond=0))
    u, q, uh = ctx.init_state(torch.as_tensor(du, device="cuda"), torch.as_tensor(duh, device="cuda"))
    ctx.assemble(u, q, uh)
    b = ctx.condense(shift=0.5)
    x, st = ctx.linear_solve(b, allow_not_converged=True)
    assert st["fgmres_iters"] == 1 and bool(torch.isfinite(x).all())
    c = ctypes.c_void_p
    rc = ctx.lib.mehdg_linear_solve(ctx.h, c(b.data_ptr()), c(x.data_ptr()), None)
    assert rc == -5
    ctx.close()
    ctx = lib.Context(pr, dict(max_newton=1, newton_rtol=1e-13, lin_rtol=1e-3, precond=1))
    u, q, uh = ctx.init_state(torch.as_tensor(du, device="cuda"), torch.as_tensor(duh, device="cuda"))
    st = lib.SolveStats()
    rc = ctx.lib.mehdg_dirk_stage(ctx.h, 0, 0.0, c(u.data_ptr()), c(q.data_ptr()), c(uh.data_ptr()),
                                  ctypes.byref(st))
    assert rc == -5 and st.newton_steps == 1 and bool(torch.isfinite(u).all())
    ctx.close()


@pytest.mark.parametrize("n", [40, 300])
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_singular_matrix_returns_singular_status(lib, n, dtype):
    """mehdg_lu_batched on a batch where matrix 1 has an exactly zero column returns
    MEHDG_ERR_SINGULAR; the other matrices are factored (P A = L U).  n = 40 runs the
    small-matrix kernel, n = 300 the shared-memory panel kernel."""
    dt = getattr(torch, dtype)
    rng = np.random.default_rng(n)
    A = rng.normal(size=(3, n, n))
    A[1, :, n // 3] = 0.0
    Ad = torch.as_tensor(A, dtype=dt, device="cuda").contiguous()
    with pytest.raises(lib.MehdgError, match="SINGULAR"):
        lib.lu_batched(Ad)
    Ad = torch.as_tensor(A[[0, 2]], dtype=dt, device="cuda").contiguous()
    perm = lib.lu_batched(Ad).cpu().numpy()
    F = Ad.cpu().numpy().astype(np.float64)
    tol = 1e-12 if dtype == "float64" else 1e-4
    for b, src in enumerate((0, 2)):
        L = np.tril(F[b], -1) + np.eye(n)
        U = np.triu(F[b])
        PA = A[src][perm[b]]
        assert np.linalg.norm(PA - L @ U) <= tol * n * np.linalg.norm(A[src])
