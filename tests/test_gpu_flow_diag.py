"""Taylor-Green diagnostics (Sec. 5.3, eq. C5321) through the C ABI (mehdg_flow_integrals)
against the oracle's flow_integrals on the same seeded states.

The states come from the oracle (its lifted initial condition) or from the seeded generator
in workloads, never from the CUDA path.  Bar: 1e-12 relative on each integral (the same
quadrature, summed in a different order).  Box meshes in 2D and 3D with p = 1, 2, 3, and the
curved shell (per-point weights).
"""
import ctypes

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


def to_dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


CASES = {
    "tgv_4cubed_p2": lambda: W.tgv(nmac=4, Re=100.0),
    "tgv_3cubed_p3_m1": lambda: W.tgv(nmac=3, m=1, p=3, Re=100.0),
    "mms2d_p1_m3": lambda: W.mms(dim=2, nmac=3, m=3, p=1),
    "mms2d_p3": lambda: W.mms(dim=2, nmac=2, m=2, p=3),
    "sphere_p2": lambda: W.sphere(nq=2, nr=2, m=2, p=2),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_flow_integrals_match_oracle(lib, case):
    pr = CASES[case]()
    P = solve.Problem(pr)
    if pr["name"] == "tgv":
        u, q, _ = solve.initial_state(P, lift=True)
        du, _ = W.perturbation(pr, 11, amp=1e-3)
        u = u + du
    else:
        u, q, _ = W.random_state(pr, 7)
    ref = solve.flow_integrals(P, u, q)
    ctx = lib.Context(pr, dict(precision=0, precond=1, apply_mode=0))
    du_, dq_ = to_dev(u), to_dev(q)
    got = ctx.flow_integrals(du_, dq_)
    print(case, "GPU", got, "oracle", ref)
    for g, r in zip(got, ref):
        assert abs(g - r) <= 1e-12 * abs(r), (g, r)
    # the same state gives the same bits (fixed-order sums)
    assert ctx.flow_integrals(du_, dq_) == got
    ctx.close()


def test_tgv_diagnostics_of_the_initial_state(lib):
    """The library's own lifted TGV initial state gives E_k / V0^2 and eps L / V0^3 within 1e-3
    of the closed-form field's (1/8 and 3/4 Re^-1 up to O(M^2) density weighting; 4^3 macros)."""
    pr = W.tgv(nmac=4, Re=100.0)
    ctx = lib.Context(pr, dict(precision=0, precond=1, apply_mode=0))
    u, q, _ = ctx.init_state(None, None, lift=True)
    ek, eps = ctx.tgv_diagnostics(u, q, V0=0.1)
    print("E_k", ek, "eps", eps)
    assert abs(ek / 0.125 - 1.0) < 3e-3
    assert abs(eps / (0.75 / 100.0) - 1.0) < 5e-3
    ctx.close()


def test_flow_integrals_rejects_null_pointers(lib):
    pr = W.mms(dim=2, nmac=2, m=2, p=2)
    ctx = lib.Context(pr, dict(precision=0))
    u, q, _ = ctx.new_state()
    out = (ctypes.c_double * 3)()
    assert ctx.lib.mehdg_flow_integrals(ctx.h, None, ctypes.c_void_p(q.data_ptr()), out) == -1
    assert ctx.lib.mehdg_flow_integrals(ctx.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                        None) == -1
    ctx.close()
