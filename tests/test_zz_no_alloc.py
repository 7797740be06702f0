"""The allocation-free trace apply gives the same result as the context's apply.

mehdg_apply_trace_noalloc serves callers that cannot call cudaMalloc (a host
application that owns all device memory through its own pool and gives the
solver a fixed budget, or a loop that must not stall on an allocation).  It
takes every array from the caller and keeps its one scratch array in a fixed
array inside the library.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import solve

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

c_int, c_void_p = ctypes.c_int, ctypes.c_void_p


def _fn():
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg
    lib = ctypes.CDLL(pkg.LIB_PATH)
    f = lib.mehdg_apply_trace_noalloc
    f.restype = c_int
    f.argtypes = [c_int] * 5 + [c_void_p] * 10
    return pkg, f


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_noalloc_apply_matches_context_apply_twice():
    pkg, fn = _fn()
    pr = W.mms(dim=3, nmac=2, m=2, p=1)
    P = solve.Problem(pr)
    u, q, uh = W.random_state(pr, 31)
    ctx = pkg.Context(pr)
    ctx.assemble(_dev(u), _dev(q), _dev(uh))
    ctx.condense(shift=0.2)
    Nu, Nt = ctx.info["Nu"], ctx.info["Nt"]
    S = _dev(np.stack([ctx.get_block(0, e) for e in range(P.E)]))
    perm = _dev(np.stack([ctx.get_block(15, e) for e in range(P.E)]), torch.int32)
    C = _dev(np.stack([ctx.get_block(4, e) for e in range(P.E)]))
    B = _dev(np.stack([ctx.get_block(5, e) for e in range(P.E)]))
    D = _dev(np.stack([ctx.get_block(9, e) for e in range(P.E)]))
    gather = _dev(np.stack([P.maps[e].reshape(-1) for e in range(P.E)]), torch.int32)
    own = -np.ones((P.F, 2), dtype=np.int64)
    for f, lst in enumerate(P.mesh.face_owners()):
        for i, (e, fl) in enumerate(lst):
            own[f, i] = e * 2 * P.d + fl
    owner = _dev(own, torch.int32)
    x = _dev(W.random_vector(P.F * P.ns * P.Nfn, 77))
    y_ref = ctx.apply(x)
    stream = c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: c_void_p(t.data_ptr())
    for call in range(2):
        y = torch.full_like(x, float("nan"))
        rc = fn(P.d, P.E, P.F, Nu, P.Nfn, ptr(S), ptr(perm), ptr(B), ptr(C), ptr(D), ptr(gather), ptr(owner),
                ptr(x), ptr(y), stream)
        assert rc == 0
        torch.cuda.synchronize()
        err = (y - y_ref).abs().max().item() / y_ref.abs().max().item()
        assert err < 1e-11, (call, err)
    # sizes beyond the fixed scratch are refused before any launch
    rc = fn(P.d, 1 << 20, P.F, Nu, P.Nfn, ptr(S), ptr(perm), ptr(B), ptr(C), ptr(D), ptr(gather), ptr(owner),
            ptr(x), ptr(y), stream)
    assert rc == -8
    ctx.close()
