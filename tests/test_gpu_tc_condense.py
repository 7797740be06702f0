"""Tensor-core (tcgen05) condensation and LU against the FP64 CUDA path.

The FP64 path agrees with the oracle to 1e-11 (test_gpu_parity); here the mixed
path (FP32 blocks) with each tensor-core mode condenses the same blocks of a 3D
problem large enough for several 128 x 256 tiles and a ragged tail (S is
625 x 625), and its trace apply is compared with the FP64 one:

* mode 0, FP32 SIMT products: the FP32 reference level e0;
* modes 1 and 2, split TF32 (hi*hi + hi*lo + lo*hi) in the LU trailing update,
  then also the condensation and A^T_i products: the dropped lo*lo term leaves an
  operand rounding of ~2^-21 instead of FP32's 2^-24, so the error stays at the FP32
  level, below 2^-13 (three orders under plain TF32);
* mode 3, plain TF32 (10-bit mantissa) in the products: e0 scaled by the ratio of
  the unit roundoffs (2^-11 / 2^-24 = 2^13), with a factor 2 margin.
"""
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


def _apply(lib, pr, state, x, opts):
    ctx = lib.Context(pr, opts)
    ctx.assemble(*[torch.as_tensor(a, device="cuda") for a in state])
    ctx.condense(shift=0.3)
    y = ctx.apply(torch.as_tensor(x, device="cuda")).cpu().numpy()
    ctx.close()
    return y


@pytest.mark.parametrize("apply_mode", [0, 1])
def test_tensor_core_condensation_modes(lib, apply_mode):
    pr = W.mms(dim=3, nmac=2, m=2, p=2)
    state = W.random_state(pr, 5)
    z = W.sizes(pr)
    x = W.random_vector(z["F"] * z["ns"] * z["Nfn"], 9)
    y64 = _apply(lib, pr, state, x, dict(precision=0, apply_mode=apply_mode))
    scale = np.abs(y64).max()
    err = {}
    for mode in (0, 1, 2, 3):
        y = _apply(lib, pr, state, x, dict(precision=1, apply_mode=apply_mode, tc_mode=mode))
        err[mode] = np.abs(y - y64).max() / scale
    print("apply_mode", apply_mode, "relative error per tc_mode", err)
    e0 = err[0]
    assert e0 < 1e-4
    assert err[1] < 2.0 ** -13
    assert err[2] < 2.0 ** -13
    assert err[3] < 2.0 * 2.0 ** 13 * e0
