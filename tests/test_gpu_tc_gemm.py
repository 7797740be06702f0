"""The tcgen05 TF32 batched GEMM against a plain PyTorch FP32 product of the same op.

TF32 keeps 10 mantissa bits, so entries agree to a few 1e-3 relative to the
product's scale; the error word must stay 0 (no timed-out wait)."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _fn():
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg
    lib = ctypes.CDLL(pkg.LIB_PATH)
    f = lib.mehdg_tc_gemm_tf32
    f.restype = ctypes.c_int
    L, P, F = ctypes.c_longlong, ctypes.c_void_p, ctypes.c_float
    f.argtypes = [ctypes.c_int] * 3 + [P, L, L, P, L, L, P, L, L, F, F, ctypes.c_int, ctypes.c_int, P, P]
    return f


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("M,N,K,batch,beta", [(128, 128, 32, 1, 0.0), (625, 125, 125, 3, 1.0),
                                              (750, 150, 625, 2, 1.0), (113, 77, 45, 4, 0.5),
                                              (300, 256, 200, 1, 0.0), (64, 200, 17, 2, 1.0)])
def test_tc_gemm_tf32_matches_fp32_reference(M, N, K, batch, beta, split):
    f = _fn()
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N)
    A = torch.randn(batch, M, K, device="cuda", generator=g)
    B = torch.randn(batch, K, N, device="cuda", generator=g)
    C0 = torch.randn(batch, M, N, device="cuda", generator=g)
    C = C0.clone()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    alpha = -0.75
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = f(M, N, K, P(A), K, M * K, P(B), N, K * N, P(C), N, M * N, alpha, beta, batch, split, P(err),
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    torch.backends.cuda.matmul.allow_tf32 = False
    ref = alpha * torch.bmm(A, B) + beta * C0
    scale = torch.sqrt(torch.tensor(float(K))) * max(abs(alpha), 1e-3)
    e = ((C - ref).abs().max() / scale).item()
    # TF32: ~2^-11 relative per operand, sqrt(K) growth, max over all entries; the
    # split (3xTF32) form drops the operand rounding to ~2^-21 (observed 3e-5 at K = 625, set by the
    # tensor-core FP32 accumulation)
    assert e < (1e-2 if split == 0 else 1e-4), e


@pytest.mark.parametrize("M,N,K,batch,beta", [(128, 128, 32, 1, 0.0), (750, 750, 625, 2, 1.0),
                                              (113, 77, 45, 3, 0.5), (300, 256, 200, 1, 0.0),
                                              (64, 300, 17, 2, 1.0), (129, 257, 33, 2, 1.0)])
def test_tc_gemm_nt_matches_fp64_reference(M, N, K, batch, beta):
    """The swizzled K-major tcgen05 product (split TF32: three products of the hi and lo TF32
    parts) against an FP64 product of the same FP32 inputs: the missing lo x lo term and the
    TF32 rounding of the remainders leave about 2^-21 of the operands' scale per term, and the
    FP32 accumulation over K adds rounding growing like sqrt(K): bound 8 sqrt(K) 2^-24 of the
    scale sum_k |a_ik| |b_jk|.
    Ragged M, N, K (not multiples of the 128 x BN x 32 tiles), batches and beta exercised."""
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N + K)
    A = torch.randn(batch, M, K, generator=g).float().cuda()
    Bt = torch.randn(batch, N, K, generator=g).float().cuda()
    C0 = torch.randn(batch, M, N, generator=g).float().cuda()
    C = C0.clone()
    err = pkg.tc_gemm_nt(A, Bt, C, alpha=1.5, beta=beta)
    torch.cuda.synchronize()
    assert err == 0
    ref = 1.5 * torch.bmm(A.double(), Bt.double().transpose(1, 2)) + beta * C0.double()
    scale = (A.double().abs().bmm(Bt.double().abs().transpose(1, 2))).max().item()
    e = (C.double() - ref).abs().max().item() / scale
    bound = 8 * K ** 0.5 * 2.0 ** -24
    print("tc_gemm_nt M %d N %d K %d: max error / scale %.2e (bound %.2e)" % (M, N, K, e, bound))
    assert e < bound
