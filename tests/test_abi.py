"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point.

No compute call is made (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|long long|const char\*|mehdg_ctx\*)\s+\**(mehdg_\w+)\s*\(", src,
                                flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as ge
    ge.build()
    from paper_2402_11361_gb300 import LIB_PATH, EXPORTS
    lib = ctypes.CDLL(LIB_PATH)
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(EXPORTS) <= set(names)


def test_binding_refuses_without_gpu():
    import torch
    import paper_2402_11361_gb300 as pkg
    import workloads as W
    if torch.cuda.is_available():
        return
    try:
        pkg.Context(W.couette2d())
    except pkg.MehdgError as e:
        assert "CUDA" in str(e)
    else:
        raise AssertionError("Context must fail loudly without a GPU")
