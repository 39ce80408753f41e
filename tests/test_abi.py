"""The C ABI library loads without a GPU and exports every function include/ccpnk.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ccpnk.h")
LIB = os.path.join(ROOT, "paper_2608_06669_b300", "libccpnk.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def library():
    if not os.path.exists(LIB):
        from paper_2608_06669_b300 import build

        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("cc_residual", "cc_jvp", "cc_apply_AF", "cc_solve", "cc_serve_submit", "cc_serve_poll"):
        assert required in names


def test_every_declared_symbol_is_exported(library):
    missing = [n for n in declared_functions() if not hasattr(library, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2608_06669_b300 import ccpnk

    L = ccpnk.lib()
    for n in declared_functions():
        assert getattr(L, n).argtypes is not None, n


def test_context_creation_fails_cleanly_without_a_device():
    """No GPU in this process: the context call returns an error status instead of crashing."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2608_06669_b300 import ccpnk

    h = ctypes.c_void_p()
    st = ccpnk.lib().cc_ctx_create(ctypes.byref(h), 0, 0, None)
    assert st < 0 and not h.value


def test_default_options_follow_the_paper():
    """App. F.1: gamma = 0.9, alpha = 1.5; tolerance 1e-8 as in every experiment."""
    from paper_2608_06669_b300 import ccpnk

    o = ccpnk.default_opts("pnk", "fp64")
    assert o.gamma == 0.9 and o.alpha == 1.5 and o.tol == 1e-8 and o.eta_max == 0.9
    assert o.method == 2 and o.prec == 0 and o.m_max == 30


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-12), ("df64", 1e-12), ("tf32", 1e-6), ("tf32x3", 1e-8),
                                       ("bf16x3", 1e-7)])
def test_inner_tolerance_follows_the_precision(prec, rtol):
    """The inner A_F GMRES asks for no more than the precision of its operator delivers."""
    from paper_2608_06669_b300 import ccpnk

    o = ccpnk.default_opts("pnk", prec)
    assert o.inner_rtol == rtol and o.inner_max == 50 and o.af_direct == 0
    assert ccpnk.PREC[prec] == o.prec


def test_precision_codes_match_the_header():
    from paper_2608_06669_b300 import ccpnk

    text = open(HEADER).read()
    codes = dict(re.findall(r"(CC_(?:FP64|MIXED_TF32|MIXED_BF16X3|MIXED_TF32X3|DF64))\s*=\s*(\d+)", text))
    assert {k: int(v) for k, v in codes.items()} == {"CC_FP64": ccpnk.PREC["fp64"], "CC_MIXED_TF32": ccpnk.PREC["tf32"],
                                                     "CC_MIXED_BF16X3": ccpnk.PREC["bf16x3"],
                                                     "CC_MIXED_TF32X3": ccpnk.PREC["tf32x3"],
                                                     "CC_DF64": ccpnk.PREC["df64"]}
