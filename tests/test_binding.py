"""CPU checks of the Python binding's marshalling (no device calls): the
descriptor a call builds carries the caller's shapes, leading dimensions,
enum codes and flags, and malformed arguments are refused before the C ABI
is reached."""

import ctypes

import numpy as np
import pytest

from paper_1604_07893_gb300 import _lib
from paper_1604_07893_gb300._lib import FINISH, KIND, PREC, STOP, VARIANT, Desc, Handle


def host_desc(A, X, **kw):
    return Handle.make_desc(A, X, host=True, **kw)


def test_host_descriptor_fields():
    A = np.zeros((7, 5))
    X = np.zeros((5, 7))
    d = host_desc(A, X, kind="moore_penrose", alpha=0.25, tol=1e-9, stop="order18", max_iter=12,
                  prec="fp64_tc", variant="stabilized", switch_tol=0.5, finish="clean", check=True)
    assert (d.m, d.n, d.lda, d.ldx) == (7, 5, 5, 7)
    assert d.A == A.ctypes.data and d.X == X.ctypes.data and not d.G
    assert d.kind == KIND["moore_penrose"] and d.stop == STOP["order18"] and d.prec == PREC["fp64_tc"]
    assert d.variant == VARIANT["stabilized"] and d.finish == FINISH["clean"]
    assert (d.alpha, d.tol, d.max_iter, d.switch_tol) == (0.25, 1e-9, 12, 0.5)
    assert (d.host_buffers, d.check, d.profile, d.symmetric) == (1, 1, 0, 0)


def test_host_descriptor_with_g_and_complex():
    A = np.zeros((4, 3), dtype=np.complex128)
    X = np.zeros((3, 4), dtype=np.complex128)
    G = np.zeros((3, 4), dtype=np.complex128)
    d = host_desc(A, X, kind="outer_g", G=G, cplx=True)
    assert d.G == G.ctypes.data and d.ldg == 4 and d.kind == KIND["outer_g"]
    assert (d.lda, d.ldx) == (3, 4)        # leading dimensions in complex elements


def test_enum_codes_match_the_header():
    header = open(_lib.HERE + "/../include/pinv.h").read()
    for name, code in [("PINV_MOORE_PENROSE", 0), ("PINV_DRAZIN", 1), ("PINV_OUTER_G", 2),
                       ("PINV_DRAZIN_NORMAL", 3), ("PINV_STOP_ORDER18", 2), ("PINV_PREC_FP64_TC", 4),
                       ("PINV_PREC_BF16_FP32", 5), ("PINV_FINISH_CLEAN", 1), ("PINV_VARIANT_STABILIZED", 1)]:
        assert f"{name}" in header
    assert KIND == {"moore_penrose": 0, "drazin": 1, "outer_g": 2, "drazin_normal": 3}
    assert PREC["fp64_tc"] == 4 and PREC["bf16_fp32"] == 5 and STOP["order18"] == 2


@pytest.mark.parametrize("bad", ["dtype", "shape", "order", "complex_for_real"])
def test_malformed_host_arguments_are_refused(bad):
    A = np.zeros((6, 4))
    X = np.zeros((4, 6))
    if bad == "dtype":
        A = A.astype(np.float32)
    elif bad == "shape":
        X = np.zeros((6, 4))
    elif bad == "order":
        A = np.asfortranarray(np.zeros((6, 4)))
    else:
        A = A.astype(np.complex128)
    with pytest.raises((TypeError, ValueError)):
        host_desc(A, X)


def test_descriptor_layout_is_the_ctypes_struct():
    assert ctypes.sizeof(Desc) == ctypes.sizeof(_lib.Desc)
    d = host_desc(np.zeros((2, 2)), np.zeros((2, 2)))
    assert isinstance(d, Desc)
