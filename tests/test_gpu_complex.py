"""GPU parity of complex solves (pinv_solve_complex) against the FP64 oracle
run in complex128 (Section 1.1: the method is stated over C, X0 = alpha A^*).

The library solves the real embedding [[Re A, -Im A], [Im A, Re A]] with
half-width products; the oracle iterates on the complex matrices directly, so
the two share nothing but the generated inputs.  Tolerances are those of the
real FP64 path: 1e-12 of the largest entry where the oracle converges to
~1e-14, 1e-9 (the FP64-finished bar) on rank-deficient problems.
"""

import numpy as np
import pytest

from oracle import hyperpower as H
from paper_1604_07893_gb300 import workloads as W
from tests.helpers import drazin_closed_form, pinv_closed_form, rel, spd_inverse

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07893_gb300 import Handle
    h = Handle(0)
    yield h
    h.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy()


def assert_close(got, ref, tol):
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol * scale, np.abs(got - ref).max() / scale
    assert rel(got, ref) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_complex_mp_64x48_matches_the_oracle(handle, prec):
    """Small enough for the device-side loop (embedding 128 x 96): loop count,
    per-loop stop measures and the result agree with the complex oracle."""
    w = W.rectangular_complex(64, 48, None, 1.0, 1e-2, seed=0)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref, oinfo = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    X, info = handle.solve_complex(dev(w.A), alpha=alpha, tol=1e-12, prec=prec)
    assert info["status"] == 0 and info["iters"] == oinfo.iters
    for got, want in zip(info["history"], oinfo.history):
        if want > 1e-9:
            assert abs(got - want) <= 1e-6 * want
    assert_close(host(X), ref, 1e-12)
    assert rel(host(X), pinv_closed_form(w)) < 1e-12


@pytest.mark.parametrize("variant", ["plain", "stabilized"])
def test_complex_mp_rank_deficient_with_finish(handle, variant):
    """300 x 200 of rank 150, kappa 1e3, FP64-class tensor-core products on the
    600 x 400 embedding (host-driven loop): closed form and Penrose residuals
    (with conjugate transposes) at the FP64-finished bar."""
    w = W.rectangular_complex(300, 200, 150, 1.0, 1e-3, seed=22)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref = pinv_closed_form(w)
    X, info = handle.solve_complex(dev(w.A), alpha=alpha, tol=1e-12, prec="fp64_tc", variant=variant,
                                   finish="clean", check=True)
    assert info["status"] == 0
    assert rel(host(X), ref) < 1e-9
    assert max(info["penrose"]) < 1e-9
    oref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha,
                      variant="stabilised" if variant == "stabilized" else "plain", finish="moore_penrose")
    assert rel(host(X), oref) < 1e-9
    assert max(H.penrose_residuals(w.A, host(X))) < 1e-9


def test_complex_refinement_schedule_rank_deficient(handle):
    """The refinement schedule on a complex rank-deficient problem (kappa 1e4,
    alpha = 1/s_1^2): FP32-class loops, X A X, order-2 steps and the finish on
    the real embedding give the oracle's answer and the closed form to 1e-9."""
    w = W.rectangular_complex(300, 200, 150, 1.0, 1e-4, seed=22)
    alpha = 1.0 / w.s[0] ** 2
    X, info = handle.solve_complex(dev(w.A), alpha=alpha, tol=1e-2, stop="order18", prec="fp32_refine",
                                   variant="stabilized", switch_tol=0.9, finish="clean", check=True)
    assert info["status"] == 0
    assert info["precision"][0] == 3 and info["precision"][-1] == 6
    assert rel(host(X), pinv_closed_form(w)) < 1e-9
    assert max(info["penrose"]) < 1e-9
    oref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-2, stop=H.STOP_ORDER18, alpha=alpha,
                      finish="moore_penrose")
    assert rel(host(X), oref) < 1e-9


def test_complex_alpha_recipe_uses_complex_moduli(handle):
    w = W.rectangular_complex(40, 28, None, 1.0, 1e-2, seed=21)
    X, info = handle.solve_complex(dev(w.A), alpha=0.0, tol=1e-12)
    a = H.alpha_rectangular(w.A)
    assert abs(info["alpha"] - a) <= 1e-14 * a
    ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, a), tol=1e-12, alpha=a)
    assert_close(host(X), ref, 1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_complex_drazin_against_closed_form_and_oracle(handle, prec):
    """A = P blockdiag(C, N) P^{-1} over C, index 2, eigenvalues in the sector
    |arg| <= pi/8 (not closed under conjugation)."""
    d = W.drazin_complex(96, 24, seed=23)
    ref = drazin_closed_form(d)
    tr = H.trace(H.matpow(d.A, 3))
    alpha = 1.0 / tr.real
    oref, _ = H.solve(d.A, H.x0_drazin(d.A, 2, alpha), tol=1e-13, alpha=1.0)
    X, info = handle.solve_complex(dev(d.A), kind="drazin", drazin_index=2, alpha=alpha, tol=1e-13,
                                   prec=prec, finish="clean", check=True)
    assert info["status"] == 0
    assert rel(host(X), ref) < 1e-10
    assert rel(host(X), oref) < 1e-10
    assert max(info["drazin"]) < 1e-10
    # alpha = 0: the real part of the paper's 1/Tr(A^{l+1})
    X0, info0 = handle.solve_complex(dev(d.A), kind="drazin", drazin_index=2, alpha=0.0, tol=1e-13, prec=prec)
    assert abs(info0["alpha"] - alpha) <= 1e-12 * alpha
    assert rel(host(X0), ref) < 1e-10


def test_complex_drazin_normal_any_spectrum(handle):
    d = W.drazin_complex(96, 24, seed=24, sector=np.pi)
    X, info = handle.solve_complex(dev(d.A), kind="drazin_normal", drazin_index=2, alpha=0.0, tol=1e-2,
                                   stop="order18", prec="fp64_tc", finish="clean")
    assert info["status"] == 0
    assert rel(host(X), drazin_closed_form(d)) < 1e-10


def test_complex_inverse_with_identity_g(handle):
    s = W.hpd_complex(160, 1e-2, 1.0, seed=8)
    alpha = 2.0 / (1.0 + 1e-2)
    G = np.eye(160, dtype=np.complex128)
    ref, _ = H.solve(s.A, H.x0_general(G, alpha), tol=1e-13, alpha=alpha)
    X, info = handle.solve_complex(dev(s.A), kind="outer_g", G=dev(G), alpha=alpha, tol=1e-13, prec="fp64_tc")
    assert info["status"] == 0
    assert_close(host(X), ref, 1e-12)
    assert rel(host(X), spd_inverse(s)) < 1e-12


def test_complex_host_buffers_equal_device_buffers(handle):
    w = W.rectangular_complex(200, 120, 90, 1.0, 1e-3, seed=25)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    kw = dict(alpha=alpha, tol=1e-12, prec="fp64_tc", finish="clean")
    Xd, _ = handle.solve_complex(dev(w.A), **kw)
    Xh, info = handle.solve_complex(np.ascontiguousarray(w.A), host=True, **kw)
    assert info["status"] == 0
    assert np.array_equal(Xh, host(Xd))
    assert rel(Xh, pinv_closed_form(w)) < 1e-9
    # and a caller G on the host
    s = W.hpd_complex(64, 1e-1, 1.0, seed=9)
    G = np.eye(64, dtype=np.complex128)
    Xg, _ = handle.solve_complex(np.ascontiguousarray(s.A), host=True, kind="outer_g", G=G, alpha=1.8, tol=1e-13)
    assert rel(Xg, spd_inverse(s)) < 1e-12


def test_complex_solve_of_a_real_matrix(handle):
    """Zero imaginary parts stay exactly zero; the real part is the real solve."""
    w = W.rectangular(80, 60, None, 1.0, 1e-2, seed=3)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    Xr, _ = handle.solve(dev(w.A), alpha=alpha, tol=1e-12)
    Xc, info = handle.solve_complex(dev(w.A.astype(np.complex128)), alpha=alpha, tol=1e-12)
    Xc = host(Xc)
    assert np.abs(Xc.imag).max() == 0.0
    assert rel(Xc.real, host(Xr)) < 1e-13


def test_complex_rejects_the_symmetric_hint(handle):
    from paper_1604_07893_gb300 import PinvError
    s = W.hpd_complex(32, 1e-1, 1.0, seed=9)
    G = dev(np.eye(32, dtype=np.complex128))
    with pytest.raises(PinvError):
        handle.solve_complex(dev(s.A), kind="outer_g", G=G, alpha=1.0, symmetric=True)


@pytest.mark.parametrize("m,n,prec", [(129, 257, "fp64"), (257, 129, "fp64_tc"), (1, 1, "fp64"), (3, 7, "fp64_tc")])
def test_complex_ragged_and_both_sides(handle, m, n, prec):
    """Odd sizes (ragged tiles on the 2m x 2n embedding, half-width products of
    odd width), the right residual side (m < n) and the 1 x 1 case."""
    r = min(m, n)
    w = W.rectangular_complex(m, n, r, 1.0, 1e-2, seed=m + 7 * n)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref, oinfo = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-12, alpha=alpha)
    X, info = handle.solve_complex(dev(w.A), alpha=alpha, tol=1e-12, prec=prec)
    assert info["status"] == 0
    assert info["side"] == ("left" if m > n else "right")
    assert_close(host(X), ref, 1e-12)
    assert rel(host(X), pinv_closed_form(w)) < 1e-12


def test_complex_mixed_precision_full_rank(handle):
    """BF16 growth loops, FP32-class, then FP64-class on a full-rank complex
    problem (alpha <= 1/sigma_max^2 as the schedule requires) with the finish."""
    w = W.rectangular_complex(300, 180, None, 1.0, 1e-3, seed=26)
    X, info = handle.solve_complex(dev(w.A), alpha=1.0 / w.s[0] ** 2, tol=1e-12, prec="mixed_bf16",
                                   finish="clean", check=True)
    assert info["status"] == 0
    assert 1 in info["precision"] and 3 in info["precision"]
    assert rel(host(X), pinv_closed_form(w)) < 1e-9
    assert max(info["penrose"]) < 1e-9


def test_complex_paper_stop_rule_uses_complex_norms(handle):
    """Eq. stopreliable measures ||X_{k+1} - X_k||_F / (18^k alpha) with the
    complex Frobenius norm: each loop's measure equals the oracle's."""
    w = W.rectangular_complex(48, 36, None, 1.0, 1e-2, seed=27)
    alpha = H.alpha_pan_schreiber(w.s[0], w.s[-1])
    ref, oinfo = H.solve(w.A, H.x0_moore_penrose(w.A, alpha), tol=1e-6, stop=H.STOP_PAPER, alpha=alpha)
    X, info = handle.solve_complex(dev(w.A), alpha=alpha, tol=1e-6, stop="paper")
    assert info["iters"] == oinfo.iters
    for got, want in zip(info["history"], oinfo.history):
        if want > 1e-9:
            assert abs(got - want) <= 1e-9 * want
    assert rel(host(X), ref) < 1e-9
