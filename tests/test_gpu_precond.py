"""GPU parity of the approximate-inverse preconditioner (pinv_preconditioner;
Section 8, Example 3: loops of Eq. PM from the Jacobi X0 = diag(1/a_ii), each
followed by a chop) against the FP64 oracle, on the shifted grid operators that
stand in for the paper's sparse test matrix.

The chop is a threshold decision taken on values both sides compute to within
rounding: decisions are compared bit for bit wherever the oracle's unchopped
value is not within 1e-9 (relative) of the threshold, values to the FP64 bar
(1e-12 of the largest entry) everywhere."""

import numpy as np
import pytest

from oracle import hyperpower as H
from paper_1604_07893_gb300 import workloads as W
from tests.helpers import rel

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


def parts(x):
    return [x.real, x.imag] if np.iscomplexobj(x) else [x]


def assert_chopped_like(got, ref_chopped, ref_unchopped, eps, tol):
    scale = np.abs(ref_unchopped).max()
    for g, r, u in zip(parts(got), parts(ref_chopped), parts(ref_unchopped)):
        clear = np.abs(np.abs(u) - eps) > 1e-9 * eps
        assert np.array_equal(g[clear] == 0, r[clear] == 0)
        assert np.abs(g - r)[clear].max() <= tol * scale


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_one_loop_real_grid(handle, prec):
    A = W.grid_operator(24, seed=7, complex_=False)
    n = A.shape[0]
    ref, steps = H.preconditioner(A, loops=1)
    X, info = handle.preconditioner(dev(A), loops=1, prec=prec)
    assert info["status"] == 0 and info["iters"] == 1
    assert abs(info["history"][0] - steps[0]) <= 1e-12 * steps[0]
    X = host(X)
    assert np.abs(X - ref).max() <= 1e-12 * np.abs(ref).max()
    # I - X1 A = (I - X0 A)^18 holds for the GPU result too
    I = np.eye(n)
    L0 = I - H.x0_jacobi(A) @ A
    assert rel(I - X @ A, np.linalg.matrix_power(L0, 18)) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp64_tc"])
def test_chopped_complex_grid_841(handle, prec):
    """n = 841 complex (a 29 x 29 grid, the size of the paper's example),
    chop 1e-5 as in Example 3."""
    A = W.grid_operator(29, seed=7)
    eps = 1e-5
    unchopped, _ = H.preconditioner(A, loops=1)
    ref, _ = H.preconditioner(A, loops=1, chop_eps=eps)
    X, info = handle.preconditioner(dev(A), loops=1, chop=eps, prec=prec)
    assert info["status"] == 0
    assert_chopped_like(host(X), ref, unchopped, eps, 1e-12)
    assert np.count_nonzero(host(X)) < 0.5 * A.size


def test_two_chopped_loops_complex(handle):
    A = W.grid_operator(20, seed=9)
    ref, steps = H.preconditioner(A, loops=2, chop_eps=1e-5)
    X, info = handle.preconditioner(dev(A), loops=2, chop=1e-5, prec="fp64_tc")
    assert info["iters"] == 2
    for got, want in zip(info["history"], steps):
        assert abs(got - want) <= 1e-9 * want
    assert rel(host(X), ref) < 1e-10


def test_alpha_scales_the_jacobi_initial_value(handle):
    A = W.grid_operator(16, seed=10, complex_=False)
    ref, _ = H.preconditioner(A, loops=1, alpha=0.9)
    X, info = handle.preconditioner(dev(A), loops=1, alpha=0.9, prec="fp64")
    assert info["alpha"] == 0.9
    assert np.abs(host(X) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec,bound", [("fp32", 1e-6), ("mixed_bf16", 5e-2)])
def test_low_precision_preconditioner(handle, prec, bound):
    """A preconditioner need not be FP64-accurate: FP32-class and BF16 products
    give X1 to their unit roundoff times the growth, and X1 A stays near I."""
    A = W.grid_operator(29, seed=7)
    n = A.shape[0]
    ref, _ = H.preconditioner(A, loops=1)
    X, info = handle.preconditioner(dev(A), loops=1, prec=prec)
    X = host(X)
    assert rel(X, ref) < bound
    assert np.linalg.norm(np.eye(n) - X @ A) / np.sqrt(n) < 0.1


def test_host_buffers_equal_device_buffers(handle):
    A = W.grid_operator(12, seed=11)
    Xd, _ = handle.preconditioner(dev(A), loops=2, chop=1e-5, prec="fp64_tc")
    Xh, info = handle.preconditioner(np.ascontiguousarray(A), loops=2, chop=1e-5, prec="fp64_tc", host=True)
    assert info["status"] == 0
    assert np.array_equal(Xh, host(Xd))


def test_zero_diagonal_is_rejected(handle):
    from paper_1604_07893_gb300 import PinvError
    A = W.grid_operator(6, seed=12, complex_=False)
    A[3, 3] = 0.0
    with pytest.raises(PinvError):
        handle.preconditioner(dev(A), loops=1)
    Z = W.grid_operator(6, seed=12)
    Z[5, 5] = 0.0
    with pytest.raises(PinvError):
        handle.preconditioner(dev(Z), loops=1)


def test_bad_requests_are_rejected_before_any_work(handle):
    from paper_1604_07893_gb300 import PinvError
    A = dev(W.grid_operator(6, seed=12, complex_=False))
    for kw in (dict(loops=0), dict(loops=129), dict(chop=-1.0), dict(alpha=float("nan")), dict(prec="mixed_fp8")):
        with pytest.raises(PinvError):
            handle.preconditioner(A, **{"loops": 1, **kw})
    with pytest.raises(ValueError):
        handle.preconditioner(dev(np.zeros((4, 5))))
