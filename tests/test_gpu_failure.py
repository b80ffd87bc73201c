"""Failure detection on the GPU without a fault: a bounded device-side wait of
the tensor-core product kernel is made to run out (its poll limit shortened to
a few polls, far less than the operand copies take), and the library must
report PINV_ERR_TIMEOUT, leave the context usable and give the exact result on
the next call.  The kernel's waits all have a bound; when one gives up the
kernel waits (with the normal bound) for its own copies and MMAs in flight,
releases its tensor memory and returns."""

import numpy as np
import pytest

from paper_1604_07893_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture()
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07893_gb300 import Handle
    h = Handle(0)
    yield h
    h.set_wait_limit(0)
    h.close()


def test_gemm_wait_runs_out_and_the_next_call_succeeds(handle):
    from paper_1604_07893_gb300 import PinvError
    rng = np.random.default_rng(3)
    A = torch.from_numpy(rng.standard_normal((1024, 8192))).cuda()
    B = torch.from_numpy(rng.standard_normal((8192, 640))).cuda()
    ref = handle.gemm(A, B, prec="fp64_tc").clone()
    handle.set_wait_limit(2)
    for _ in range(2):
        with pytest.raises(PinvError) as e:
            handle.gemm(A, B, prec="fp64_tc")
        assert e.value.code == -6          # PINV_ERR_TIMEOUT
    handle.set_wait_limit(0)
    got = handle.gemm(A, B, prec="fp64_tc")
    torch.cuda.synchronize()
    assert torch.equal(got, ref)           # the engine is deterministic


def test_solve_reports_timeout_then_solves(handle):
    w = W.rectangular(600, 500, None, 1.0, 1e-2, seed=8)
    A = torch.from_numpy(w.A).cuda()
    X0, info0 = handle.solve(A, alpha=1.0, tol=1e-12, prec="fp64_tc")
    handle.set_wait_limit(2)
    _, info = handle.solve(A, alpha=1.0, tol=1e-12, prec="fp64_tc", raise_on_error=False)
    assert info["status"] == -6
    handle.set_wait_limit(0)
    X1, info1 = handle.solve(A, alpha=1.0, tol=1e-12, prec="fp64_tc")
    torch.cuda.synchronize()
    assert info1["status"] == 0 and info1["iters"] == info0["iters"]
    assert torch.equal(X1, X0)
