"""pinv_step_noalloc against pinv_step and the FP64 oracle, through the C ABI.

pinv_step_noalloc serves callers that cannot allocate device memory (their
host framework owns the allocator, or allocation is forbidden or would
synchronise at the wrong time): it runs the same FP64 loop with all scratch in
a static device array.  This file sorts last so that a run stopping at the
first failure has run every other test before it.  It passes alone in a fresh
process and after the other tests.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("m,n,stabilized", [(64, 48, False), (48, 64, False), (128, 100, True),
                                            (37, 128, False)])
def test_noalloc_step_matches_pinv_step_twice(m, n, stabilized):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import hyperpower as H
    from paper_1604_07893_gb300 import Handle, workloads as W
    from paper_1604_07893_gb300._lib import step_noalloc
    w = W.rectangular(m, n, None, 1.0, 1e-2, seed=m + n)
    A = torch.from_numpy(w.A).cuda()
    X = torch.from_numpy(np.ascontiguousarray(0.9 * w.A.T)).cuda()
    side = H.choose_side(m, n)
    h = Handle(0)
    for _ in range(2):           # two calls in a row: the static scratch is reused
        ref, rel_ref = h.step(A, X, stabilized=stabilized)
        got, rel_got = step_noalloc(A, X, stabilized=stabilized)
        torch.cuda.synchronize()
        diff = float((got - ref).abs().max() / ref.abs().max())
        assert diff <= 1e-12
        assert rel_got == pytest.approx(rel_ref, rel=1e-12)
        # the oracle's naive order-18 step (17 successive products), then X A X
        # for the stabilised loop
        Xh = X.cpu().numpy()
        want = (H.stabilised_step(w.A, Xh, side=side) if stabilized
                else H.hyperpower_step(w.A, Xh, side=side))
        g = got.cpu().numpy()
        assert np.linalg.norm(g - want) / np.linalg.norm(want) <= 1e-12
        assert rel_got == pytest.approx(np.linalg.norm(want - Xh) / np.linalg.norm(Xh), rel=1e-10)
        X = got
    h.close()


def test_noalloc_rejects_shapes_beyond_the_static_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07893_gb300 import PinvError
    from paper_1604_07893_gb300._lib import NOALLOC_MAX_DIM, step_noalloc
    A = torch.zeros((NOALLOC_MAX_DIM + 1, 8), dtype=torch.float64, device="cuda")
    X = torch.zeros((8, NOALLOC_MAX_DIM + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(PinvError) as e:
        step_noalloc(A, X)
    assert e.value.code == -2
