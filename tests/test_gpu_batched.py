"""pinv_solve_batched: uneven independent problems solved in padded buckets,
checked per instance against the closed-form inverse, the oracle and the
single-problem entry point."""

import numpy as np
import pytest

from oracle import hyperpower as H
from paper_1604_07893_gb300 import workloads as W
from tests.helpers import pinv_closed_form, rel

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


@pytest.mark.parametrize("prec,tol_err", [("fp64", 1e-9), ("fp64_tc", 1e-9), ("mixed_bf16", 1e-9),
                                          ("fp32", 1e-9)])
def test_batched_uneven_matches_closed_form(handle, prec, tol_err):
    """The uneven batch family (m ~ U{32..512}, n ~ U{16..m}, full rank,
    singular values log-uniform in [1e-3, 1]) at 40 instances."""
    ws = W.uneven_batch(40, seed=3)
    As = [dev(w.A) for w in ws]
    alphas = [1.0 / w.s[0] ** 2 for w in ws]
    Xs = [torch.empty(w.A.shape[1], w.A.shape[0], dtype=torch.float64, device="cuda") for w in ws]
    from paper_1604_07893_gb300._lib import Desc, Info
    import ctypes as C
    descs = (Desc * len(ws))(*[handle.make_desc(A, X, alpha=a, tol=1e-12, prec=prec, finish="clean")
                               for A, X, a in zip(As, Xs, alphas)])
    infos = (Info * len(ws))()
    rc = handle._lib.pinv_solve_batched(handle._h, len(ws), descs, C.c_void_p(0), infos)
    torch.cuda.synchronize()
    assert rc == 0, [i.status for i in infos]
    for w, X, info in zip(ws, Xs, infos):
        assert info.status == 0
        assert rel(X.cpu().numpy(), pinv_closed_form(w)) <= tol_err


def test_batched_equals_single_solves_and_oracle(handle):
    ws = W.uneven_batch(12, seed=7, m_hi=300)
    As = [dev(w.A) for w in ws]
    Xs, infos = handle.solve_batched(As, alpha=0.0, tol=1e-12)
    for w, A, X, info in zip(ws, As, Xs, infos):
        assert info["status"] == 0
        X1, i1 = handle.solve(A, alpha=0.0, tol=1e-12)
        assert rel(X.cpu().numpy(), X1.cpu().numpy()) <= 1e-11
        a = H.alpha_rectangular(w.A)
        ref, _ = H.solve(w.A, H.x0_moore_penrose(w.A, a), tol=1e-12, alpha=a)
        assert rel(X.cpu().numpy(), ref) <= 1e-11
        assert info["alpha"] == pytest.approx(a, rel=1e-12)


def test_batched_rank_deficient_stabilised(handle):
    ws = [W.rectangular(m, n, r, 1.0, 1e-3, seed=i) for i, (m, n, r) in
          enumerate([(200, 150, 100), (190, 140, 90), (256, 128, 96), (130, 70, 50)])]
    As = [dev(w.A) for w in ws]
    alphas = [2.0 / (w.s[0] ** 2 + w.s[-1] ** 2) for w in ws]
    from paper_1604_07893_gb300._lib import Desc, Info
    import ctypes as C
    Xs = [torch.empty(w.A.shape[1], w.A.shape[0], dtype=torch.float64, device="cuda") for w in ws]
    descs = (Desc * len(ws))(*[handle.make_desc(A, X, alpha=a, tol=1e-12, prec="fp64_tc",
                                                variant="stabilized", finish="clean")
                               for A, X, a in zip(As, Xs, alphas)])
    infos = (Info * len(ws))()
    rc = handle._lib.pinv_solve_batched(handle._h, len(ws), descs, C.c_void_p(0), infos)
    torch.cuda.synchronize()
    assert rc == 0
    for w, X, info in zip(ws, Xs, infos):
        assert rel(X.cpu().numpy(), pinv_closed_form(w)) <= 1e-9
        assert H.penrose_residuals(w.A, X.cpu().numpy()).max() <= 1e-9


def test_batched_empty_and_single(handle):
    Xs, infos = handle.solve_batched([], alpha=0.0)
    assert Xs == [] and infos == []
    w = W.rectangular(33, 17, None, 1.0, 1e-2, seed=1)
    Xs, infos = handle.solve_batched([dev(w.A)], alpha=0.0, tol=1e-13)
    assert rel(Xs[0].cpu().numpy(), pinv_closed_form(w)) < 1e-11
